// api.cu -- the C ABI declared in include/mms.h: argument checks, the planner
// (base-case tile and per-round fanout, Sec. 6.2), the workspace layout, and
// the launch sequence of one sort: base case, then for every merge round the
// splitter and the merge pass, ping-ponging between the caller's buffer and
// the workspace copy so that the last round lands in the caller's buffer.
// The splitters and merge passes are launched with programmatic stream
// serialization, each right behind one of this library's kernels.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include "../../include/mms.h"
#include "mms_kernels.cuh"
#include "merge_pipelined.cuh"

namespace {

thread_local char g_detail[256] = "";

mms_status fail(mms_status s, const char* fmt, const char* what = "") {
  snprintf(g_detail, sizeof g_detail, fmt, what);
  return s;
}

mms_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_detail, sizeof g_detail, "%s: %s", where, cudaGetErrorString(e));
  return MMS_ERR_CUDA;
}

int key_bytes_of(mms_key_type kt) { return kt == MMS_KEY_U64 ? 8 : 4; }
bool valid_kt(int kt) { return kt == MMS_KEY_U32 || kt == MMS_KEY_U64 || kt == MMS_KEY_F32; }
bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
// Key and value arrays need only their element's alignment; the kernels take
// their vectorised paths on the parts that lie on the 16-byte grid.
bool aligned_to(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

constexpr size_t kStatusBytes = 256;
size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct WsLayout {
  size_t keys_off, vals_off, table_off, total;
  size_t comp0_off, comp1_off;   // key-value sort: the two 64-bit composite buffers
  // key-value sort of 8-byte keys: a 4-byte half of every key, the position
  // list of the two passes, and copies of the keys and values
  size_t half_off, perm_off, kcopy_off, vcopy_off;
};

// Key-only sort: status | ping-pong copy of the keys | pivot table.
// Key-value sort (4-byte keys): status | composites 0 | composites 1 | copy of
// the values | pivot table (the rounds run on 8-byte composites).
WsLayout ws_layout(mms_key_type kt, size_t n, int with_values) {
  WsLayout L{};
  const size_t kb = (size_t)key_bytes_of(kt);
  if (!with_values) {
    const size_t S = (kb == 8 ? 2048 : 4096);      // smallest tile a sort may use
    L.keys_off = kStatusBytes;
    L.vals_off = round_up(L.keys_off + n * kb, 256);
    L.table_off = L.vals_off;
    const size_t rows = (n + S - 1) / S + 1;
    L.total = round_up(L.table_off + rows * mms::kMaxFanout * sizeof(long long), 256);
    return L;
  }
  L.comp0_off = kStatusBytes;
  L.comp1_off = round_up(L.comp0_off + n * 8, 256);
  L.vals_off = round_up(L.comp1_off + n * 8, 256);
  L.table_off = round_up(L.vals_off + n * 4, 256);
  L.keys_off = L.comp0_off;
  const size_t rows = (n + 2047) / 2048 + 1;
  L.total = round_up(L.table_off + rows * mms::kMaxFanout * sizeof(long long), 256);
  if (kt == MMS_KEY_U64) {
    L.half_off = L.total;
    L.perm_off = round_up(L.half_off + n * 4, 256);
    L.kcopy_off = round_up(L.perm_off + n * 4, 256);
    L.vcopy_off = round_up(L.kcopy_off + n * 8, 256);
    L.total = round_up(L.vcopy_off + n * 4, 256);
  }
  return L;
}

// Tile width (warps per CTA, 1024 items each) a sort uses.
int tile_warps_for(int key_bytes, const mms_options* opt) {
  if (opt && opt->tile_items > 0) return opt->tile_items / 1024;
  return mms::default_tile_warps(key_bytes);
}

// Length of the sorted runs the base case of a keys-only sort produces: one
// CTA tile by default, or the caller's mms_options.base_items (for 4-byte keys
// also one thread-block cluster of 2, 4 or 8 tiles per run).  Runs of one tile
// are the default because on GB300 a cluster merge level (co-ranks and copies
// through distributed shared memory between two cluster barriers) measured
// dearer than the merge-round level it saves: 10^8 u32 keys sorted at 37.1
// Gkeys/s from runs of 8192, 36.5 / 35.0 / 33.7 from runs of 16384 / 32768 /
// 65536 (base case 0.605 -> 0.779 / 0.995 / 1.309 ms).
long long base_run_items(int key_bytes, size_t n, const mms_options* opt) {
  (void)n;
  const long long T = 1024ll * tile_warps_for(key_bytes, opt);
  if (opt && opt->base_items > 0) return opt->base_items;
  return T;
}

// Whether base_items is a run length the keys-only base case can produce.
bool valid_base_items(int key_bytes, int tw, int base_items) {
  if (base_items == 0 || base_items == 1024 * tw) return true;
  if (key_bytes != 4 || tw != mms::default_tile_warps(4)) return false;
  return base_items == 2 * 1024 * tw || base_items == 4 * 1024 * tw || base_items == 8 * 1024 * tw;
}

// Fanouts of the merge rounds.  Sec. 6.2 tunes K per platform by
// measurement; here the planner picks, per sort, the sequence of power-of-two
// fanouts that minimises a cost model measured on GB300.  A round of fanout K
// over n items costs about c0 + n * c1[K], where c1 is the merge pass plus
// splitter time per item at n = 10^8 over the rounds that merged K runs per
// group (bench.py --workload sweep, fitted by autotune.fit_plan_costs) and c0
// the fixed cost of its two launches.  A last round over fewer runs builds
// its tree over those runs only, so it costs what a round of the next power
// of two does.  Merge levels cost about the same for
// K = 4..16, so the optimum first minimises the tree levels ceil(log2 runs)
// and then the rounds (e.g. (16,16,8,8) for 10^8 4-byte keys).  The choice is
// a coin-change dynamic program over log2 of the coverage.  opt->fanout fixes
// every round's K instead; the result does not depend on the plan.
namespace plan_model {
// ms per 10^8 items of one round (merge pass + splitter), for K = 2, 4, 8, 16, 32
constexpr double kCost4[5] = {0.221, 0.332, 0.465, 0.621, 1.001};   // 4-byte keys
constexpr double kCost8[5] = {0.466, 0.727, 1.035, 1.566, 2.873};   // 8-byte keys / composites
constexpr double kLaunchMs = 0.010;                                 // two launches per round
}  // namespace plan_model

int plan_rounds(int key_bytes, size_t n, const mms_options* opt, int* K, int maxr) {
  const long long S = base_run_items(key_bytes, n, opt);
  const long long runs = ((long long)n + S - 1) / S;
  if (runs <= 1) return 0;
  if (opt && opt->fanout >= 2) {
    const int fanout = opt->fanout;
    int rounds = 0;
    long long cover = 1;
    while (cover < runs) {
      cover *= fanout;
      if (rounds < maxr) K[rounds] = fanout;
      ++rounds;
    }
    return rounds;
  }
  int L = 0;                                   // levels needed: 2^L >= runs
  while ((1ll << L) < runs) ++L;
  const double* c1 = key_bytes == 8 ? plan_model::kCost8 : plan_model::kCost4;
  const double scale = (double)n / 1e8;
  // best[l]: least cost of rounds covering at least 2^l; pick[l]: log2 of its first fanout
  double best[64];
  int pick[64];
  best[0] = 0.0;
  pick[0] = 0;
  for (int l = 1; l <= L; ++l) {
    best[l] = 1e300;
    pick[l] = 1;
    for (int b = 1; b <= 5; ++b) {
      const int rest = l - b > 0 ? l - b : 0;
      const double c = best[rest] + plan_model::kLaunchMs + scale * c1[b - 1];
      if (c < best[l]) {
        best[l] = c;
        pick[l] = b;
      }
    }
  }
  int rounds = 0;
  for (int l = L; l > 0;) {
    const int b = pick[l];
    if (rounds < maxr) K[rounds] = 1 << b;
    ++rounds;
    l = l - b > 0 ? l - b : 0;
  }
  // larger fanouts first (the cost model does not depend on the order)
  const int m = rounds < maxr ? rounds : maxr;
  for (int a = 0; a < m; ++a)
    for (int c = a + 1; c < m; ++c)
      if (K[c] > K[a]) {
        const int t = K[a];
        K[a] = K[c];
        K[c] = t;
      }
  return rounds;
}

// Output tile of the merge rounds (a multiple of 1024, at most the base-case
// tile T).  The default is T.  A smaller tile can keep every tree level within
// one block per warp (with K = 4 on 8 warps an 8192-item tile's first level
// has 9 blocks in general, a 7168-item tile's at most 8), but on GB300 the
// extra tiles cost more than that saves (10^8 u32, K = 4: 0.325 ms per pass
// at 7168 against 0.313 ms at 8192, splitters 0.54 ms against 0.47 ms); the
// caller's mms_options.merge_tile_items selects one.  The workspace's pivot
// table holds n / S_min + 1 rows; a tile that would need more falls back to T.
long long merge_tile_for(int key_bytes, int tw, int K, const mms_options* opt, size_t n,
                         long long run_len) {
  const long long T = 1024ll * tw;
  long long S = T;
  if (opt && opt->merge_tile_items > 0) S = opt->merge_tile_items;
  const long long S_min = key_bytes == 8 ? 2048 : 4096;
  const long long cap = ((long long)n + S_min - 1) / S_min + 1;
  if (mms::num_tiles(S, (long long)n, run_len, K) + 1 > cap) S = T;
  return S;
}

mms_status check_launch(cudaError_t e, const char* where) {
  return e == cudaSuccess ? MMS_OK : cuda_fail(e, where);
}

// Status of the sorts whose workspace the library allocated: before the
// workspace is freed, its status word is forwarded here (the first error
// since the last mms_stream_status wins).  One word per device.
__device__ int g_stream_status;

__global__ void forward_status_kernel(const int* __restrict__ ws_status) {
  const int w = *ws_status;
  if (w != 0) atomicCAS(&g_stream_status, 0, w);
}

// Allocates a workspace stream-ordered and clears its status word.
mms_status alloc_workspace(void** d_ws, size_t bytes, cudaStream_t s) {
  cudaError_t e = cudaMallocAsync(d_ws, bytes, s);
  if (e != cudaSuccess) return fail(MMS_ERR_NO_MEMORY, "cudaMallocAsync of the workspace failed%s");
  e = cudaMemsetAsync(*d_ws, 0, kStatusBytes, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(*d_ws, s);
    return cuda_fail(e, "workspace init");
  }
  return MMS_OK;
}

// Ends a sort on a library-allocated workspace without waiting for it: the
// status word goes to the per-device word, then the workspace is freed, both
// in stream order.
mms_status release_workspace(void* d_ws, cudaStream_t s, mms_status st) {
  forward_status_kernel<<<1, 1, 0, s>>>(static_cast<const int*>(d_ws));
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(d_ws, s);
  if (st == MMS_OK && e1 != cudaSuccess) st = cuda_fail(e1, "status forwarding");
  if (st == MMS_OK && e2 != cudaSuccess) st = cuda_fail(e2, "workspace release");
  return st;
}

// Clears the status word of a caller's workspace on the stream, so that a
// stale or uninitialised word never reads as this call's error.
mms_status clear_status(void* d_ws, cudaStream_t s) {
  const cudaError_t e = cudaMemsetAsync(d_ws, 0, sizeof(int), s);
  return e == cudaSuccess ? MMS_OK : cuda_fail(e, "status word");
}

mms_status status_of_word(int word) {
  if (word == mms::kDevErrTimeout) return fail(MMS_ERR_TIMEOUT, "a device wait timed out%s");
  if (word != 0) return fail(MMS_ERR_INTERNAL, "device consistency check failed%s");
  return MMS_OK;
}

}  // namespace

namespace mms {
void set_error_detail(const char* msg) { snprintf(g_detail, sizeof g_detail, "%s", msg); }
}  // namespace mms

extern "C" {

const char* mms_status_string(mms_status s) {
  switch (s) {
    case MMS_OK: return "ok";
    case MMS_ERR_INVALID_ARG: return "invalid argument";
    case MMS_ERR_UNSUPPORTED: return "unsupported";
    case MMS_ERR_NO_MEMORY: return "out of memory / workspace too small";
    case MMS_ERR_CUDA: return "CUDA error";
    case MMS_ERR_TIMEOUT: return "device-side wait timed out";
    case MMS_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

mms_status mms_last_error_detail(char* buf, size_t len) {
  if (!buf || len == 0) return MMS_ERR_INVALID_ARG;
  snprintf(buf, len, "%s", g_detail);
  return MMS_OK;
}

size_t mms_tile_items(mms_key_type kt) {
  return valid_kt(kt) ? (size_t)1024 * mms::default_tile_warps(key_bytes_of(kt)) : 0;
}

size_t mms_base_run_items(mms_key_type kt, size_t n, const mms_options* opt) {
  if (!valid_kt(kt)) return 0;
  const int kb = key_bytes_of(kt);
  if (opt && (opt->tile_items != 0 && !mms::valid_tile_warps(kb, opt->tile_items / 1024)))
    return 0;
  if (opt && !valid_base_items(kb, tile_warps_for(kb, opt), opt->base_items)) return 0;
  return (size_t)base_run_items(kb, n, opt);
}

size_t mms_sort_workspace_bytes(mms_key_type kt, size_t n, int with_values) {
  if (!valid_kt(kt)) return 0;
  return ws_layout(kt, n, with_values).total;
}

int mms_plan(mms_key_type kt, size_t n, const mms_options* opt, int* fanouts, int max_rounds) {
  if (!valid_kt(kt)) return -1;
  int K[64];
  const int r = plan_rounds(key_bytes_of(kt), n, opt, K, 64);
  for (int i = 0; i < r && i < max_rounds && fanouts; ++i) fanouts[i] = K[i];
  return r;
}

mms_status mms_workspace_status(void* d_ws, size_t ws_bytes, void* stream) {
  if (!d_ws || ws_bytes < kStatusBytes) return fail(MMS_ERR_INVALID_ARG, "workspace missing%s");
  cudaStream_t s = (cudaStream_t)stream;
  int word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, d_ws, sizeof word, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && word != 0) e = cudaMemsetAsync(d_ws, 0, sizeof word, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mms_workspace_status");
  return status_of_word(word);
}

mms_status mms_stream_status(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int word = 0;
  const int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&word, g_stream_status, sizeof word, 0,
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && word != 0)
    e = cudaMemcpyToSymbolAsync(g_stream_status, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mms_stream_status");
  return status_of_word(word);
}

mms_status mms_sort_keys_ex(mms_key_type kt, void* d_keys, size_t n, void* d_ws, size_t ws_bytes,
                            void* stream, const mms_options* opt) {
  if (!valid_kt(kt)) return fail(MMS_ERR_INVALID_ARG, "unknown key type%s");
  if (n <= 1) return MMS_OK;
  if (!d_keys || !aligned_to(d_keys, (size_t)key_bytes_of(kt)))
    return fail(MMS_ERR_INVALID_ARG, "keys pointer null or not aligned to the key size%s");
  if (opt && (opt->test_flags & ~MMS_TEST_STAGING_TIMEOUT))
    return fail(MMS_ERR_INVALID_ARG, "unknown test flag%s");
  if (opt && opt->fanout != 0 && (opt->fanout < 2 || opt->fanout > mms::kMaxFanout))
    return fail(MMS_ERR_INVALID_ARG, "fanout must be 0 or in 2..32%s");
  const int kb = key_bytes_of(kt);
  if (opt && opt->tile_items != 0 &&
      (opt->tile_items % 1024 != 0 || !mms::valid_tile_warps(kb, opt->tile_items / 1024)))
    return fail(MMS_ERR_INVALID_ARG, "tile_items must be 0, 4096/8192 (4-byte keys) or 2048/4096 (8-byte keys)%s");
  const int tw = tile_warps_for(kb, opt);
  const long long S = 1024ll * tw;
  if (opt && !valid_base_items(kb, tw, opt->base_items))
    return fail(MMS_ERR_INVALID_ARG, "base_items must be 0, tile_items, or 2, 4 or 8 times the 8192-key tile (4-byte keys)%s");
  if (opt && opt->merge_tile_items != 0 &&
      (opt->merge_tile_items % 1024 != 0 || opt->merge_tile_items < (kb == 8 ? 2048 : 4096) ||
       opt->merge_tile_items > S))
    return fail(MMS_ERR_INVALID_ARG, "merge_tile_items must be 0 or a multiple of 1024 from the smallest tile up to tile_items%s");
  const int variant = opt ? opt->merge_variant : MMS_MERGE_TREE;
  if (variant != MMS_MERGE_TREE && variant != MMS_MERGE_PARTITION && variant != MMS_MERGE_PIPELINED)
    return fail(MMS_ERR_INVALID_ARG, "merge_variant must be MMS_MERGE_TREE, MMS_MERGE_PARTITION or MMS_MERGE_PIPELINED%s");
  const bool partition = variant == MMS_MERGE_PARTITION;
  const bool pipelined = variant == MMS_MERGE_PIPELINED;
  if ((partition || pipelined) && (opt->tile_items != 0 || opt->merge_tile_items != 0 || opt->test_flags != 0))
    return fail(MMS_ERR_INVALID_ARG, "the partition and pipelined merge variants take the default tile geometry (tile_items and merge_tile_items 0) and no test flags%s");
  const WsLayout L = ws_layout(kt, n, 0);
  cudaStream_t s = (cudaStream_t)stream;
  bool owned = false;
  if (d_ws) {
    if (!aligned16(d_ws)) return fail(MMS_ERR_INVALID_ARG, "workspace not 16-byte aligned%s");
    if (ws_bytes < L.total) return fail(MMS_ERR_NO_MEMORY, "workspace smaller than mms_sort_workspace_bytes()%s");
    const mms_status cs = clear_status(d_ws, s);
    if (cs != MMS_OK) return cs;
  } else {
    const mms_status as = alloc_workspace(&d_ws, L.total, s);
    if (as != MMS_OK) return as;
    owned = true;
  }
  unsigned char* ws = static_cast<unsigned char*>(d_ws);
  int* dev_err = reinterpret_cast<int*>(ws);
  const bool test_timeout = opt && (opt->test_flags & MMS_TEST_STAGING_TIMEOUT);
  void* tmp = ws + L.keys_off;
  long long* table = reinterpret_cast<long long*>(ws + L.table_off);

  int K[64];
  const int rounds = plan_rounds(kb, n, opt, K, 64);
  const bool is_f32 = kt == MMS_KEY_F32;
  mms_status st = MMS_OK;
  // Base case writes to the caller's buffer when an even number of rounds follows.
  void* cur = (rounds % 2 == 1) ? tmp : d_keys;
  void* other = (cur == tmp) ? d_keys : tmp;
  int ev = 0;
  auto mark = [&]() {
    if (opt && opt->events && ev < opt->num_events && opt->events[ev])
      cudaEventRecord((cudaEvent_t)opt->events[ev], s);
    ++ev;
  };
  mark();
  // The base case: one CTA per tile, or one thread-block cluster per run of
  // several tiles.
  long long run_len = base_run_items(kb, n, opt);
  st = check_launch(run_len == S
                        ? mms::launch_tile_sort(kb, tw, is_f32, is_f32 && rounds == 0, d_keys, cur,
                                                (long long)n, s)
                        : mms::launch_tile_sort_cluster((int)(run_len / S), is_f32,
                                                        is_f32 && rounds == 0, d_keys, cur,
                                                        (long long)n, s),
                    "tile_sort");
  mark();
  for (int r = 0; r < rounds && st == MMS_OK; ++r) {
    const long long Sm = merge_tile_for(kb, tw, K[r], opt, n, run_len);
    st = check_launch(mms::launch_splitter(kb, Sm, cur, (long long)n, run_len, K[r], table, s, true),
                      "splitter");
    mark();
    if (st != MMS_OK) break;
    st = check_launch(pipelined
                          ? mms::launch_merge_pipelined(kb, is_f32 && r == rounds - 1, cur, other,
                                                        (long long)n, run_len, K[r], table, dev_err,
                                                        s, true)
                          : mms::launch_merge_pass(kb, tw, Sm, is_f32 && r == rounds - 1, cur, other,
                                                   (long long)n, run_len, K[r], table, dev_err, s,
                                                   test_timeout, true, partition),
                      "merge_pass");
    mark();
    void* t = cur;
    cur = other;
    other = t;
    run_len *= K[r];
  }
  if (owned) st = release_workspace(d_ws, s, st);
  return st;
}

mms_status mms_sort_keys(mms_key_type kt, void* d_keys, size_t n, void* d_ws, size_t ws_bytes,
                         void* stream) {
  return mms_sort_keys_ex(kt, d_keys, n, d_ws, ws_bytes, stream, nullptr);
}

// The 4-byte key-value sort on the composite buffers of layout L (the values
// are copied first, so d_keys / d_values are overwritten only by the last
// kernel): composite base case, merge rounds, key write-back and value gather.
static mms_status pairs32_run(bool is_f32, void* d_keys, uint32_t* d_values, size_t n,
                              unsigned char* ws, const WsLayout& L, cudaStream_t s,
                              const mms_options* opt, int& ev) {
  int* dev_err = reinterpret_cast<int*>(ws);
  void* comp[2] = {ws + L.comp0_off, ws + L.comp1_off};
  void* vcopy = ws + L.vals_off;
  long long* table = reinterpret_cast<long long*>(ws + L.table_off);

  // The rounds run on 8-byte composites with the 8-byte tile geometry.
  mms_options o8{};
  if (opt) o8 = *opt;
  const int tw = (opt && opt->tile_items) ? opt->tile_items / 1024 : mms::default_tile_warps(8);
  o8.tile_items = 1024 * tw;
  o8.base_items = 0;                    // one CTA per composite tile
  const long long S = 1024ll * tw;
  int K[64];
  const int rounds = plan_rounds(8, n, &o8, K, 64);

  auto mark = [&]() {
    if (opt && opt->events && ev < opt->num_events && opt->events[ev])
      cudaEventRecord((cudaEvent_t)opt->events[ev], s);
    ++ev;
  };
  mms_status st = MMS_OK;
  mark();
  cudaError_t ce = cudaMemcpyAsync(vcopy, d_values, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  if (ce != cudaSuccess) st = cuda_fail(ce, "copy of the values");
  if (st == MMS_OK)
    st = check_launch(mms::launch_tile_sort_composite(tw, is_f32, d_keys, comp[0], (long long)n, s),
                      "tile_sort (key-value)");
  mark();
  long long run_len = S;
  int cur = 0;
  for (int r = 0; r < rounds && st == MMS_OK; ++r) {
    st = check_launch(mms::launch_splitter(8, S, comp[cur], (long long)n, run_len, K[r], table, s, true),
                      "splitter");
    mark();
    if (st != MMS_OK) break;
    st = check_launch(opt && opt->merge_variant == MMS_MERGE_PIPELINED
                          ? mms::launch_merge_pipelined(8, false, comp[cur], comp[1 - cur],
                                                        (long long)n, run_len, K[r], table, dev_err,
                                                        s, true)
                          : mms::launch_merge_pass(8, tw, S, false, comp[cur], comp[1 - cur],
                                                   (long long)n, run_len, K[r], table, dev_err, s,
                                                   false, true,
                                                   opt && opt->merge_variant == MMS_MERGE_PARTITION),
                      "merge_pass");
    mark();
    cur = 1 - cur;
    run_len *= K[r];
  }
  if (st == MMS_OK)
    st = check_launch(mms::launch_pairs_finalize(is_f32, comp[cur], vcopy, d_keys, d_values,
                                                 (long long)n, s), "pairs_finalize");
  mark();
  return st;
}

mms_status mms_sort_pairs_ex(mms_key_type kt, void* d_keys, uint32_t* d_values, size_t n,
                             void* d_ws, size_t ws_bytes, void* stream, const mms_options* opt) {
  if (!valid_kt(kt)) return fail(MMS_ERR_INVALID_ARG, "unknown key type%s");
  if (n <= 1) return MMS_OK;
  if (n > 0xFFFFFFFEull) return fail(MMS_ERR_UNSUPPORTED, "key-value sorting takes fewer than 2^32 items%s");
  if (!d_keys || !d_values || !aligned_to(d_keys, (size_t)key_bytes_of(kt)) ||
      !aligned_to(d_values, sizeof(uint32_t)))
    return fail(MMS_ERR_INVALID_ARG, "keys/values pointer null or not aligned to the element size%s");
  if (opt && opt->fanout != 0 && (opt->fanout < 2 || opt->fanout > mms::kMaxFanout))
    return fail(MMS_ERR_INVALID_ARG, "fanout must be 0 or in 2..32%s");
  if (opt && opt->tile_items != 0 && opt->tile_items != 2048 && opt->tile_items != 4096)
    return fail(MMS_ERR_INVALID_ARG, "tile_items of a key-value sort must be 0, 2048 or 4096%s");
  if (opt && opt->test_flags != 0) return fail(MMS_ERR_INVALID_ARG, "test flags apply to mms_sort_keys_ex only%s");
  if (opt && opt->base_items != 0 && opt->base_items != (opt->tile_items ? opt->tile_items : 4096))
    return fail(MMS_ERR_INVALID_ARG, "base_items of a key-value sort must be 0 or its composite tile%s");
  if (opt && opt->merge_variant != MMS_MERGE_TREE && opt->merge_variant != MMS_MERGE_PARTITION &&
      opt->merge_variant != MMS_MERGE_PIPELINED)
    return fail(MMS_ERR_INVALID_ARG, "merge_variant must be MMS_MERGE_TREE, MMS_MERGE_PARTITION or MMS_MERGE_PIPELINED%s");
  if (opt && opt->merge_variant != MMS_MERGE_TREE && opt->tile_items != 0)
    return fail(MMS_ERR_INVALID_ARG, "the partition and pipelined merge variants take the default tile geometry (tile_items 0)%s");
  const WsLayout L = ws_layout(kt, n, 1);
  cudaStream_t s = (cudaStream_t)stream;
  bool owned = false;
  if (d_ws) {
    if (!aligned16(d_ws)) return fail(MMS_ERR_INVALID_ARG, "workspace not 16-byte aligned%s");
    if (ws_bytes < L.total) return fail(MMS_ERR_NO_MEMORY, "workspace smaller than mms_sort_workspace_bytes()%s");
    const mms_status cs = clear_status(d_ws, s);
    if (cs != MMS_OK) return cs;
  } else {
    const mms_status as = alloc_workspace(&d_ws, L.total, s);
    if (as != MMS_OK) return as;
    owned = true;
  }
  unsigned char* ws = static_cast<unsigned char*>(d_ws);
  int* dev_err = reinterpret_cast<int*>(ws);
  int ev = 0;
  mms_status st = MMS_OK;
  if (kt != MMS_KEY_U64) {
    st = pairs32_run(kt == MMS_KEY_F32, d_keys, d_values, n, ws, L, s, opt, ev);
  } else {
    // Two stable 4-byte passes, low half first (see pairs.cu).
    void* half = ws + L.half_off;
    void* perm = ws + L.perm_off;
    void* kcopy = ws + L.kcopy_off;
    void* vcopy = ws + L.vcopy_off;
    st = check_launch(mms::launch_u64_pairs_split(d_keys, d_values, half, perm, kcopy, vcopy,
                                                  (long long)n, s), "key-value split (8-byte keys)");
    if (st == MMS_OK)
      st = pairs32_run(false, half, static_cast<uint32_t*>(perm), n, ws, L, s, opt, ev);
    if (st == MMS_OK)
      st = check_launch(mms::launch_u64_pairs_hi(kcopy, perm, half, (long long)n, s),
                        "key-value high halves (8-byte keys)");
    if (st == MMS_OK)
      st = pairs32_run(false, half, static_cast<uint32_t*>(perm), n, ws, L, s, opt, ev);
    if (st == MMS_OK)
      st = check_launch(mms::launch_u64_pairs_final(kcopy, vcopy, perm, d_keys, d_values,
                                                    (long long)n, s),
                        "key-value permutation (8-byte keys)");
  }
  if (owned) st = release_workspace(d_ws, s, st);
  return st;
}

mms_status mms_sort_pairs(mms_key_type kt, void* d_keys, uint32_t* d_values, size_t n, void* d_ws,
                          size_t ws_bytes, void* stream) {
  return mms_sort_pairs_ex(kt, d_keys, d_values, n, d_ws, ws_bytes, stream, nullptr);
}

mms_status mms_tile_sort(mms_key_type kt, const void* d_in, void* d_out, size_t n, void* stream) {
  if (!valid_kt(kt)) return fail(MMS_ERR_INVALID_ARG, "unknown key type%s");
  if (n == 0) return MMS_OK;
  const int kb = key_bytes_of(kt);
  if (!d_in || !d_out || !aligned_to(d_in, (size_t)kb) || !aligned_to(d_out, (size_t)kb))
    return fail(MMS_ERR_INVALID_ARG, "buffers null or not aligned to the key size%s");
  const bool f = kt == MMS_KEY_F32;
  return check_launch(mms::launch_tile_sort(kb, mms::default_tile_warps(kb), f, f, d_in, d_out, (long long)n,
                                            (cudaStream_t)stream), "tile_sort");
}

size_t mms_splitter_rows(mms_key_type kt, size_t n, size_t run_len, int K) {
  if (!valid_kt(kt) || K < 2 || run_len == 0) return 0;
  const long long S = 1024ll * mms::default_tile_warps(key_bytes_of(kt));
  if (run_len % S != 0) return 0;
  return (size_t)mms::num_tiles(S, (long long)n, (long long)run_len, K);
}

static mms_status check_round_args(mms_key_type kt, size_t run_len, int K) {
  if (kt != MMS_KEY_U32 && kt != MMS_KEY_U64)
    return fail(MMS_ERR_UNSUPPORTED, "merge-round steps take integer keys only%s");
  if (K < 2 || K > mms::kMaxFanout) return fail(MMS_ERR_INVALID_ARG, "K must be in 2..32%s");
  const size_t S = (size_t)1024 * mms::default_tile_warps(key_bytes_of(kt));
  if (run_len == 0 || run_len % S != 0)
    return fail(MMS_ERR_INVALID_ARG, "run_len must be a positive multiple of the tile size%s");
  return MMS_OK;
}

mms_status mms_splitter(mms_key_type kt, const void* d_in, size_t n, size_t run_len, int K,
                        int64_t* d_table, void* stream) {
  mms_status st = check_round_args(kt, run_len, K);
  if (st != MMS_OK) return st;
  if (n == 0) return MMS_OK;
  const int kb = key_bytes_of(kt);
  if (!d_in || !d_table || !aligned_to(d_in, (size_t)kb) || !aligned_to(d_table, sizeof(int64_t)))
    return fail(MMS_ERR_INVALID_ARG, "null or misaligned buffer%s");
  return check_launch(mms::launch_splitter(kb, 1024ll * mms::default_tile_warps(kb), d_in, (long long)n,
                                           (long long)run_len,
                                           K, reinterpret_cast<long long*>(d_table),
                                           (cudaStream_t)stream), "splitter");
}

static mms_status merge_pass_entry(mms_key_type kt, const void* d_in, void* d_out, size_t n,
                                   size_t run_len, int K, const int64_t* d_table, void* d_ws,
                                   size_t ws_bytes, void* stream, int variant) {
  mms_status st = check_round_args(kt, run_len, K);
  if (st != MMS_OK) return st;
  if (n == 0) return MMS_OK;
  const size_t kb = (size_t)key_bytes_of(kt);
  if (!d_in || !d_out || !d_table || !aligned_to(d_in, kb) || !aligned_to(d_out, kb) ||
      !aligned_to(d_table, sizeof(int64_t)))
    return fail(MMS_ERR_INVALID_ARG, "null or misaligned buffer%s");
  const char* a = static_cast<const char*>(d_in);
  const char* b = static_cast<const char*>(d_out);
  if (a < b + n * kb && b < a + n * kb) return fail(MMS_ERR_INVALID_ARG, "input and output overlap%s");
  if (d_ws && (ws_bytes < kStatusBytes || !aligned16(d_ws)))
    return fail(MMS_ERR_INVALID_ARG, "workspace too small or not 16-byte aligned%s");
  int* dev_err = d_ws ? static_cast<int*>(d_ws) : nullptr;
  if (variant == MMS_MERGE_PIPELINED)
    return check_launch(mms::launch_merge_pipelined((int)kb, false, d_in, d_out, (long long)n,
                                                    (long long)run_len, K,
                                                    reinterpret_cast<const long long*>(d_table),
                                                    dev_err, (cudaStream_t)stream, false),
                        "merge_pass");
  return check_launch(mms::launch_merge_pass((int)kb, mms::default_tile_warps((int)kb),
                                             1024ll * mms::default_tile_warps((int)kb), false, d_in,
                                             d_out, (long long)n,
                                             (long long)run_len, K,
                                             reinterpret_cast<const long long*>(d_table), dev_err,
                                             (cudaStream_t)stream, false, false,
                                             variant == MMS_MERGE_PARTITION),
                      "merge_pass");
}

mms_status mms_merge_pass(mms_key_type kt, const void* d_in, void* d_out, size_t n,
                          size_t run_len, int K, const int64_t* d_table, void* d_ws,
                          size_t ws_bytes, void* stream) {
  return merge_pass_entry(kt, d_in, d_out, n, run_len, K, d_table, d_ws, ws_bytes, stream,
                          MMS_MERGE_TREE);
}

mms_status mms_merge_pass_partition(mms_key_type kt, const void* d_in, void* d_out, size_t n,
                                    size_t run_len, int K, const int64_t* d_table, void* d_ws,
                                    size_t ws_bytes, void* stream) {
  return merge_pass_entry(kt, d_in, d_out, n, run_len, K, d_table, d_ws, ws_bytes, stream,
                          MMS_MERGE_PARTITION);
}

mms_status mms_merge_pass_pipelined(mms_key_type kt, const void* d_in, void* d_out, size_t n,
                                    size_t run_len, int K, const int64_t* d_table, void* d_ws,
                                    size_t ws_bytes, void* stream) {
  return merge_pass_entry(kt, d_in, d_out, n, run_len, K, d_table, d_ws, ws_bytes, stream,
                          MMS_MERGE_PIPELINED);
}

}  // extern "C"
