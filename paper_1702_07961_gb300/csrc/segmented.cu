// segmented.cu -- batched sorting: many independent arrays ("segments") of
// uneven size, laid out back to back, sorted in one call whose launch
// sequence needs no host synchronisation, so it can be captured once into a
// CUDA graph and replayed as a single graph launch.
//
// The method is the same as for one array (base case, then K-way merge
// rounds of splitter + merge pass, Sec. 4); only the bookkeeping is
// segmented:
//   - a device planner gives every segment its fanout K (per size class
//     ceil(log2 n), from a table the caller's autotuner fills), its number of
//     rounds R = ceil(log_K(tiles)), and its tile count in every phase (the
//     base case, then merge round r < R);
//   - an exclusive scan per phase and a descriptor kernel turn these counts
//     into one 16-byte descriptor per tile of the phase (segment base, size,
//     tile index, K, buffer parity, last-phase flag);
//   - persistent kernels (a grid sized to the GPU, each CTA looping over the
//     phase's descriptors) run the same CTA bodies as the whole-array kernels
//     (tile_sort.cuh, splitter.cuh, merge_tile.cuh) on each tile.
// A segment with R rounds is base-sorted into the workspace copy when R is
// odd, so that its last round lands in the caller's buffer; segments that are
// done drop out of later phases.  Key-value batches run on 64-bit composites
// (ordered key << 32 | position in the batch), which both workspace buffers
// hold; a last kernel writes keys and gathers values for the whole batch.
#include <cuda_runtime.h>
#include <stdio.h>

#include "../../include/mms.h"
#include "merge_tile.cuh"
#include "splitter.cuh"
#include "tile_sort.cuh"

namespace mms {
namespace {

constexpr int kRowStride = kMaxFanout;     // pivot-table row width of a segmented round
constexpr int kMaxRounds = 40;

struct SegPlan {
  int class_fanout[33];   // K per size class ceil(log2 n)
  int S;                  // tile items (base case and merge output tiles)
  int rounds;             // merge rounds launched
  int nphase;             // 1 + rounds
};

__host__ __device__ inline int size_class(unsigned long long n) {
  int c = 0;
  while (c < 64 && (1ull << c) < n) ++c;
  return c > 32 ? 32 : c;
}

__host__ __device__ inline int rounds_for(long long tiles, int K) {
  int r = 0;
  long long cover = 1;
  while (cover < tiles) {
    cover *= K;
    ++r;
  }
  return r;
}

// Descriptor word w: tile index (21 bits) | K (6 bits) << 21 | flip << 27 |
// last << 28.  flip: for the base case, the output goes to the workspace
// buffer; for a merge round, the input is in the workspace buffer.  last: the
// phase is the segment's last (undo the float transform on the way out).
struct Desc {
  unsigned long long base;
  unsigned n;
  unsigned w;
};
static_assert(sizeof(Desc) == 16, "descriptor is 16 bytes");

__device__ __forceinline__ Desc load_desc(const Desc* d) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(d));
  Desc r;
  r.base = (unsigned long long)v.x | ((unsigned long long)v.y << 32);
  r.n = v.z;
  r.w = v.w;
  return r;
}

// ---- planner --------------------------------------------------------------

// One thread per segment: K, R and the tile count of every phase.
__global__ void seg_plan_kernel(const unsigned long long* __restrict__ off, long long nseg,
                                unsigned long long total_n, SegPlan P, int* __restrict__ segK,
                                int* __restrict__ segR, int* __restrict__ counts, int* dev_err) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const unsigned long long a = off[s], b = off[s + 1];
  long long n = 0;
  if (b < a || b > total_n || (s == 0 && a != 0) || (s == nseg - 1 && b != total_n) ||
      b - a > 0xFFFFFFFFull) {
    set_device_error(dev_err, kDevErrInternal);   // offsets out of order or too large
  } else {
    n = (long long)(b - a);
  }
  const long long tiles = (n + P.S - 1) / P.S;
  int K = P.class_fanout[size_class((unsigned long long)n)];
  K = K < 2 ? 2 : (K > kMaxFanout ? kMaxFanout : K);
  int R = rounds_for(tiles, K);
  if (R > P.rounds) {
    set_device_error(dev_err, kDevErrInternal);   // a segment above the declared maximum
    R = P.rounds;
  }
  segK[s] = K;
  segR[s] = R;
  counts[s] = (int)tiles;                         // phase 0: base case
  long long run_len = P.S;
  for (int r = 0; r < P.rounds; ++r) {
    counts[(long long)(1 + r) * nseg + s] = (r < R) ? (int)num_tiles(P.S, n, run_len, K) : 0;
    if (r < R) run_len *= K;
  }
}

// One CTA per phase: exclusive scan of the phase's counts in place, total
// into totals[phase].
__global__ void __launch_bounds__(1024) seg_scan_kernel(int* __restrict__ counts, long long nseg,
                                                        int* __restrict__ totals) {
  __shared__ int warp_sums[32];
  __shared__ int carry_s;
  int* c = counts + (long long)blockIdx.x * nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (long long base = 0; base < nseg; base += 1024) {
    const long long i = base + threadIdx.x;
    const int v = i < nseg ? c[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_sums[lane] = w;                          // inclusive over warps
    }
    __syncthreads();
    const int carry = carry_s;
    const int excl = carry + (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    if (i < nseg) c[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry_s;
}

// One thread per potential tile of a phase: finds its segment (last one whose
// offset is <= t) and writes the descriptor.
__global__ void seg_desc_kernel(const unsigned long long* __restrict__ off, long long nseg,
                                const int* __restrict__ segK, const int* __restrict__ segR,
                                const int* __restrict__ offs, const int* __restrict__ totals,
                                long long per_phase, Desc* __restrict__ desc) {
  const int p = blockIdx.y;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // Offsets that overlap (flagged by the planner) can make the counts exceed
  // the descriptor capacity of a phase: never write past it.
  if (t >= totals[p] || t >= per_phase) return;
  const int* o = offs + (long long)p * nseg;
  long long lo = 0, hi = nseg - 1;                 // last s with o[s] <= t
  while (lo < hi) {
    const long long mid = (lo + hi + 1) >> 1;
    if (o[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const long long s = lo;
  const int K = segK[s], R = segR[s];
  const unsigned idx = (unsigned)(t - o[s]);
  unsigned flip, last;
  if (p == 0) {
    flip = (unsigned)(R & 1);
    last = R == 0;
  } else {
    const int r = p - 1;
    flip = (unsigned)((R - r) & 1);
    last = r == R - 1;
  }
  Desc d;
  d.base = off[s];
  d.n = (unsigned)(off[s + 1] - off[s]);
  d.w = idx | ((unsigned)K << 21) | (flip << 27) | (last << 28);
  desc[(long long)p * per_phase + t] = d;
}

// ---- persistent phase kernels ----------------------------------------------

template <typename KeyT, int WARPS, bool XIN>
__global__ void __launch_bounds__(WARPS * 32, (MinBlocks<KeyT, WARPS>::value))
    seg_tile_sort_kernel(const KeyT* __restrict__ keys_in, KeyT* bufA, KeyT* bufB,
                         const Desc* __restrict__ desc, const int* __restrict__ total,
                         long long per_phase) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int T = WARPS * kBlockItems;
  const int cnt = (int)min((long long)*total, per_phase);
  for (int t = blockIdx.x; t < cnt; t += gridDim.x) {
    const Desc d = load_desc(desc + t);
    const unsigned idx = d.w & 0x1FFFFFu;
    KeyT* out = ((d.w >> 27) & 1u) ? bufB : bufA;
    tile_sort_tile<KeyT, WARPS, XIN>(keys_in + d.base, out + d.base, (long long)d.n,
                                     (long long)idx * T, XIN && ((d.w >> 28) & 1u), smem_raw);
  }
}

template <int WARPS, bool XIN>
__global__ void __launch_bounds__(WARPS * 32, (MinBlocks<uint64_t, WARPS>::value))
    seg_tile_sort_composite_kernel(const uint32_t* __restrict__ keys_in, uint64_t* bufA,
                                   uint64_t* bufB, const Desc* __restrict__ desc,
                                   const int* __restrict__ total, long long per_phase) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int T = WARPS * kBlockItems;
  const int cnt = (int)min((long long)*total, per_phase);
  for (int t = blockIdx.x; t < cnt; t += gridDim.x) {
    const Desc d = load_desc(desc + t);
    const unsigned idx = d.w & 0x1FFFFFu;
    uint64_t* out = ((d.w >> 27) & 1u) ? bufB : bufA;
    tile_sort_composite_tile<WARPS, XIN>(keys_in + d.base, out + d.base, (long long)d.n,
                                         (long long)idx * T, (long long)d.base, smem_raw);
  }
}

template <typename KeyT>
__global__ void __launch_bounds__(128)
    seg_splitter_kernel(const KeyT* bufA, const KeyT* bufB, const Desc* __restrict__ desc,
                        const int* __restrict__ total, long long per_phase, long long S, int r,
                        long long* __restrict__ table) {
  const int cnt = (int)min((long long)*total, per_phase);
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < cnt;
       t += warps) {
    const Desc d = load_desc(desc + t);
    const unsigned idx = d.w & 0x1FFFFFu;
    const int K = (int)((d.w >> 21) & 63u);
    const KeyT* in = (((d.w >> 27) & 1u) ? bufB : bufA) + d.base;
    long long run_len = S, tpg = K;
    for (int i = 0; i < r; ++i) {
      run_len *= K;
      tpg *= K;
    }
    splitter_row<KeyT, 32>(in, (long long)d.n, run_len, K, S, idx / tpg, idx % tpg,
                           table + t * kRowStride, 0xffffffffu, 0);
  }
}

template <typename KeyT, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, (MinBlocks<KeyT, WARPS>::value))
    seg_merge_kernel(KeyT* bufA, KeyT* bufB, const Desc* __restrict__ desc,
                     const int* __restrict__ total, long long per_phase, int r, bool is_f32,
                     const long long* __restrict__ table, size_t bar_off, int* dev_err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int S = WARPS * kBlockItems;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + bar_off);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  const int cnt = (int)min((long long)*total, per_phase);
  unsigned phase = 0;
  for (int t = blockIdx.x; t < cnt; t += gridDim.x) {
    const Desc d = load_desc(desc + t);
    const unsigned idx = d.w & 0x1FFFFFu;
    const int K = (int)((d.w >> 21) & 63u);
    const bool flip = (d.w >> 27) & 1u;
    const KeyT* in = (flip ? bufB : bufA) + d.base;
    KeyT* out = (flip ? bufA : bufB) + d.base;
    long long run_len = S, tpg = K;
    for (int i = 0; i < r; ++i) {
      run_len *= K;
      tpg *= K;
    }
    if (!merge_tile<KeyT, WARPS>(in, out, (long long)d.n, run_len, K, idx / tpg, idx % tpg,
                                 table + (long long)t * kRowStride,
                                 table + (long long)(t + 1) * kRowStride,
                                 is_f32 && ((d.w >> 28) & 1u), dev_err, smem_raw, bar, phase, S))
      return;
    phase ^= 1u;
  }
}

// ---- host side -------------------------------------------------------------

int key_bytes_of(mms_key_type kt) { return kt == MMS_KEY_U64 ? 8 : 4; }
size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
constexpr size_t kStatusBytes = 256;

mms_status seg_fail(mms_status s, const char* what) {
  set_error_detail(what);
  return s;
}

// Tile warps of a segmented sort: the whole-array default, or opt->tile_items.
int seg_tile_warps(int unit_bytes, const mms_segmented_options* opt) {
  if (opt && opt->tile_items > 0) return opt->tile_items / 1024;
  return default_tile_warps(unit_bytes);
}

// Fanout per size class: the caller's table where set, else the whole-array
// default (4 for 4-byte units, 8 for 8-byte units).
void fill_plan(SegPlan& P, int unit_bytes, const mms_segmented_options* opt) {
  const int def = unit_bytes == 8 ? 8 : 4;
  for (int c = 0; c <= 32; ++c) {
    const int k = opt ? opt->class_fanout[c] : 0;
    P.class_fanout[c] = (k >= 2 && k <= kMaxFanout) ? k : def;
  }
  P.S = 1024 * seg_tile_warps(unit_bytes, opt);
}

int max_rounds(const SegPlan& P, unsigned long long max_seg) {
  int R = 0;
  for (int c = 0; c <= 32; ++c) {
    const unsigned long long top = c >= 63 ? ~0ull : (1ull << c);
    const unsigned long long nmax = top < max_seg ? top : max_seg;
    const long long tiles = (long long)((nmax + P.S - 1) / P.S);
    const int r = rounds_for(tiles, P.class_fanout[c]);
    R = r > R ? r : R;
    if (top >= max_seg) break;
  }
  return R;
}

struct SegLayout {
  size_t tmp0, tmp1, vals, segK, segR, counts, totals, desc, table, total;
  long long per_phase;
};

// Workspace: status | unit buffers | values copy | per-segment K, R | counts
// (scanned in place) | totals | descriptors | pivot table.
SegLayout seg_layout(int unit_bytes, bool pairs, size_t total_n, size_t nseg, const SegPlan& P) {
  SegLayout L{};
  size_t o = kStatusBytes;
  L.tmp0 = o;
  o = round_up(o + total_n * unit_bytes, 256);
  L.tmp1 = o;
  if (pairs) o = round_up(o + total_n * unit_bytes, 256);
  L.vals = o;
  if (pairs) o = round_up(o + total_n * 4, 256);
  L.segK = o;
  o = round_up(o + nseg * 4, 256);
  L.segR = o;
  o = round_up(o + nseg * 4, 256);
  L.counts = o;
  o = round_up(o + (size_t)P.nphase * nseg * 4, 256);
  L.totals = o;
  o = round_up(o + (size_t)P.nphase * 4, 256);
  L.per_phase = (long long)((total_n + P.S - 1) / P.S + nseg);
  L.desc = o;
  o = round_up(o + (size_t)P.nphase * (size_t)L.per_phase * sizeof(Desc), 256);
  L.table = o;
  o = round_up(o + ((size_t)L.per_phase + 1) * kRowStride * sizeof(long long), 256);
  L.total = o;
  return L;
}

// Key-value batches of 8-byte keys: two stable 4-byte passes (low half, then
// high half; see pairs.cu) over the 4-byte batch layout, plus a 4-byte half
// of every key, the position list, and copies of the keys and values.
struct SegLayout64 {
  SegLayout inner;
  size_t half, perm, kcopy, vcopy, total;
};

SegLayout64 seg_layout64(size_t total_n, size_t nseg, const SegPlan& P) {
  SegLayout64 L{};
  L.inner = seg_layout(8, true, total_n, nseg, P);
  size_t o = L.inner.total;
  L.half = o;
  o = round_up(o + total_n * 4, 256);
  L.perm = o;
  o = round_up(o + total_n * 4, 256);
  L.kcopy = o;
  o = round_up(o + total_n * 8, 256);
  L.vcopy = o;
  o = round_up(o + total_n * 4, 256);
  L.total = o;
  return L;
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Raises a kernel's dynamic shared-memory limit, except while `s` is being
// captured into a graph: the capture is preceded by a preparing pass that
// sets every attribute (attribute calls are not stream work).
template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) return cudaSuccess;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename Kern>
cudaError_t persistent_grid(Kern k, int threads, size_t smem, long long upper, unsigned* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long g = (long long)per_sm * sm_count();
  if (g > upper) g = upper;
  if (g < 1) g = 1;
  *grid = (unsigned)g;
  return cudaSuccess;
}

template <typename KeyT, int WARPS, bool XIN>
cudaError_t launch_seg_tile(const void* keys_in, void* a, void* b, const Desc* desc,
                            const int* total, long long upper, cudaStream_t s) {
  auto k = seg_tile_sort_kernel<KeyT, WARPS, XIN>;
  const size_t smem = tile_sort_smem_bytes(sizeof(KeyT), WARPS);
  cudaError_t e = set_smem(k, smem, s);
  unsigned grid = 1;
  if (e == cudaSuccess) e = persistent_grid(k, WARPS * 32, smem, upper, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, WARPS * 32, smem, s>>>(static_cast<const KeyT*>(keys_in), static_cast<KeyT*>(a),
                                   static_cast<KeyT*>(b), desc, total, upper);
  return cudaGetLastError();
}

template <int WARPS, bool XIN>
cudaError_t launch_seg_tile_comp(const void* keys_in, void* a, void* b, const Desc* desc,
                                 const int* total, long long upper, cudaStream_t s) {
  auto k = seg_tile_sort_composite_kernel<WARPS, XIN>;
  const size_t smem = tile_sort_smem_bytes(8, WARPS);
  cudaError_t e = set_smem(k, smem, s);
  unsigned grid = 1;
  if (e == cudaSuccess) e = persistent_grid(k, WARPS * 32, smem, upper, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, WARPS * 32, smem, s>>>(static_cast<const uint32_t*>(keys_in),
                                   static_cast<uint64_t*>(a), static_cast<uint64_t*>(b), desc,
                                   total, upper);
  return cudaGetLastError();
}

template <typename KeyT>
cudaError_t launch_seg_split(const void* a, const void* b, const Desc* desc, const int* total,
                             long long upper, long long S, int r, long long* table,
                             cudaStream_t s) {
  auto k = seg_splitter_kernel<KeyT>;
  unsigned grid = 1;
  cudaError_t e = persistent_grid(k, 128, 0, (upper + 3) / 4, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, 128, 0, s>>>(static_cast<const KeyT*>(a), static_cast<const KeyT*>(b), desc, total,
                         upper, S, r, table);
  return cudaGetLastError();
}

template <typename KeyT, int WARPS>
size_t seg_merge_bar_off(int kmax) {
  return round_up(sizeof(KeyT) * 2 * (size_t)MergeGeom<KeyT, WARPS>::cap(kmax), 16);
}

template <typename KeyT, int WARPS>
cudaError_t launch_seg_merge(void* a, void* b, const Desc* desc, const int* total,
                             long long upper, int r, bool is_f32, int kmax,
                             const long long* table, int* dev_err, cudaStream_t s) {
  auto k = seg_merge_kernel<KeyT, WARPS>;
  const size_t bar_off = seg_merge_bar_off<KeyT, WARPS>(kmax);
  const size_t smem = bar_off + 16 + kMergeCtlBytes;
  cudaError_t e = set_smem(k, smem, s);
  unsigned grid = 1;
  if (e == cudaSuccess) e = persistent_grid(k, WARPS * 32, smem, upper, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, WARPS * 32, smem, s>>>(static_cast<KeyT*>(a), static_cast<KeyT*>(b), desc, total,
                                   upper, r, is_f32, table, bar_off, dev_err);
  return cudaGetLastError();
}

cudaError_t seg_tile_phase(mms_key_type kt, bool pairs, int tw, const void* keys, void* a,
                           void* b, const Desc* desc, const int* total, long long upper,
                           cudaStream_t s) {
  const bool f = kt == MMS_KEY_F32;
  if (pairs) {
    if (tw == 4) return f ? launch_seg_tile_comp<4, true>(keys, a, b, desc, total, upper, s)
                          : launch_seg_tile_comp<4, false>(keys, a, b, desc, total, upper, s);
    if (tw == 2) return f ? launch_seg_tile_comp<2, true>(keys, a, b, desc, total, upper, s)
                          : launch_seg_tile_comp<2, false>(keys, a, b, desc, total, upper, s);
    return cudaErrorInvalidValue;
  }
  if (kt == MMS_KEY_U64) {
    if (tw == 4) return launch_seg_tile<uint64_t, 4, false>(keys, a, b, desc, total, upper, s);
    if (tw == 2) return launch_seg_tile<uint64_t, 2, false>(keys, a, b, desc, total, upper, s);
    return cudaErrorInvalidValue;
  }
  if (tw == 8) return f ? launch_seg_tile<uint32_t, 8, true>(keys, a, b, desc, total, upper, s)
                        : launch_seg_tile<uint32_t, 8, false>(keys, a, b, desc, total, upper, s);
  if (tw == 4) return f ? launch_seg_tile<uint32_t, 4, true>(keys, a, b, desc, total, upper, s)
                        : launch_seg_tile<uint32_t, 4, false>(keys, a, b, desc, total, upper, s);
  return cudaErrorInvalidValue;
}

cudaError_t seg_round(int unit_bytes, int tw, bool is_f32, int kmax, void* a, void* b,
                      const Desc* desc, const int* total, long long upper, long long S, int r,
                      long long* table, int* dev_err, cudaStream_t s) {
  cudaError_t e;
  if (unit_bytes == 8) {
    e = launch_seg_split<uint64_t>(a, b, desc, total, upper, S, r, table, s);
    if (e != cudaSuccess) return e;
    if (tw == 4) return launch_seg_merge<uint64_t, 4>(a, b, desc, total, upper, r, false, kmax, table, dev_err, s);
    if (tw == 2) return launch_seg_merge<uint64_t, 2>(a, b, desc, total, upper, r, false, kmax, table, dev_err, s);
    return cudaErrorInvalidValue;
  }
  e = launch_seg_split<uint32_t>(a, b, desc, total, upper, S, r, table, s);
  if (e != cudaSuccess) return e;
  if (tw == 8) return launch_seg_merge<uint32_t, 8>(a, b, desc, total, upper, r, is_f32, kmax, table, dev_err, s);
  if (tw == 4) return launch_seg_merge<uint32_t, 4>(a, b, desc, total, upper, r, is_f32, kmax, table, dev_err, s);
  return cudaErrorInvalidValue;
}

template <typename Kern>
cudaError_t attr(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Sets the shared-memory attribute of every kernel a batch of this shape
// launches (before a graph capture, during which attributes are not set).
mms_status seg_prepare(mms_key_type kt, bool pairs, int tw, int kmax) {
  cudaError_t e = cudaSuccess;
  const bool f = kt == MMS_KEY_F32;
  if (pairs) {
    const size_t t = tile_sort_smem_bytes(8, tw);
    if (tw == 4) e = f ? attr(seg_tile_sort_composite_kernel<4, true>, t) : attr(seg_tile_sort_composite_kernel<4, false>, t);
    if (tw == 2) e = f ? attr(seg_tile_sort_composite_kernel<2, true>, t) : attr(seg_tile_sort_composite_kernel<2, false>, t);
  } else if (kt == MMS_KEY_U64) {
    const size_t t = tile_sort_smem_bytes(8, tw);
    if (tw == 4) e = attr(seg_tile_sort_kernel<uint64_t, 4, false>, t);
    if (tw == 2) e = attr(seg_tile_sort_kernel<uint64_t, 2, false>, t);
  } else {
    const size_t t = tile_sort_smem_bytes(4, tw);
    if (tw == 8) e = f ? attr(seg_tile_sort_kernel<uint32_t, 8, true>, t) : attr(seg_tile_sort_kernel<uint32_t, 8, false>, t);
    if (tw == 4) e = f ? attr(seg_tile_sort_kernel<uint32_t, 4, true>, t) : attr(seg_tile_sort_kernel<uint32_t, 4, false>, t);
  }
  if (e == cudaSuccess) {
    if (pairs || kt == MMS_KEY_U64) {
      if (tw == 4) e = attr(seg_merge_kernel<uint64_t, 4>, seg_merge_bar_off<uint64_t, 4>(kmax) + 16 + kMergeCtlBytes);
      if (tw == 2) e = attr(seg_merge_kernel<uint64_t, 2>, seg_merge_bar_off<uint64_t, 2>(kmax) + 16 + kMergeCtlBytes);
    } else {
      if (tw == 8) e = attr(seg_merge_kernel<uint32_t, 8>, seg_merge_bar_off<uint32_t, 8>(kmax) + 16 + kMergeCtlBytes);
      if (tw == 4) e = attr(seg_merge_kernel<uint32_t, 4>, seg_merge_bar_off<uint32_t, 4>(kmax) + 16 + kMergeCtlBytes);
    }
  }
  return e == cudaSuccess ? MMS_OK : seg_fail(MMS_ERR_CUDA, cudaGetErrorString(e));
}

bool seg_args_ok(mms_key_type kt, const uint32_t* vals, const mms_segmented_options* opt,
                 const char** why) {
  if (kt != MMS_KEY_U32 && kt != MMS_KEY_U64 && kt != MMS_KEY_F32) { *why = "unknown key type"; return false; }
  if (opt && opt->tile_items) {
    const int unit = (vals || kt == MMS_KEY_U64) ? 8 : 4;
    const int w = opt->tile_items / 1024;
    if (opt->tile_items % 1024 || !valid_tile_warps(unit, w)) {
      *why = "tile_items must be 0, 4096/8192 (4-byte keys) or 2048/4096 (8-byte keys, key-value batches)";
      return false;
    }
  }
  return true;
}

}  // namespace
}  // namespace mms

using namespace mms;

extern "C" {

int mms_segmented_rounds(mms_key_type kt, size_t max_segment_items, int with_values,
                         const mms_segmented_options* opt) {
  const int unit = (with_values || kt == MMS_KEY_U64) ? 8 : 4;
  SegPlan P{};
  fill_plan(P, unit, opt);
  return max_rounds(P, max_segment_items);
}

size_t mms_segmented_workspace_bytes(mms_key_type kt, size_t total_n, size_t num_segments,
                                     int with_values, const mms_segmented_options* opt) {
  const char* why = "";
  if (!seg_args_ok(kt, with_values ? reinterpret_cast<const uint32_t*>(1) : nullptr, opt, &why)) return 0;
  const int unit = (with_values || kt == MMS_KEY_U64) ? 8 : 4;
  SegPlan P{};
  fill_plan(P, unit, opt);
  const size_t mx = (opt && opt->max_segment_items) ? opt->max_segment_items : total_n;
  P.rounds = max_rounds(P, mx);
  P.nphase = 1 + P.rounds;
  if (with_values && kt == MMS_KEY_U64) return seg_layout64(total_n, num_segments, P).total;
  return seg_layout(unit, with_values != 0, total_n, num_segments, P).total;
}

static mms_status seg_sort_impl(mms_key_type kt, void* d_keys, uint32_t* d_values,
                                const uint64_t* d_offsets, size_t num_segments, size_t total_n,
                                void* d_ws, size_t ws_bytes, void* stream,
                                const mms_segmented_options* opt, bool prepare_only,
                                bool clear_status = true) {
  const char* why = "";
  if (!seg_args_ok(kt, d_values, opt, &why)) return seg_fail(MMS_ERR_INVALID_ARG, why);
  if (num_segments == 0 || total_n == 0) return MMS_OK;
  if (!d_keys || !d_offsets || ((uintptr_t)d_keys & 15u) || ((uintptr_t)d_offsets & 7u) ||
      (d_values && ((uintptr_t)d_values & 15u)))
    return seg_fail(MMS_ERR_INVALID_ARG, "keys/values not 16-byte aligned, or offsets not 8-byte aligned");
  if (d_values && total_n > 0xFFFFFFFEull)
    return seg_fail(MMS_ERR_UNSUPPORTED, "key-value batches take fewer than 2^32 items in all");
  if (num_segments > 0x7FFFFFFFull) return seg_fail(MMS_ERR_UNSUPPORTED, "at most 2^31 - 1 segments");
  const bool pairs = d_values != nullptr;
  const int unit = (pairs || kt == MMS_KEY_U64) ? 8 : 4;
  SegPlan P{};
  fill_plan(P, unit, opt);
  const size_t mx = (opt && opt->max_segment_items) ? opt->max_segment_items : total_n;
  P.rounds = max_rounds(P, mx);
  if (P.rounds > kMaxRounds) return seg_fail(MMS_ERR_UNSUPPORTED, "too many merge rounds");
  P.nphase = 1 + P.rounds;
  if (pairs && kt == MMS_KEY_U64) {
    // Two stable passes of the 4-byte key-value batch, low key halves first.
    const SegLayout64 L = seg_layout64(total_n, num_segments, P);
    if (!d_ws || ((uintptr_t)d_ws & 255u)) return seg_fail(MMS_ERR_INVALID_ARG, "workspace missing or not 256-byte aligned");
    if (ws_bytes < L.total) return seg_fail(MMS_ERR_NO_MEMORY, "workspace smaller than mms_segmented_workspace_bytes()");
    unsigned char* ws = static_cast<unsigned char*>(d_ws);
    void* half = ws + L.half;
    uint32_t* perm = reinterpret_cast<uint32_t*>(ws + L.perm);
    cudaStream_t s = (cudaStream_t)stream;
    if (prepare_only)
      return seg_sort_impl(MMS_KEY_U32, half, perm, d_offsets, num_segments, total_n, d_ws,
                           L.inner.total, stream, opt, true);
    if (clear_status && cudaMemsetAsync(d_ws, 0, sizeof(int), s) != cudaSuccess)
      return seg_fail(MMS_ERR_CUDA, "status word");
    if (launch_u64_pairs_split(d_keys, d_values, half, perm, ws + L.kcopy, ws + L.vcopy,
                               (long long)total_n, s) != cudaSuccess)
      return seg_fail(MMS_ERR_CUDA, "key-value split (8-byte keys)");
    mms_status st = seg_sort_impl(MMS_KEY_U32, half, perm, d_offsets, num_segments, total_n, d_ws,
                                  L.inner.total, stream, opt, false, false);
    if (st != MMS_OK) return st;
    if (launch_u64_pairs_hi(ws + L.kcopy, perm, half, (long long)total_n, s) != cudaSuccess)
      return seg_fail(MMS_ERR_CUDA, "key-value high halves (8-byte keys)");
    st = seg_sort_impl(MMS_KEY_U32, half, perm, d_offsets, num_segments, total_n, d_ws,
                       L.inner.total, stream, opt, false, false);
    if (st != MMS_OK) return st;
    if (launch_u64_pairs_final(ws + L.kcopy, ws + L.vcopy, perm, d_keys, d_values,
                               (long long)total_n, s) != cudaSuccess)
      return seg_fail(MMS_ERR_CUDA, "key-value permutation (8-byte keys)");
    return MMS_OK;
  }
  const SegLayout L = seg_layout(unit, pairs, total_n, num_segments, P);
  if (L.per_phase > 0x7FFFFFFFll) return seg_fail(MMS_ERR_UNSUPPORTED, "too many tiles per phase");
  if (!d_ws || ((uintptr_t)d_ws & 255u)) return seg_fail(MMS_ERR_INVALID_ARG, "workspace missing or not 256-byte aligned");
  if (ws_bytes < L.total) return seg_fail(MMS_ERR_NO_MEMORY, "workspace smaller than mms_segmented_workspace_bytes()");

  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* ws = static_cast<unsigned char*>(d_ws);
  int* dev_err = reinterpret_cast<int*>(ws);
  int* segK = reinterpret_cast<int*>(ws + L.segK);
  int* segR = reinterpret_cast<int*>(ws + L.segR);
  int* counts = reinterpret_cast<int*>(ws + L.counts);
  int* totals = reinterpret_cast<int*>(ws + L.totals);
  Desc* desc = reinterpret_cast<Desc*>(ws + L.desc);
  long long* table = reinterpret_cast<long long*>(ws + L.table);
  const auto* off = reinterpret_cast<const unsigned long long*>(d_offsets);
  const long long nseg = (long long)num_segments;
  const int tw = P.S / 1024;
  int kmax = 2;
  for (int c = 0; c <= size_class(mx); ++c) kmax = P.class_fanout[c] > kmax ? P.class_fanout[c] : kmax;

  if (prepare_only) return seg_prepare(kt, pairs, tw, kmax);

  int ev = 0;
  auto mark = [&]() {
    if (opt && opt->events && ev < opt->num_events && opt->events[ev])
      cudaEventRecord((cudaEvent_t)opt->events[ev], s);
    ++ev;
  };
  auto chk = [&](cudaError_t e, const char* where) {
    if (e == cudaSuccess) return MMS_OK;
    char buf[200];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    set_error_detail(buf);
    return MMS_ERR_CUDA;
  };
  mark();
  mms_status st = clear_status ? chk(cudaMemsetAsync(dev_err, 0, sizeof(int), s), "status word")
                               : MMS_OK;
  if (st == MMS_OK) {
    seg_plan_kernel<<<(unsigned)((nseg + 255) / 256), 256, 0, s>>>(off, nseg, total_n, P, segK, segR,
                                                                  counts, dev_err);
    st = chk(cudaGetLastError(), "seg_plan");
  }
  if (st == MMS_OK) {
    seg_scan_kernel<<<(unsigned)P.nphase, 1024, 0, s>>>(counts, nseg, totals);
    st = chk(cudaGetLastError(), "seg_scan");
  }
  if (st == MMS_OK) {
    dim3 g((unsigned)((L.per_phase + 255) / 256), (unsigned)P.nphase);
    seg_desc_kernel<<<g, 256, 0, s>>>(off, nseg, segK, segR, counts, totals, L.per_phase, desc);
    st = chk(cudaGetLastError(), "seg_desc");
  }
  void* bufA = pairs ? (void*)(ws + L.tmp0) : d_keys;     // where every segment ends
  void* bufB = pairs ? (void*)(ws + L.tmp1) : (void*)(ws + L.tmp0);
  if (st == MMS_OK && pairs)
    st = chk(cudaMemcpyAsync(ws + L.vals, d_values, total_n * 4, cudaMemcpyDeviceToDevice, s), "copy of the values");
  mark();
  if (st == MMS_OK)
    st = chk(seg_tile_phase(kt, pairs, tw, d_keys, bufA, bufB, desc, totals, L.per_phase, s), "seg base case");
  mark();
  for (int r = 0; r < P.rounds && st == MMS_OK; ++r) {
    st = chk(seg_round(unit, tw, kt == MMS_KEY_F32 && !pairs, kmax, bufA, bufB,
                       desc + (long long)(1 + r) * L.per_phase, totals + 1 + r, L.per_phase, P.S,
                       r, table, dev_err, s),
             "seg merge round");
    mark();
  }
  if (st == MMS_OK && pairs)
    st = chk(launch_pairs_finalize(kt == MMS_KEY_F32, bufA, ws + L.vals, d_keys, d_values,
                                   (long long)total_n, s),
             "pairs_finalize");
  mark();
  return st;
}

mms_status mms_segmented_sort(mms_key_type kt, void* d_keys, uint32_t* d_values,
                              const uint64_t* d_offsets, size_t num_segments, size_t total_n,
                              void* d_ws, size_t ws_bytes, void* stream,
                              const mms_segmented_options* opt) {
  return seg_sort_impl(kt, d_keys, d_values, d_offsets, num_segments, total_n, d_ws, ws_bytes,
                       stream, opt, false);
}

// ---- CUDA graph of one batched sort ----------------------------------------

struct mms_graph_s {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

mms_status mms_segmented_graph_create(mms_key_type kt, void* d_keys, uint32_t* d_values,
                                      const uint64_t* d_offsets, size_t num_segments,
                                      size_t total_n, void* d_ws, size_t ws_bytes,
                                      const mms_segmented_options* opt, mms_graph* out) {
  if (!out) return seg_fail(MMS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  mms_segmented_options o{};
  if (opt) o = *opt;
  o.events = nullptr;
  o.num_events = 0;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return seg_fail(MMS_ERR_CUDA, "stream creation failed");
  // The preparing pass checks the arguments and sets every kernel attribute;
  // it queues no work.
  mms_status st = seg_sort_impl(kt, d_keys, d_values, d_offsets, num_segments, total_n, d_ws,
                                ws_bytes, s, &o, true);
  cudaGraph_t g = nullptr;
  if (st == MMS_OK) {
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = seg_fail(MMS_ERR_CUDA, "stream capture could not start");
    } else {
      st = seg_sort_impl(kt, d_keys, d_values, d_offsets, num_segments, total_n, d_ws, ws_bytes,
                         s, &o, false);
      const cudaError_t e = cudaStreamEndCapture(s, &g);
      if (st == MMS_OK && e != cudaSuccess) st = seg_fail(MMS_ERR_CUDA, "stream capture failed");
    }
  }
  cudaGraphExec_t x = nullptr;
  if (st == MMS_OK && cudaGraphInstantiate(&x, g, 0) != cudaSuccess)
    st = seg_fail(MMS_ERR_CUDA, "graph instantiation failed");
  cudaStreamDestroy(s);
  if (st != MMS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  *out = new mms_graph_s{g, x};
  return MMS_OK;
}

mms_status mms_graph_launch(mms_graph g, void* stream) {
  if (!g) return seg_fail(MMS_ERR_INVALID_ARG, "graph is NULL");
  const cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return seg_fail(MMS_ERR_CUDA, cudaGetErrorString(e));
  return MMS_OK;
}

void mms_graph_destroy(mms_graph g) {
  if (!g) return;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
}

}  // extern "C"
