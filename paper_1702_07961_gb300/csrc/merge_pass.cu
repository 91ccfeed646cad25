// merge_pass.cu -- one K-way merge round of GPU Multiway Mergesort (Sec. 4.2
// "I/O Efficient Merging", Sec. 5.1 I/O analysis).
//
// One CTA produces one output tile of S = 1024 * WARPS items of its group of K
// runs.  The splitter table gives, for the tile's start and end, the pivot in
// every run (Sec. 4.1), so the tile's inputs are K contiguous segments whose
// lengths sum to S.  The CTA:
//   1. stages the K segments into shared memory with 1-D TMA bulk copies
//      (cp.async.bulk, one mbarrier; the < 16-byte ragged ends of each
//      segment by plain loads), so every input byte is read from HBM once;
//   2. merges them in ceil(log2 K) levels of pairwise block merges, each warp
//      producing 1024-item output blocks with the conflict-free bitonic block
//      merge (the paper merges 32+32 blocks in a minBlockHeap; the levels here
//      play the heap's levels);
//   3. writes the tile with coalesced 128-bit stores, so every output byte is
//      written once: 2 * S * sizeof(key) bytes of HBM traffic per tile.
#include "mms_common.cuh"
#include "mms_kernels.cuh"

namespace mms {

template <typename KeyT>
struct MergeVec;
template <>
struct MergeVec<uint32_t> {
  using T = uint4;
  static constexpr int E = 4;
};
template <>
struct MergeVec<uint64_t> {
  using T = ulonglong2;
  static constexpr int E = 2;
};

// Items of slack per segment in the staging buffer: the copied head before a
// segment start (< E) and the rounding of its end (< E).
template <typename KeyT, int WARPS>
struct MergeGeom {
  static constexpr int E = MergeVec<KeyT>::E;
  static constexpr int S = WARPS * kBlockItems;
  static constexpr int XCAP = S + kMaxFanout * 2 * E;   // staging buffer (also a level buffer)
  static constexpr int YCAP = S;
  static constexpr size_t bytes() {
    return sizeof(KeyT) * ((size_t)XCAP + YCAP + (size_t)WARPS * kScratchItems);
  }
};

size_t merge_pass_smem_bytes(int key_bytes, int warps) {
  if (key_bytes == 4) return MergeGeom<uint32_t, kTileWarps32>::bytes();
  return MergeGeom<uint64_t, kTileWarps64>::bytes();
  (void)warps;
}

template <typename KeyT, int WARPS, bool XOUT>
__global__ void __launch_bounds__(WARPS * 32)
    merge_pass_kernel(const KeyT* __restrict__ in, KeyT* __restrict__ out, long long n,
                      long long run_len, int K, const long long* __restrict__ table,
                      long long tpg, int* dev_err) {
  using G = MergeGeom<KeyT, WARPS>;
  constexpr int E = G::E;
  constexpr int S = G::S;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  KeyT* bufX = reinterpret_cast<KeyT*>(smem_raw);
  KeyT* bufY = bufX + G::XCAP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  KeyT* scr = bufY + G::YCAP + warp * kScratchItems;

  const long long t = blockIdx.x;
  const long long g = t / tpg, j = t % tpg;
  const long long gstart = g * run_len * K;
  const long long grest = n - gstart;
  const long long gsize = grest < run_len * K ? grest : run_len * K;
  const long long tiles_here = (gsize + S - 1) / S;

  // Segment of run `lane` for this tile (every warp computes the same).
  const bool act = lane < K;
  const long long rstart = gstart + (long long)lane * run_len;
  long long rlen = n - rstart;
  rlen = rlen < 0 ? 0 : (rlen > run_len ? run_len : rlen);
  long long lo = 0, hi = 0;
  if (act) {
    lo = (j == 0) ? 0 : table[t * K + lane];
    hi = (j + 1 < tiles_here) ? table[(t + 1) * K + lane] : rlen;
  }
  // The pivot rows must describe segments inside their runs whose lengths sum
  // to this tile's size; anything else would overrun the staging buffer.
  {
    const long long want = (gsize - j * S) < S ? (gsize - j * S) : S;
    const bool bad_seg = act && (lo < 0 || hi < lo || hi > rlen);
    long long sum = act ? hi - lo : 0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (__any_sync(0xffffffffu, bad_seg) || sum != want || K > kMaxFanout) {
      if (threadIdx.x == 0) set_device_error(dev_err, kDevErrInternal);
      return;                                          // uniform over the CTA
    }
  }
  const long long gsrc = rstart + lo;                  // first item, global index
  const int len = act ? (int)(hi - lo) : 0;
  const int head = act ? (int)(gsrc % E) : 0;          // items copied before the segment
  const int span = (head + len + E - 1) / E * E;       // staged extent, multiple of E
  int incl = span;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  const int place = incl - span;                       // staged extent start (multiple of E)
  const int my_off0 = place + head;
  // Bulk part: [gsrc - head, floor_E(gsrc + len)); the rest by plain loads.
  const long long bulk_lo = gsrc - head;
  const long long bulk_hi = (gsrc + len) / E * E;
  const unsigned bulk_bytes = (act && bulk_hi > bulk_lo) ? (unsigned)((bulk_hi - bulk_lo) * sizeof(KeyT)) : 0u;

  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (warp == 0) {
    unsigned total = bulk_bytes;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) mbar_arrive_expect_tx(&bar, total);
    __syncwarp();
    if (bulk_bytes) bulk_g2s(bufX + place, in + bulk_lo, bulk_bytes, &bar);
  } else if (warp == 1) {
    // Ragged ends, one segment at a time, consecutive lanes -> consecutive words.
    for (int r = 0; r < K; ++r) {
      const long long s_src = __shfl_sync(0xffffffffu, gsrc, r);
      const int s_len = __shfl_sync(0xffffffffu, len, r);
      const int s_off = __shfl_sync(0xffffffffu, my_off0, r);
      const long long s_bhi = __shfl_sync(0xffffffffu, bulk_hi, r);
      const long long s_blo = __shfl_sync(0xffffffffu, bulk_lo, r);
      const long long from = (s_bhi > s_blo) ? s_bhi : s_src;   // first item not bulk-copied
      const long long e = from + lane;
      if (e < s_src + s_len) bufX[s_off + (int)(e - s_src)] = in[e];
    }
  }
  const bool ok = mbar_wait_bounded(&bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) set_device_error(dev_err, kDevErrTimeout);
    return;
  }

  // ceil(log2 K) merge levels between the two buffers.
  int my_off = my_off0, my_len = len;
  int nseq = K;
  KeyT* src = bufX;
  KeyT* dst = bufY;
  while (nseq > 1) {
    cta_merge_level(src, dst, my_off, my_len, nseq, scr, warp, WARPS, lane);
    next_seq(my_off, my_len, nseq, lane);
    nseq = (nseq + 1) >> 1;
    __syncthreads();
    KeyT* tmp = src;
    src = dst;
    dst = tmp;
  }
  // src now holds the tile at offset my_off of lane 0 (0 when K > 1).
  const int m = __shfl_sync(0xffffffffu, my_len, 0);
  const KeyT* res = src + __shfl_sync(0xffffffffu, my_off, 0);
  KeyT* dstg = out + gstart + j * S;
  using V = typename MergeVec<KeyT>::T;
  const int nv = m / E;
  if (((size_t)res & 15) == 0) {
    const V* s4 = reinterpret_cast<const V*>(res);
    V* d4 = reinterpret_cast<V*>(dstg);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      V x = s4[i];
      if constexpr (XOUT) {
        uint32_t* w = reinterpret_cast<uint32_t*>(&x);
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = ordered_to_f32(w[c]);
      }
      d4[i] = x;
    }
  } else {
    for (int i = threadIdx.x; i < nv * E; i += blockDim.x) {
      KeyT x = res[i];
      if constexpr (XOUT) x = (KeyT)ordered_to_f32((uint32_t)x);
      dstg[i] = x;
    }
  }
  for (int i = nv * E + (int)threadIdx.x; i < m; i += blockDim.x) {
    KeyT x = res[i];
    if constexpr (XOUT) x = (KeyT)ordered_to_f32((uint32_t)x);
    dstg[i] = x;
  }
}

template <typename KeyT, int WARPS, bool XOUT>
static cudaError_t launch_merge_t(const void* in, void* out, long long n, long long run_len, int K,
                                  const long long* table, int* dev_err, cudaStream_t s) {
  const size_t smem = MergeGeom<KeyT, WARPS>::bytes();
  auto k = merge_pass_kernel<KeyT, WARPS, XOUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ntiles = num_tiles(sizeof(KeyT), n, run_len, K);
  const long long tpg = tiles_per_group(sizeof(KeyT), run_len, K);
  k<<<(unsigned)ntiles, WARPS * 32, smem, s>>>(static_cast<const KeyT*>(in), static_cast<KeyT*>(out),
                                              n, run_len, K, table, tpg, dev_err);
  return cudaGetLastError();
}

cudaError_t launch_merge_pass(int key_bytes, bool xout, const void* in, void* out, long long n,
                              long long run_len, int K, const long long* table, int* dev_err,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (key_bytes == 4) {
    if (xout)
      return launch_merge_t<uint32_t, kTileWarps32, true>(in, out, n, run_len, K, table, dev_err, s);
    return launch_merge_t<uint32_t, kTileWarps32, false>(in, out, n, run_len, K, table, dev_err, s);
  }
  return launch_merge_t<uint64_t, kTileWarps64, false>(in, out, n, run_len, K, table, dev_err, s);
}

}  // namespace mms
