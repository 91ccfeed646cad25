// merge_pass.cu -- one K-way merge round over a whole array: one CTA per
// output tile, running the CTA body of merge_tile.cuh (the CTA merge tree, or
// the heap-free partition variant).
#include "merge_tile.cuh"

namespace mms {

size_t merge_pass_smem_bytes(int key_bytes, int warps, int K) {
  return merge_pass_smem_bytes_impl(key_bytes, warps, K);
}

template <typename KeyT, int WARPS, bool XOUT, bool PART>
__global__ void __launch_bounds__(WARPS * 32, (PART ? kPartitionMinBlocks : MinBlocks<KeyT, WARPS>::value))
    merge_pass_kernel(const KeyT* __restrict__ in, KeyT* __restrict__ out, long long n,
                      long long run_len, int K, const long long* __restrict__ table,
                      long long tpg, int S, int* dev_err, int test_timeout) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int cap = MergeGeom<KeyT, WARPS>::cap(K);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + sizeof(KeyT) * 2 * (size_t)cap);
  const long long t = blockIdx.x;
  const unsigned tq = (unsigned)blockIdx.x / (unsigned)tpg;    // tiles and tpg fit in 32 bits
  const long long g = tq, j = (long long)((unsigned)blockIdx.x - tq * (unsigned)tpg);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    if (test_timeout) mbar_init(bar + 1, 1);   // the test hook's barrier (bar[1] is spare)
  }
  griddep_wait();                                // the pivot table and the runs: earlier kernels'
  griddep_launch_dependents();
  merge_tile<KeyT, WARPS, PART>(in, out, n, run_len, K, g, j, table + t * K, table + (t + 1) * K,
                                XOUT, dev_err, smem_raw, bar, 0u, S, test_timeout != 0);
}

template <typename KeyT, int WARPS, bool XOUT, bool PART = false>
static cudaError_t launch_merge_t(long long S, const void* in, void* out, long long n,
                                  long long run_len, int K, const long long* table, int* dev_err,
                                  cudaStream_t s, bool test_timeout, bool pdl) {
  const size_t smem = PART ? MergeGeom<KeyT, WARPS>::bytes_partition(K) : MergeGeom<KeyT, WARPS>::bytes(K);
  auto k = merge_pass_kernel<KeyT, WARPS, XOUT, PART>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (S < kBlockItems || S > (long long)WARPS * kBlockItems || S % kBlockItems) return cudaErrorInvalidValue;
  const long long ntiles = num_tiles(S, n, run_len, K);
  long long tpg = tiles_per_group(S, run_len, K);
  if (tpg > 0xFFFFFFFFll) tpg = 0xFFFFFFFFll;   // more than the grid: every tile is in group 0
  return launch_k(k, dim3((unsigned)ntiles), dim3(WARPS * 32), smem, s, pdl,
                  static_cast<const KeyT*>(in), static_cast<KeyT*>(out), n, run_len, K, table, tpg,
                  (int)S, dev_err, test_timeout ? 1 : 0);
}

cudaError_t launch_merge_pass(int key_bytes, int tile_warps, long long S, bool xout, const void* in,
                              void* out, long long n, long long run_len, int K,
                              const long long* table, int* dev_err, cudaStream_t s,
                              bool test_timeout, bool pdl, bool partition) {
  if (n <= 0) return cudaSuccess;
  if (partition) {   // the heap-free variant: default tile geometry only
    if (tile_warps != default_tile_warps(key_bytes)) return cudaErrorInvalidValue;
    if (key_bytes == 4)
      return xout ? launch_merge_t<uint32_t, 8, true, true>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl)
                  : launch_merge_t<uint32_t, 8, false, true>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl);
    return launch_merge_t<uint64_t, 4, false, true>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl);
  }
  if (key_bytes == 4) {
    if (tile_warps == 8)
      return xout ? launch_merge_t<uint32_t, 8, true>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl)
                  : launch_merge_t<uint32_t, 8, false>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl);
    if (tile_warps == 4)
      return xout ? launch_merge_t<uint32_t, 4, true>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl)
                  : launch_merge_t<uint32_t, 4, false>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl);
    return cudaErrorInvalidValue;
  }
  if (tile_warps == 4) return launch_merge_t<uint64_t, 4, false>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl);
  if (tile_warps == 2) return launch_merge_t<uint64_t, 2, false>(S, in, out, n, run_len, K, table, dev_err, s, test_timeout, pdl);
  return cudaErrorInvalidValue;
}

}  // namespace mms
