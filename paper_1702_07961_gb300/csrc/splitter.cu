// splitter.cu -- the whole-array splitter: one warp per output tile of a
// merge round, running splitter_row of splitter.cuh.
#include "splitter.cuh"

namespace mms {

template <typename KeyT>
__global__ void __launch_bounds__(128)
    splitter_kernel(const KeyT* __restrict__ in, long long n, long long run_len, int K,
                    long long S, long long tpg, long long ntiles, long long* __restrict__ table) {
  const long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= ntiles) return;                      // warp-uniform
  splitter_row<KeyT>(in, n, run_len, K, S, t / tpg, t % tpg, table + t * K);
}

cudaError_t launch_splitter(int key_bytes, long long S, const void* in, long long n,
                            long long run_len, int K, long long* table, cudaStream_t s) {
  const long long ntiles = num_tiles(S, n, run_len, K);
  if (ntiles <= 0) return cudaSuccess;
  const long long tpg = tiles_per_group(S, run_len, K);
  const unsigned grid = (unsigned)((ntiles + 3) / 4);
  if (key_bytes == 4)
    splitter_kernel<uint32_t><<<grid, 128, 0, s>>>(static_cast<const uint32_t*>(in), n, run_len, K,
                                                   S, tpg, ntiles, table);
  else
    splitter_kernel<uint64_t><<<grid, 128, 0, s>>>(static_cast<const uint64_t*>(in), n, run_len, K,
                                                   S, tpg, ntiles, table);
  return cudaGetLastError();
}

}  // namespace mms
