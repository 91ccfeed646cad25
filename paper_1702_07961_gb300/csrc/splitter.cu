// splitter.cu -- the whole-array splitter: one warp per output tile of a
// merge round, running splitter_row of splitter.cuh.
#include "splitter.cuh"

namespace mms {

// Warps per splitter CTA: 4 measured fastest on GB300 at 10^8 u32 keys
// (splitters 0.302 ms, against 0.306 with 2 warps and 0.307 with 8).
constexpr int kSplitterWarps = 4;

template <typename KeyT, int W, typename Idx>
__global__ void __launch_bounds__(32 * kSplitterWarps)
    splitter_kernel(const KeyT* __restrict__ in, long long n, long long run_len, int K,
                    long long S, long long tpg, long long ntiles, long long* __restrict__ table) {
  const int lane = threadIdx.x & 31;
  const int gb = lane & ~(W - 1);                 // first lane of this lane group
  const unsigned gm = W == 32 ? 0xffffffffu : (((1u << W) - 1u) << gb);
  griddep_wait();                                 // the runs are the previous kernel's output
  griddep_launch_dependents();
  const long long t = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / W) + gb / W;
  if (t >= ntiles) return;                        // uniform over the lane group
  splitter_row<KeyT, W, Idx>(in, n, run_len, K, S, t / tpg, t % tpg, table + t * K, gm, gb);
}

template <typename KeyT, int W>
static cudaError_t launch_w(const void* in, long long n, long long run_len, int K, long long S,
                            long long tpg, long long ntiles, long long* table, cudaStream_t s,
                            bool pdl) {
  const long long per_block = kSplitterWarps * (32 / W);   // warps of 32 / W tiles each
  const unsigned grid = (unsigned)((ntiles + per_block - 1) / per_block);
  const KeyT* kin = static_cast<const KeyT*>(in);
  // 32-bit counts and positions while no probe can pass 2^31 (n < 2^30)
  if (n < (1ll << 30))
    return launch_k(splitter_kernel<KeyT, W, int>, dim3(grid), dim3(32 * kSplitterWarps), 0, s, pdl, kin, n, run_len,
                    K, S, tpg, ntiles, table);
  return launch_k(splitter_kernel<KeyT, W, long long>, dim3(grid), dim3(32 * kSplitterWarps), 0, s, pdl, kin, n,
                  run_len, K, S, tpg, ntiles, table);
}

// One output tile per warp (W = 32).  Packing 32 / W tiles into a warp's lane
// groups was measured slower on GB300 (10^8 u32: 0.65 ms of splitters at
// K = 4 against 0.47 ms): the search is bound by the latency of its
// dependent loads and needs the independent warps, and lane groups of one
// warp diverge in their per-tile pop loops.
cudaError_t launch_splitter(int key_bytes, long long S, const void* in, long long n,
                            long long run_len, int K, long long* table, cudaStream_t s, bool pdl) {
  const long long ntiles = num_tiles(S, n, run_len, K);
  if (ntiles <= 0) return cudaSuccess;
  if (K < 2 || K > kMaxFanout) return cudaErrorInvalidValue;
  const long long tpg = tiles_per_group(S, run_len, K);
  if (key_bytes == 4) return launch_w<uint32_t, 32>(in, n, run_len, K, S, tpg, ntiles, table, s, pdl);
  return launch_w<uint64_t, 32>(in, n, run_len, K, S, tpg, ntiles, table, s, pdl);
}

}  // namespace mms
