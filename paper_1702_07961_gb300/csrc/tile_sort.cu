// tile_sort.cu -- the whole-array base case: one CTA per tile, running the
// CTA body of tile_sort.cuh.
#include "tile_sort.cuh"

namespace mms {

template <typename KeyT, int WARPS, bool XIN, bool XOUT>
__global__ void __launch_bounds__(WARPS * 32, (MinBlocks<KeyT, WARPS>::value))
    tile_sort_kernel(const KeyT* __restrict__ in, KeyT* out, long long n) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int T = WARPS * kBlockItems;
  griddep_launch_dependents();                    // the first splitter may get resident early
  tile_sort_tile<KeyT, WARPS, XIN>(in, out, n, (long long)blockIdx.x * T, XOUT, smem_raw);
}

// Base case of the key-value sort: 32-bit keys -> sorted tiles of unique
// 64-bit composites (ordered key << 32 | position in the array).
template <int WARPS, bool XIN>
__global__ void __launch_bounds__(WARPS * 32, (MinBlocks<uint64_t, WARPS>::value))
    tile_sort_composite_kernel(const uint32_t* __restrict__ in, uint64_t* out, long long n) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int T = WARPS * kBlockItems;
  griddep_launch_dependents();
  tile_sort_composite_tile<WARPS, XIN>(in, out, n, (long long)blockIdx.x * T, 0, smem_raw);
}

size_t tile_sort_smem_bytes(int key_bytes, int warps) {
  return (size_t)key_bytes * 2 * (warps * kBlockItems + kTileSlack);
}

template <typename KeyT, int WARPS, bool XIN, bool XOUT>
static cudaError_t launch_tile_sort_t(const void* in, void* out, long long n, cudaStream_t s) {
  const size_t smem = tile_sort_smem_bytes(sizeof(KeyT), WARPS);
  auto k = tile_sort_kernel<KeyT, WARPS, XIN, XOUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long T = (long long)WARPS * kBlockItems;
  const unsigned grid = (unsigned)((n + T - 1) / T);
  k<<<grid, WARPS * 32, smem, s>>>(static_cast<const KeyT*>(in), static_cast<KeyT*>(out), n);
  return cudaGetLastError();
}

template <int WARPS>
static cudaError_t launch_tile_sort_w(int key_bytes, bool xin, bool xout, const void* in, void* out,
                                      long long n, cudaStream_t s) {
  if (key_bytes == 8 && WARPS == 8) return cudaErrorInvalidValue;
  if (key_bytes == 4) {
    if (xin && xout) return launch_tile_sort_t<uint32_t, WARPS, true, true>(in, out, n, s);
    if (xin) return launch_tile_sort_t<uint32_t, WARPS, true, false>(in, out, n, s);
    return launch_tile_sort_t<uint32_t, WARPS, false, false>(in, out, n, s);
  }
  if constexpr (WARPS != 8) return launch_tile_sort_t<uint64_t, WARPS, false, false>(in, out, n, s);
  return cudaErrorInvalidValue;
}

template <int WARPS, bool XIN>
static cudaError_t launch_composite_t(const void* in, void* out, long long n, cudaStream_t s) {
  const size_t smem = tile_sort_smem_bytes(8, WARPS);
  auto k = tile_sort_composite_kernel<WARPS, XIN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long T = (long long)WARPS * kBlockItems;
  const unsigned grid = (unsigned)((n + T - 1) / T);
  k<<<grid, WARPS * 32, smem, s>>>(static_cast<const uint32_t*>(in), static_cast<uint64_t*>(out), n);
  return cudaGetLastError();
}

cudaError_t launch_tile_sort_composite(int tile_warps, bool xin, const void* keys32, void* out64,
                                       long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (tile_warps == 4)
    return xin ? launch_composite_t<4, true>(keys32, out64, n, s) : launch_composite_t<4, false>(keys32, out64, n, s);
  if (tile_warps == 2)
    return xin ? launch_composite_t<2, true>(keys32, out64, n, s) : launch_composite_t<2, false>(keys32, out64, n, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tile_sort(int key_bytes, int tile_warps, bool xin, bool xout, const void* in,
                             void* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  switch (tile_warps) {
    case 2: return launch_tile_sort_w<2>(key_bytes, xin, xout, in, out, n, s);
    case 4: return launch_tile_sort_w<4>(key_bytes, xin, xout, in, out, n, s);
    case 8: return launch_tile_sort_w<8>(key_bytes, xin, xout, in, out, n, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mms
