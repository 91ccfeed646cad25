// tile_sort.cu -- base case of GPU Multiway Mergesort (Sec. 4.3 "Internal
// Memory Sort"): every tile of T = 1024 * WARPS consecutive keys is sorted on
// its own, producing the sorted runs the K-way merge rounds start from.
//
// The paper's base case is a per-warp shearsort of a 32 x 32 grid, extended
// by bitonic merges between warps.  Here each lane sorts the 32 keys it loaded
// with an in-register sorting network, the warp finishes its 1024 keys with
// register/shuffle bitonic merges (no shared memory, so no bank traffic), and
// the CTA merges the warps' blocks with the same conflict-free block merge the
// merge rounds use.  HBM traffic: one coalesced 128-bit read and one coalesced
// 128-bit write of every key.
#include "mms_common.cuh"
#include "mms_kernels.cuh"

namespace mms {

// Bitonic sorting network over a lane's 32 registers (ascending).
template <typename KeyT>
__device__ __forceinline__ void lane_sort32(KeyT (&v)[32]) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int ixj = i ^ j;
        if (ixj > i) {
          if ((i & k) == 0)
            cas(v[i], v[ixj]);
          else
            cas(v[ixj], v[i]);
        }
      }
    }
  }
}

// Sorts 1024 keys held as 32 per lane (any assignment) into the blocked
// layout: after the call register j of lane l holds sorted item
// 32*l + (j ^ flip_mask(l)), the layout warp_store_block writes out.
// Level lg merges runs of 2^(lg-1) lanes: a reversed-partner stage across the
// run pair, lane half-cleaners by shuffle, then in-lane half-cleaners.
template <typename KeyT>
__device__ __forceinline__ void warp_sort_1024(KeyT (&v)[32], int lane) {
  lane_sort32(v);
#pragma unroll
  for (int lg = 1; lg <= 5; ++lg) {
    const int mask = (1 << lg) - 1;
    const bool upper = (lane & (1 << (lg - 1))) != 0;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const KeyT a = v[r], b = v[31 - r];
      const KeyT pa = shfl_xor(b, mask);   // partner's register 31-r pairs with my r
      const KeyT pb = shfl_xor(a, mask);   // partner's register r pairs with my 31-r
      v[r] = upper ? kmax(a, pa) : kmin(a, pa);
      v[31 - r] = upper ? kmax(b, pb) : kmin(b, pb);
    }
#pragma unroll
    for (int ls = (1 << lg) >> 2; ls >= 1; ls >>= 1) {
      const bool up = (lane & ls) != 0;
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const KeyT p = shfl_xor(v[r], ls);
        v[r] = up ? kmax(v[r], p) : kmin(v[r], p);
      }
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const bool f = (lg == 5) && ((flip_mask<KeyT>(lane) & s) != 0);
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if ((k & s) == 0) cas_dir(v[k], v[k + s], f);
    }
  }
}

template <typename KeyT, bool XIN>
__device__ __forceinline__ KeyT xform_in(KeyT k) {
  if constexpr (XIN) return (KeyT)f32_to_ordered((uint32_t)k);
  return k;
}
template <typename KeyT, bool XOUT>
__device__ __forceinline__ KeyT xform_out(KeyT k) {
  if constexpr (XOUT) return (KeyT)ordered_to_f32((uint32_t)k);
  return k;
}

// Writes the sorted tile src[0, m) to global memory: one TMA bulk store of the
// 16-byte-aligned body, plain stores for the < 16-byte tail.  Every thread
// must call it (it contains a barrier).
template <typename KeyT>
__device__ __forceinline__ void cta_store_tile(const KeyT* src, KeyT* dst, int m) {
  constexpr int E = 16 / sizeof(KeyT);
  const int body = m / E * E;
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0 && body > 0) bulk_s2g_and_wait(dst, src, (unsigned)(body * sizeof(KeyT)));
  for (int i = body + (int)threadIdx.x; i < m; i += blockDim.x) dst[i] = src[i];
}

// Everything after the load: warp sorts, CTA merge levels, store of the tile.
template <typename KeyT, int WARPS, bool XOUT>
__device__ __forceinline__ void tile_sort_finish(KeyT (&v)[32], KeyT* out, long long n,
                                                 long long base, unsigned char* smem_raw) {
  constexpr int T = WARPS * kBlockItems;
  KeyT* bufX = reinterpret_cast<KeyT*>(smem_raw);
  KeyT* bufY = bufX + T + kTileSlack;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  warp_sort_1024(v, lane);
  const long long trem = n - base;
  const int m = trem >= T ? T : (int)trem;
  if constexpr (WARPS == 1) {
    warp_store_block<KeyT>(bufX, kBlockItems, v, lane, XOUT);
    cta_store_tile(bufX, out + base, m);
    return;
  }
  warp_store_block<KeyT>(bufX + warp * kBlockItems, kBlockItems, v, lane, false);
  __syncthreads();

  // CTA levels: merge the warps' sorted blocks pairwise up to the tile.
  int my_off = lane * kBlockItems;
  int my_len = 0;
  {
    const long long r2 = n - (base + (long long)lane * kBlockItems);
    my_len = (lane < WARPS && r2 > 0) ? (r2 >= kBlockItems ? kBlockItems : (int)r2) : 0;
  }
  KeyT* src = bufX;
  KeyT* dst = bufY;
  int nseq = WARPS;
  while (nseq > 1) {
    cta_merge_level<KeyT>(src, dst, my_off, my_len, nseq, warp, WARPS, lane, XOUT && nseq <= 2);
    next_seq<KeyT>(my_off, my_len, nseq, lane);
    nseq = (nseq + 1) >> 1;
    __syncthreads();
    KeyT* t = src;
    src = dst;
    dst = t;
  }
  cta_store_tile(src, out + base, m);
}

template <typename KeyT, int WARPS, bool XIN, bool XOUT>
__global__ void __launch_bounds__(WARPS * 32, (MinBlocks<KeyT, WARPS>::value))
    tile_sort_kernel(const KeyT* __restrict__ in, KeyT* out, long long n) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int T = WARPS * kBlockItems;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = (long long)blockIdx.x * T;
  const long long wbase = base + (long long)warp * kBlockItems;
  const long long rem = n - wbase;
  const int cnt = rem <= 0 ? 0 : (rem >= kBlockItems ? kBlockItems : (int)rem);

  using V = Vec16<KeyT>;
  constexpr int NV = 32 / V::E;          // 16-byte vectors per lane
  KeyT v[32];
  if (cnt == kBlockItems) {
    const typename V::T* src = reinterpret_cast<const typename V::T*>(in + wbase);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const typename V::T x = __ldg(src + q * 32 + lane);
      KeyT t[V::E];
      V::unpack(x, t);
#pragma unroll
      for (int c = 0; c < V::E; ++c) v[q * V::E + c] = xform_in<KeyT, XIN>(t[c]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
      for (int c = 0; c < V::E; ++c) {
        const int e = q * 32 * V::E + lane * V::E + c;
        v[q * V::E + c] = e < cnt ? xform_in<KeyT, XIN>(in[wbase + e]) : key_pad<KeyT>();
      }
    }
  }
  tile_sort_finish<KeyT, WARPS, XOUT>(v, out, n, base, smem_raw);
}

// Base case of the key-value sort: 32-bit keys (floats through the order
// transform when XIN) are read and turned into unique 64-bit composites
// (ordered key << 32 | position in the array), whose ascending order is the
// stable key order; tiles of composites are then sorted like 64-bit keys.
template <int WARPS, bool XIN>
__global__ void __launch_bounds__(WARPS * 32, (MinBlocks<uint64_t, WARPS>::value))
    tile_sort_composite_kernel(const uint32_t* __restrict__ in, uint64_t* out, long long n) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int T = WARPS * kBlockItems;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = (long long)blockIdx.x * T;
  const long long wbase = base + (long long)warp * kBlockItems;
  const long long rem = n - wbase;
  const int cnt = rem <= 0 ? 0 : (rem >= kBlockItems ? kBlockItems : (int)rem);
  uint64_t v[32];
  if (cnt == kBlockItems) {
    const uint4* src = reinterpret_cast<const uint4*>(in + wbase);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 x = __ldg(src + q * 32 + lane);
      const uint32_t k[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t key = XIN ? f32_to_ordered(k[c]) : k[c];
        const uint64_t pos = (uint64_t)(wbase + q * 128 + lane * 4 + c);
        v[q * 4 + c] = ((uint64_t)key << 32) | pos;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int e = q * 128 + lane * 4 + c;
        uint64_t x = key_pad<uint64_t>();
        if (e < cnt) {
          const uint32_t key = XIN ? f32_to_ordered(in[wbase + e]) : in[wbase + e];
          x = ((uint64_t)key << 32) | (uint64_t)(wbase + e);
        }
        v[q * 4 + c] = x;
      }
    }
  }
  tile_sort_finish<uint64_t, WARPS, false>(v, out, n, base, smem_raw);
}

// Two tile buffers, each with room for a partial block's transpose past the
// tile's end (the last, partial tile of an array).
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
