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
// layout: after the call register j of lane l holds sorted item 32*l + (j ^ l).
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
      v[r] = upper ? (a > pa ? a : pa) : (a < pa ? a : pa);
      v[31 - r] = upper ? (b > pb ? b : pb) : (b < pb ? b : pb);
    }
#pragma unroll
    for (int ls = (1 << lg) >> 2; ls >= 1; ls >>= 1) {
      const bool up = (lane & ls) != 0;
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const KeyT p = shfl_xor(v[r], ls);
        v[r] = up ? (v[r] > p ? v[r] : p) : (v[r] < p ? v[r] : p);
      }
    }
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const bool f = (lg == 5) && ((lane & s) != 0);
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if ((k & s) == 0) cas_dir(v[k], v[k + s], f);
    }
  }
}

// Vector of 16 bytes.
template <typename KeyT>
struct Vec16;
template <>
struct Vec16<uint32_t> {
  using T = uint4;
  static constexpr int E = 4;
  __device__ static void unpack(const uint4& x, uint32_t* o) {
    o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
  }
  __device__ static uint4 pack(const uint32_t* o) { return make_uint4(o[0], o[1], o[2], o[3]); }
};
template <>
struct Vec16<uint64_t> {
  using T = ulonglong2;
  static constexpr int E = 2;
  __device__ static void unpack(const ulonglong2& x, uint64_t* o) {
    o[0] = x.x; o[1] = x.y;
  }
  __device__ static ulonglong2 pack(const uint64_t* o) { return make_ulonglong2(o[0], o[1]); }
};

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

// Coalesced 128-bit copy of `m` items from shared memory to global memory.
template <typename KeyT, bool XOUT>
__device__ __forceinline__ void cta_store_out(const KeyT* src, KeyT* dst, int m) {
  using V = Vec16<KeyT>;
  const int nv = m / V::E;
  const typename V::T* s4 = reinterpret_cast<const typename V::T*>(src);
  typename V::T* d4 = reinterpret_cast<typename V::T*>(dst);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    typename V::T x = s4[i];
    if constexpr (XOUT) {
      KeyT t[V::E];
      V::unpack(x, t);
#pragma unroll
      for (int c = 0; c < V::E; ++c) t[c] = xform_out<KeyT, XOUT>(t[c]);
      x = V::pack(t);
    }
    d4[i] = x;
  }
  for (int i = nv * V::E + (int)threadIdx.x; i < m; i += blockDim.x)
    dst[i] = xform_out<KeyT, XOUT>(src[i]);
}

template <typename KeyT, int WARPS, bool XIN, bool XOUT>
__global__ void __launch_bounds__(WARPS * 32)
    tile_sort_kernel(const KeyT* __restrict__ in, KeyT* out, long long n) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int T = WARPS * kBlockItems;
  KeyT* bufX = reinterpret_cast<KeyT*>(smem_raw);
  KeyT* bufY = bufX + T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  KeyT* scr = bufY + T + warp * kScratchItems;

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

  warp_sort_1024(v, lane);
  warp_store_block(bufX + warp * kBlockItems, kBlockItems, v, lane);
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
    cta_merge_level(src, dst, my_off, my_len, nseq, scr, warp, WARPS, lane);
    next_seq(my_off, my_len, nseq, lane);
    nseq = (nseq + 1) >> 1;
    __syncthreads();
    KeyT* t = src;
    src = dst;
    dst = t;
  }
  const long long trem = n - base;
  const int m = trem >= T ? T : (int)trem;
  cta_store_out<KeyT, XOUT>(src, out + base, m);
}

size_t tile_sort_smem_bytes(int key_bytes, int warps) {
  return (size_t)key_bytes * (2 * warps * kBlockItems + warps * kScratchItems);
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

cudaError_t launch_tile_sort(int key_bytes, bool xin, bool xout, const void* in, void* out,
                             long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (key_bytes == 4) {
    if (xin && xout) return launch_tile_sort_t<uint32_t, kTileWarps32, true, true>(in, out, n, s);
    if (xin) return launch_tile_sort_t<uint32_t, kTileWarps32, true, false>(in, out, n, s);
    return launch_tile_sort_t<uint32_t, kTileWarps32, false, false>(in, out, n, s);
  }
  return launch_tile_sort_t<uint64_t, kTileWarps64, false, false>(in, out, n, s);
}

}  // namespace mms
