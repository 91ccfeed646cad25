// tile_sort.cuh -- the CTA body of the base case of GPU Multiway Mergesort
// (Sec. 4.3 "Internal Memory Sort"), shared by the whole-array base case and
// the segmented (batched) one: a tile of T = 1024 * WARPS consecutive keys is
// sorted on its own, producing a sorted run the K-way merge rounds start from.
//
// The paper's base case is a per-warp shearsort of a 32 x 32 grid, extended
// by bitonic merges between warps.  Here each lane sorts the 32 keys it loaded
// with an in-register sorting network, the warp finishes its 1024 keys with
// bitonic merges through conflict-free transposes in its share of the tile
// buffer (the row/column transposes of shearsort, swizzled), and the CTA
// merges the warps' blocks with the same conflict-free block merge the merge
// rounds use.  HBM traffic: one coalesced 128-bit read and one coalesced
// 128-bit write of every key.
#pragma once

#include "mms_common.cuh"
#include "mms_kernels.cuh"

namespace mms {

// Sorting network over a lane's 32 registers (ascending): Batcher's odd-even
// merge sort (K. E. Batcher, "Sorting networks and their applications",
// AFIPS 1968), 191 compare-exchanges in 15 stages against the bitonic
// sorter's 240.  Stage (p, k) of the network compares items x and x + k for
// x = j + i with j running from k mod p in steps of 2k and i from 0 to k - 1,
// whenever both lie in the same block of 2p items.  Every index is a
// compile-time constant once the loops are unrolled, so each compare-exchange
// is register to register; within a stage about two of three pairs take the
// multiply-add form (by their ordinal in the stage), as in the other networks.
template <typename KeyT, typename M>
__device__ __forceinline__ void lane_sort32(KeyT (&v)[32], const M& c) {
#pragma unroll
  for (int lp = 0; lp < 5; ++lp) {
#pragma unroll
    for (int lk = lp; lk >= 0; --lk) {
      const int p = 1 << lp, k = 1 << lk;
      const int j0 = k & (p - 1);                      // first j of the stage: k mod p
      int ord = 0;                                     // ordinal of the pair in its stage
#pragma unroll
      for (int x = 0; x < 31; ++x) {                   // x = j + i, j = j0 + 2kt, i < k
        if (x + k < 32 && x >= j0 && ((x - j0) & (2 * k - 1)) < k &&
            (x >> (lp + 1)) == ((x + k) >> (lp + 1))) {
          cas_mix(v[x], v[x + k], ord, c);
          ++ord;
        }
      }
    }
  }
}

// Blocked -> striped through `scratch` (16-byte aligned, 1024 items), with the
// second half of every block of R rows read backwards.  On return register k
// of lane l holds item 32k + l of the sequence in which every block of R rows
// is its first R/2 rows in order followed by its last R/2 rows in reverse
// (row qR + R - 1 - i into register qR + R/2 + i, column 31 - l into lane l):
// a bitonic sequence when both halves of the block are ascending, so an
// ascending half-cleaner cascade sorts it, with no per-lane directions.  Each
// lane writes its row as 16-byte chunks XOR-swizzled by row & 7, and each
// register load reads 32 distinct words of one row: no bank conflicts.
template <int R, typename KeyT>
__device__ __forceinline__ void blocked_to_striped_rev(KeyT (&v)[32], KeyT* scratch, int lane) {
  constexpr int E = Vec16<KeyT>::E;
  const uint32_t row = smem_u32addr(scratch + 32 * lane);
  const int sw = lane & 7;
#pragma unroll
  for (int ch = 0; ch < 32 / E; ++ch)
    sts128(row + (uint32_t)((ch ^ sw) * E * (int)sizeof(KeyT)), &v[ch * E]);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int kq = k % R;
    const bool rev = kq >= R / 2;
    const int src = rev ? k - kq + R - 1 - (kq - R / 2) : k;   // source row
    const int w = rev ? 31 - lane : lane;                      // source column
    v[k] = scratch[32 * src + (w ^ (E * (src & 7)))];
  }
  __syncwarp();
}

// One level of the warp sort: every block of R rows, whose two halves are
// each sorted, becomes sorted (blocked layout in and out).
template <int R, typename KeyT, typename M>
__device__ __forceinline__ void warp_merge_rows(KeyT (&v)[32], KeyT* scratch, int lane,
                                                const M& c) {
  blocked_to_striped_rev<R>(v, scratch, lane);
  striped_stages<R / 2>(v, c);                       // strides 16R .. 32
  striped_to_blocked(v, scratch, 32, lane);
  blocked_stages<false>(v, lane, c);                 // strides 16 .. 1
}

// Sorts 1024 keys held as 32 per lane (any assignment): each lane sorts its
// 32 keys (a row), then levels of 64, 128, 256, 512 and 1024 keys merge pairs
// of sorted blocks with bitonic cascades -- strides of 32 and more between
// registers in the striped layout, the rest inside the lane -- through
// conflict-free transposes in the warp's 1024-item `scratch` (no shuffles).
// After the call register j of lane l holds sorted item 32*l + (j ^
// flip_mask(l)), the layout warp_store_block writes out.
template <typename KeyT>
__device__ __forceinline__ void warp_sort_1024(KeyT (&v)[32], KeyT* scratch, int lane) {
  const TileMix c = mad_ones<TileMix>();
  lane_sort32(v, c);
  warp_merge_rows<2>(v, scratch, lane, c);
  warp_merge_rows<4>(v, scratch, lane, c);
  warp_merge_rows<8>(v, scratch, lane, c);
  warp_merge_rows<16>(v, scratch, lane, c);
  blocked_to_striped_rev<32>(v, scratch, lane);      // the last level: the block merge's network
  striped_stages<16>(v, c);
  striped_to_blocked(v, scratch, 32, lane);
  blocked_stages<true>(v, lane, c);
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
  // A destination off the 16-byte grid (a segment of a batch may start
  // anywhere) is written with plain coalesced stores.
  const int body = (((uintptr_t)dst & 15u) == 0) ? m / E * E : 0;
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0 && body > 0) bulk_s2g_and_wait(dst, src, (unsigned)(body * sizeof(KeyT)));
  for (int i = body + (int)threadIdx.x; i < m; i += blockDim.x) dst[i] = src[i];
}

// Everything after the load up to the sorted tile in shared memory: warp
// sorts, then the CTA merge levels.  Returns the buffer (bufX or bufY of
// smem_raw) that holds the tile's keys in order; its first min(T, n - base)
// entries are the tile's.  xout: write the last level's output as floats.
template <typename KeyT, int WARPS>
__device__ __forceinline__ KeyT* tile_sort_smem(KeyT (&v)[32], long long n, long long base,
                                                bool xout, unsigned char* smem_raw) {
  constexpr int T = WARPS * kBlockItems;
  KeyT* bufX = reinterpret_cast<KeyT*>(smem_raw);
  KeyT* bufY = bufX + T + kTileSlack;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // The previous tile of a persistent CTA has been read out of shared memory
  // before the warps use it as transpose scratch.
  __syncthreads();
  warp_sort_1024(v, bufX + warp * kBlockItems, lane);
  if constexpr (WARPS == 1) {
    warp_store_block<KeyT>(bufX, kBlockItems, v, lane, xout);
    return bufX;
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
    cta_merge_level<KeyT, TileMix>(src, dst, my_off, my_len, nseq, warp, WARPS, lane,
                                   xout && nseq <= 2);
    next_seq<KeyT>(my_off, my_len, nseq, lane);
    nseq = (nseq + 1) >> 1;
    __syncthreads();
    KeyT* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// Everything after the load: the sort in shared memory and the store of the tile.
template <typename KeyT, int WARPS>
__device__ __forceinline__ void tile_sort_finish(KeyT (&v)[32], KeyT* out, long long n,
                                                 long long base, bool xout,
                                                 unsigned char* smem_raw) {
  constexpr int T = WARPS * kBlockItems;
  KeyT* res = tile_sort_smem<KeyT, WARPS>(v, n, base, xout, smem_raw);
  const long long trem = n - base;
  const int m = trem >= T ? T : (int)trem;
  cta_store_tile(res, out + base, m);
}

// Loads this warp's 1024 keys of the tile of 1024 * WARPS keys that starts at
// `base` (32 per lane, any assignment; pads past n), through the float order
// transform when XIN.
template <typename KeyT, int WARPS, bool XIN>
__device__ __forceinline__ void tile_load(const KeyT* __restrict__ in, long long n, long long base,
                                          KeyT (&v)[32]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wbase = base + (long long)warp * kBlockItems;
  const long long rem = n - wbase;
  const int cnt = rem <= 0 ? 0 : (rem >= kBlockItems ? kBlockItems : (int)rem);

  using V = Vec16<KeyT>;
  constexpr int NV = 32 / V::E;          // 16-byte vectors per lane
  if (cnt == kBlockItems && ((uintptr_t)(in + wbase) & 15u) == 0) {
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
}

// Sorts the tile of 1024 * WARPS keys of in[0, n) that starts at `base` into
// the same positions of out (in == out allowed): the CTA body of the base case.
template <typename KeyT, int WARPS, bool XIN>
__device__ __forceinline__ void tile_sort_tile(const KeyT* __restrict__ in, KeyT* out, long long n,
                                               long long base, bool xout,
                                               unsigned char* smem_raw) {
  KeyT v[32];
  tile_load<KeyT, WARPS, XIN>(in, n, base, v);
  tile_sort_finish<KeyT, WARPS>(v, out, n, base, xout, smem_raw);
}

// Base case of the key-value sort: 32-bit keys (floats through the order
// transform when XIN) are read and turned into unique 64-bit composites
// (ordered key << 32 | pos0 + position in the array), whose ascending order is the
// stable key order; tiles of composites are then sorted like 64-bit keys.
template <int WARPS, bool XIN>
__device__ __forceinline__ void tile_sort_composite_tile(const uint32_t* __restrict__ in,
                                                         uint64_t* out, long long n,
                                                         long long base, long long pos0,
                                                         unsigned char* smem_raw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wbase = base + (long long)warp * kBlockItems;
  const long long rem = n - wbase;
  const int cnt = rem <= 0 ? 0 : (rem >= kBlockItems ? kBlockItems : (int)rem);
  uint64_t v[32];
  if (cnt == kBlockItems && ((uintptr_t)(in + wbase) & 15u) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(in + wbase);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 x = __ldg(src + q * 32 + lane);
      const uint32_t k[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t key = XIN ? f32_to_ordered(k[c]) : k[c];
        const uint64_t pos = (uint64_t)(pos0 + wbase + q * 128 + lane * 4 + c);
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
          x = ((uint64_t)key << 32) | (uint64_t)(pos0 + wbase + e);
        }
        v[q * 4 + c] = x;
      }
    }
  }
  tile_sort_finish<uint64_t, WARPS>(v, out, n, base, false, smem_raw);
}

}  // namespace mms
