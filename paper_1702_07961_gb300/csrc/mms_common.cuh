// mms_common.cuh -- shared device building blocks of the GPU Multiway Mergesort
// kernels for sm_103a: key traits, the order-preserving float transform,
// compare-exchange, the conflict-free warp merge of a 1024-item block, the
// warp co-rank (merge-path) search in shared memory, and TMA/mbarrier PTX.
//
// Shared-memory discipline (Sec. 3.2 and Sec. 5.2): every shared-memory access
// a warp makes is either 32 consecutive items (any base: one bank each), a
// fixed permutation of banks inside 32-word windows (padded rows, XOR
// swizzle), or a probe at an odd stride -- never a data-dependent gather -- so
// no input can cause a bank conflict.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mms_kernels.cuh"

namespace mms {

constexpr int kWarpSize = 32;
constexpr int kBlockItems = 1024;       // one warp block: 32 lanes x 32 registers
constexpr int kScratchRow = 33;         // padded row of the per-warp transpose scratch
constexpr int kScratchItems = 32 * kScratchRow;

// ---------------------------------------------------------------------------
// Keys.  KeyT is uint32_t (u32 keys, and f32 keys after the transform) or
// uint64_t.  The all-ones pattern is the padding value: for key-only sorting
// a pad that ties with a real all-ones key is bit-identical to it.
// ---------------------------------------------------------------------------
template <typename KeyT>
__device__ __forceinline__ KeyT key_pad() { return ~KeyT(0); }

// IEEE-754 binary32 -> unsigned order-preserving bits (totalOrder on bit
// patterns): negative values are complemented, non-negative ones get the
// sign bit set.  The inverse undoes it exactly, so output bits are unchanged.
__device__ __forceinline__ uint32_t f32_to_ordered(uint32_t x) {
  return x ^ ((uint32_t)((int32_t)x >> 31) | 0x80000000u);
}
__device__ __forceinline__ uint32_t ordered_to_f32(uint32_t y) {
  return y ^ ((uint32_t)((int32_t)~y >> 31) | 0x80000000u);
}

template <typename KeyT>
__device__ __forceinline__ void cas(KeyT& a, KeyT& b) {
  const KeyT lo = a < b ? a : b;
  const KeyT hi = a < b ? b : a;
  a = lo;
  b = hi;
}

// Compare-exchange whose direction is chosen per lane: with flip set the
// larger key goes to a.  Flipping every stage of a bitonic merge whose stride
// bit is set in the lane id leaves the lane's sorted items XOR-permuted by the
// lane id, which makes the following shared-memory store conflict-free.
template <typename KeyT>
__device__ __forceinline__ void cas_dir(KeyT& a, KeyT& b, bool flip) {
  const KeyT lo = a < b ? a : b;
  const KeyT hi = a < b ? b : a;
  a = flip ? hi : lo;
  b = flip ? lo : hi;
}

template <typename KeyT>
__device__ __forceinline__ KeyT shfl_xor(KeyT v, int mask) {
  return __shfl_xor_sync(0xffffffffu, v, mask);
}

// ---------------------------------------------------------------------------
// Shared-memory loads that the compiler may not merge: the two halves of a
// register that straddles the A/B boundary are fetched by two instructions,
// each with its own lanes active, so neither can conflict.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void lds_pred(uint32_t& v, const uint32_t* p, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.shared.b32 %0, [%1];\n\t}\n"
      : "+r"(v)
      : "r"(smem_u32addr(p)), "r"((int)pred)
      : "memory");
}
__device__ __forceinline__ void lds_pred(uint64_t& v, const uint64_t* p, bool pred) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.shared.b64 %0, [%1];\n\t}\n"
      : "+l"(v)
      : "r"(smem_u32addr(p)), "r"((int)pred)
      : "memory");
}

// ---------------------------------------------------------------------------
// Warp co-rank (merge path) search, Sec. 4.1 specialised to two lists:
// returns the number of items of A among the first d items of merge(A, B),
// ties taken from A (stable).  32-ary: each round all lanes probe positions
// at an odd stride (distinct banks), a ballot narrows the range 32-fold.
// ---------------------------------------------------------------------------
template <typename KeyT>
__device__ __forceinline__ int warp_corank(const KeyT* A, int lenA, const KeyT* B, int lenB,
                                           int d, int lane) {
  int lo = d - lenB > 0 ? d - lenB : 0;
  int hi = d < lenA ? d : lenA;
  while (hi > lo) {
    const int range = hi - lo;
    const int step = ((range + 31) >> 5) | 1;
    const int i = lo + lane * step;
    bool p = true;                                 // positions >= hi count as "true"
    if (i < hi) p = A[i] > B[d - 1 - i];           // A[i] comes after B[d-1-i]
    const unsigned bal = __ballot_sync(0xffffffffu, p);
    if (bal == 0u) {
      lo = lo + 31 * step + 1;
    } else {
      const int f = __ffs(bal) - 1;
      if (f == 0) {
        hi = lo;
      } else {
        const int nlo = lo + (f - 1) * step + 1;
        const int top = lo + f * step;
        hi = top < hi ? top : hi;
        lo = nlo;
      }
    }
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Warp merge of one output block (Sec. 4.2 "I/O Efficient Merging", merging
// two blocks with a bitonic network as in the minBlockHeap's fillEmptyNode,
// widened from 32+32 to 1024 items per warp).
//
// Merges A[0, X) and B[0, Y) (ascending, shared memory, X + Y = m <= 1024)
// into out[0, m) ascending.  The warp reads C = A ascending ++ pads ++ B
// descending -- a bitonic sequence -- in the striped layout (item 32k+lane in
// register k: 32 consecutive words per load), runs the five half-cleaners of
// stride >= 32 inside registers, transposes through a padded scratch to the
// blocked layout (items 32*lane .. 32*lane+31 in one lane), runs the five
// half-cleaners of stride < 32 inside registers with lane-flipped directions,
// and stores item 32*lane + (j ^ lane) from register j: every shared-memory
// access of the warp touches 32 distinct banks (16 per half-warp for 64-bit
// keys), whatever the data.
// ---------------------------------------------------------------------------
template <typename KeyT>
__device__ __forceinline__ void warp_load_bitonic(const KeyT* A, int X, const KeyT* B, int Y,
                                                  KeyT (&v)[32], int lane) {
  const int kA = X >> 5;                    // registers [0, kA) come from A only
  const int kB = (kBlockItems - Y + 31) >> 5;  // registers [kB, 32) come from B only
  const KeyT* Bend = B + (kBlockItems - 1);    // C[i] = B[1023 - i] for i >= 1024 - Y
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int i = 32 * k + lane;
    if (k < kA) {
      v[k] = A[i];
    } else if (k >= kB) {
      v[k] = Bend[-i];
    } else {
      KeyT t = key_pad<KeyT>();
      lds_pred(t, A + i, i < X);
      lds_pred(t, Bend - i, i >= kBlockItems - Y);
      v[k] = t;
    }
  }
}

template <typename KeyT>
__device__ __forceinline__ void warp_bitonic_1024(KeyT (&v)[32], KeyT* scr, int lane) {
  // half-cleaners of stride 512 .. 32: register distance 16 .. 1
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if ((k & s) == 0) cas(v[k], v[k + s]);
  }
  // striped -> blocked through the padded scratch (row k holds items 32k..32k+31)
#pragma unroll
  for (int k = 0; k < 32; ++k) scr[kScratchRow * k + lane] = v[k];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = scr[kScratchRow * lane + j];
  __syncwarp();
  // half-cleaners of stride 16 .. 1 inside the lane, direction flipped by lane bit
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool f = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if ((k & s) == 0) cas_dir(v[k], v[k + s], f);
  }
}

// Stores the lane-XOR-permuted sorted block: register j holds item 32*lane + (j ^ lane).
template <typename KeyT>
__device__ __forceinline__ void warp_store_block(KeyT* out, int m, const KeyT (&v)[32], int lane) {
  KeyT* base = out + 32 * lane;
  if (m == kBlockItems) {
#pragma unroll
    for (int j = 0; j < 32; ++j) base[j ^ lane] = v[j];
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int e = 32 * lane + (j ^ lane);
      if (e < m) base[j ^ lane] = v[j];
    }
  }
}

template <typename KeyT>
__device__ __forceinline__ void warp_merge_block(const KeyT* A, int X, const KeyT* B, int Y,
                                                 KeyT* out, KeyT* scr, int lane) {
  KeyT v[32];
  warp_load_bitonic(A, X, B, Y, v, lane);
  warp_bitonic_1024(v, scr, lane);
  warp_store_block(out, X + Y, v, lane);
}

// ---------------------------------------------------------------------------
// One CTA merge level.  Sequence q (q < 32) of `src` is described by lane q's
// (off, len); sequences (2p, 2p+1) are merged into `dst`, packed in pair
// order.  Work items are the 1024-item output blocks of every pair, dealt to
// the warps round-robin.  next_seq() gives the descriptors of the outputs.
// ---------------------------------------------------------------------------
template <typename KeyT>
__device__ __forceinline__ void cta_merge_level(const KeyT* src, KeyT* dst, int my_off, int my_len,
                                                int nseq, KeyT* scr, int warp, int nwarps,
                                                int lane) {
  int item = 0;
  int outoff = 0;
  for (int q = 0; 2 * q < nseq; ++q) {
    const int a_off = __shfl_sync(0xffffffffu, my_off, 2 * q);
    const int a_len = __shfl_sync(0xffffffffu, my_len, 2 * q);
    const int b_off = __shfl_sync(0xffffffffu, my_off, (2 * q + 1) & 31);
    const int b_len = (2 * q + 1 < nseq) ? __shfl_sync(0xffffffffu, my_len, (2 * q + 1) & 31) : 0;
    const int L = a_len + b_len;
    const KeyT* A = src + a_off;
    const KeyT* B = src + b_off;
    for (int d0 = 0; d0 < L; d0 += kBlockItems, ++item) {
      if (item % nwarps != warp) continue;
      const int m = (L - d0) < kBlockItems ? (L - d0) : kBlockItems;
      const int a0 = warp_corank(A, a_len, B, b_len, d0, lane);
      const int a1 = warp_corank(A, a_len, B, b_len, d0 + m, lane);
      const int X = a1 - a0;
      warp_merge_block(A + a0, X, B + (d0 - a0), m - X, dst + outoff + d0, scr, lane);
    }
    outoff += L;
  }
}

// Descriptors of the pair outputs of a level: lane p gets (packed offset, length).
__device__ __forceinline__ void next_seq(int& my_off, int& my_len, int nseq, int lane) {
  const int l0 = __shfl_sync(0xffffffffu, my_len, (2 * lane) & 31);
  const int l1 = __shfl_sync(0xffffffffu, my_len, (2 * lane + 1) & 31);
  int len = 0;
  if (2 * lane < nseq) len = l0 + ((2 * lane + 1 < nseq) ? l1 : 0);
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  my_off = incl - len;
  my_len = len;
}

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy (TMA 1-D) helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32addr(bar)),
               "r"(bytes)
               : "memory");
}

// Waits for phase `parity` of the barrier, giving up after roughly two
// seconds of polling; returns false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const uint32_t addr = smem_u32addr(bar);
  const long long t0 = clock64();
  for (long long it = 0; it < (1ll << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 4000000000ll) break;
  }
  return false;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32addr(bar))
      : "memory");
}

__device__ __forceinline__ void set_device_error(int* err, int code) {
  if (err) atomicCAS(err, kDevOk, code);
}

}  // namespace mms
