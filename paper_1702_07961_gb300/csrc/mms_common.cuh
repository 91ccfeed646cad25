// mms_common.cuh -- shared device building blocks of the GPU Multiway Mergesort
// kernels for sm_103a: key traits, the order-preserving float transform,
// compare-exchange, the conflict-free warp merge of a 1024-item block, the
// warp co-rank (merge-path) search in shared memory, and TMA/mbarrier PTX.
//
// Shared-memory discipline (Sec. 3.2 and Sec. 5.2): every shared-memory access
// a warp makes is 32 consecutive items (any base: one bank each), a row of 32
// items whose 16-byte chunks are XOR-swizzled by the row index, a 16-byte
// chunk whose position is XOR-permuted by the lane id, or a probe at an odd
// stride -- never a data-dependent gather -- so no input can cause a bank
// conflict.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "mms_kernels.cuh"

namespace mms {

constexpr int kWarpSize = 32;
constexpr int kBlockItems = 1024;       // one warp block: 32 lanes x 32 registers

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

// 16-byte vectors of keys.
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

// Compare-exchange as one min and one max (no compare-and-select pair).
__device__ __forceinline__ uint32_t kmin(uint32_t a, uint32_t b) { return min(a, b); }
__device__ __forceinline__ uint32_t kmax(uint32_t a, uint32_t b) { return max(a, b); }
__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) {
  return min((unsigned long long)a, (unsigned long long)b);
}
__device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) {
  return max((unsigned long long)a, (unsigned long long)b);
}

template <typename KeyT>
__device__ __forceinline__ void cas(KeyT& a, KeyT& b) {
  const KeyT lo = kmin(a, b);
  const KeyT hi = kmax(a, b);
  a = lo;
  b = hi;
}
// 64-bit keys: one unsigned 64-bit compare drives the four 32-bit selects of
// the pair (min and max computed apart would each compare and select).
__device__ __forceinline__ void cas(uint64_t& a, uint64_t& b) {
  const bool sw = b < a;
  const uint64_t lo = sw ? b : a;
  const uint64_t hi = sw ? a : b;
  a = lo;
  b = hi;
}

// Compare-exchange whose direction is chosen per lane: with flip set the
// larger key goes to a.  Flipping the stages of a bitonic merge whose stride
// bit is set in a lane mask leaves the lane's sorted items XOR-permuted by
// that mask, which makes the following shared-memory store conflict-free.
template <typename KeyT>
__device__ __forceinline__ void cas_dir(KeyT& a, KeyT& b, bool flip) {
  const KeyT x = a, y = b;
  a = flip ? kmax(x, y) : kmin(x, y);
  b = flip ? kmin(x, y) : kmax(x, y);
}
// 64-bit keys: the direction folds into the compare's predicate (swap when
// the pair is out of the lane's order), then four 32-bit selects.
__device__ __forceinline__ void cas_dir(uint64_t& a, uint64_t& b, bool flip) {
  const bool sw = (b < a) != flip;
  const uint64_t x = sw ? b : a;
  const uint64_t y = sw ? a : b;
  a = x;
  b = y;
}

// ---------------------------------------------------------------------------
// Compare-exchange split across two pipes (uint32 keys).  min and max run on
// the ALU pipe and integer multiply-add on the FMA pipe; on sm_103a both are
// half rate.  The larger key of a pair is also a + b - min(a, b), exact
// modulo 2^32, so a compare-exchange can take one ALU min and two multiply-adds
// instead of a min and a max.  Mixing the two forms keeps both pipes and the
// issue slot busy: in a register-only microbenchmark 11 of 16 pairs in the
// multiply-add form gave 1.41x the compare-exchange rate of min/max alone
// (10 of 16 for the per-lane-direction form, 1.38x).  Inside the kernels the
// best mix follows what else the kernel issues, measured on GB300: the base
// case (issue-bound, ALU pipe 69% busy) is fastest with 6 of 16 plain pairs
// and 12 of 16 direction pairs, the merge pass (barrier-bound, ALU 57%) with
// plain pairs as min/max and 12 of 16 direction pairs; each kernel passes its
// own Mix type.  The multiply-adds use a runtime 1 (and -1, -2) so that the
// compiler keeps them multiplies.
//
// 64-bit keys: a compare-exchange is one 64-bit compare and four 32-bit
// selects on the ALU pipe.  The selects can also be made exact multiply-adds
// on the FMA pipe: with f = 1 when the pair swaps, each half x of a and y of
// b becomes x + f (y - x) and y + f (x - y).  That form costs more issue
// slots, so it pays only where the ALU pipe is the tighter limit: measured on
// GB300 at 10^8 u64 keys, 6 of 16 plain pairs of the merge pass in it took the
// five K = 8 passes from 4.686 to 4.594 ms, while any share of the base
// case's pairs, or of direction pairs, made it slower (base case 1.85 ->
// 2.00..2.30 ms).
// ---------------------------------------------------------------------------
// MIX / MIXD: how many of a stage's 16 pairs take the multiply-add form, for
// plain pairs and for pairs whose direction is chosen per lane, with 32-bit
// keys; MIX64 / MIXD64 the same with 64-bit keys.
template <int MIX, int MIXD, int MIX64, int MIXD64>
struct Mix {
  uint32_t one, m1, m2;   // 1, -1, -2 (mod 2^32), unknown to the compiler
};
template <typename M>
__device__ __forceinline__ M mad_ones() {
  const uint32_t b = blockDim.x;
  const uint32_t one = b >> (31 - __clz(b));   // b >> floor(log2 b) == 1 for b >= 1
  return M{one, 0u - one, 0u - one - one};
}
__device__ __forceinline__ uint32_t mad_u32(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Whether the pair with ordinal i among a stage's 16 pairs takes the
// multiply-add form when `count` of 16 do: the pairs are spread evenly
// (i * count mod 16 below count).
__device__ __forceinline__ constexpr bool mad_pick(int i, int count) {
  return ((i * count) & 15) < count;
}
// Ordinal of the pair (k, k + s) among the 16 pairs of a stride-s stage.
__device__ __forceinline__ constexpr int pair_ordinal(int k, int s) {
  return (k & (s - 1)) | ((k >> 1) & ~(s - 1));
}

// Compare-exchange (ascending) of a stage pair with ordinal i.
template <int MIX, int MIXD, int MIX64, int MIXD64>
__device__ __forceinline__ void cas_mix(uint32_t& a, uint32_t& b, int i,
                                        const Mix<MIX, MIXD, MIX64, MIXD64>& c) {
  if (mad_pick(i, MIX)) {
    const uint32_t lo = min(a, b);
    const uint32_t s = mad_u32(a, c.one, b);
    a = lo;
    b = mad_u32(lo, c.m1, s);
  } else {
    cas(a, b);
  }
}

// 64-bit pair: swap when sw, the selects as multiply-adds (exact for f in
// {0, 1}).
template <typename M>
__device__ __forceinline__ void swap64_mad(uint64_t& a, uint64_t& b, bool sw, const M& c) {
  const uint32_t f = sw ? c.one : 0u;
  const uint32_t al = (uint32_t)a, ah = (uint32_t)(a >> 32);
  const uint32_t bl = (uint32_t)b, bh = (uint32_t)(b >> 32);
  const uint32_t dl = mad_u32(al, c.m1, bl), el = mad_u32(bl, c.m1, al);   // bl - al, al - bl
  const uint32_t dh = mad_u32(ah, c.m1, bh), eh = mad_u32(bh, c.m1, ah);
  const uint32_t xl = mad_u32(f, dl, al), yl = mad_u32(f, el, bl);         // sw ? b : a, sw ? a : b
  const uint32_t xh = mad_u32(f, dh, ah), yh = mad_u32(f, eh, bh);
  a = ((uint64_t)xh << 32) | xl;
  b = ((uint64_t)yh << 32) | yl;
}

template <int MIX, int MIXD, int MIX64, int MIXD64>
__device__ __forceinline__ void cas_mix(uint64_t& a, uint64_t& b, int i,
                                        const Mix<MIX, MIXD, MIX64, MIXD64>& c) {
  if (mad_pick(i, MIX64))
    swap64_mad(a, b, b < a, c);
  else
    cas(a, b);
}

// cas_dir with the direction as f in {0, 1} (1: the larger key goes to a).
template <int MIX, int MIXD, int MIX64, int MIXD64>
__device__ __forceinline__ void cas_dir_mix(uint32_t& a, uint32_t& b, uint32_t f, int i,
                                            const Mix<MIX, MIXD, MIX64, MIXD64>& c) {
  if (mad_pick(i, MIXD)) {
    const uint32_t lo = min(a, b);
    const uint32_t s = mad_u32(a, c.one, b);   // a + b
    const uint32_t d = mad_u32(lo, c.m2, s);   // max - min
    const uint32_t x = mad_u32(f, d, lo);      // f ? max : min
    a = x;
    b = mad_u32(x, c.m1, s);
  } else {
    cas_dir(a, b, f != 0);
  }
}
template <int MIX, int MIXD, int MIX64, int MIXD64>
__device__ __forceinline__ void cas_dir_mix(uint64_t& a, uint64_t& b, uint32_t f, int i,
                                            const Mix<MIX, MIXD, MIX64, MIXD64>& c) {
  if (mad_pick(i, MIXD64))
    swap64_mad(a, b, (b < a) != (f != 0), c);
  else
    cas_dir(a, b, f != 0);
}

// The mixes the kernels use (multiply-add pairs of 16: plain and per-lane
// direction, 32-bit keys then 64-bit keys).
using TileMix = Mix<kTileMadPairs, kTileMadDirPairs, kTileMad64Pairs, kTileMad64DirPairs>;
using MergeMix = Mix<kMergeMadPairs, kMergeMadDirPairs, kMergeMad64Pairs, kMergeMad64DirPairs>;


// ---------------------------------------------------------------------------
// Shared-memory accesses the compiler may not merge or reorder across.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Loads p[0] into v when idx < lim (signed), in one compare and one predicated
// load; v keeps its value otherwise.
__device__ __forceinline__ void lds_if_lt(uint32_t& v, const uint32_t* p, int idx, int lim) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.lt.s32 q, %2, %3;\n\t@q ld.shared.b32 %0, [%1];\n\t}\n"
      : "+r"(v)
      : "r"(smem_u32addr(p)), "r"(idx), "r"(lim)
      : "memory");
}
__device__ __forceinline__ void lds_if_lt(uint64_t& v, const uint64_t* p, int idx, int lim) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.lt.s32 q, %2, %3;\n\t@q ld.shared.b64 %0, [%1];\n\t}\n"
      : "+l"(v)
      : "r"(smem_u32addr(p)), "r"(idx), "r"(lim)
      : "memory");
}
// v = a[0] when idx < lim (signed), b[0] otherwise: one compare, two predicated
// loads with complementary predicates (each touching consecutive words only).
__device__ __forceinline__ void lds_pair(uint32_t& v, const uint32_t* a, const uint32_t* b, int idx,
                                         int lim) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.lt.s32 q, %3, %4;\n\t@q ld.shared.b32 %0, [%1];\n\t"
      "@!q ld.shared.b32 %0, [%2];\n\t}\n"
      : "+r"(v)
      : "r"(smem_u32addr(a)), "r"(smem_u32addr(b)), "r"(idx), "r"(lim)
      : "memory");
}
__device__ __forceinline__ void lds_pair(uint64_t& v, const uint64_t* a, const uint64_t* b, int idx,
                                         int lim) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.lt.s32 q, %3, %4;\n\t@q ld.shared.b64 %0, [%1];\n\t"
      "@!q ld.shared.b64 %0, [%2];\n\t}\n"
      : "+l"(v)
      : "r"(smem_u32addr(a)), "r"(smem_u32addr(b)), "r"(idx), "r"(lim)
      : "memory");
}
// Loads p[0] into v when idx >= lim (signed).
__device__ __forceinline__ void lds_if_ge(uint32_t& v, const uint32_t* p, int idx, int lim) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ge.s32 q, %2, %3;\n\t@q ld.shared.b32 %0, [%1];\n\t}\n"
      : "+r"(v)
      : "r"(smem_u32addr(p)), "r"(idx), "r"(lim)
      : "memory");
}
__device__ __forceinline__ void lds_if_ge(uint64_t& v, const uint64_t* p, int idx, int lim) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ge.s32 q, %2, %3;\n\t@q ld.shared.b64 %0, [%1];\n\t}\n"
      : "+l"(v)
      : "r"(smem_u32addr(p)), "r"(idx), "r"(lim)
      : "memory");
}

// ---------------------------------------------------------------------------
// Warp co-rank (merge path) search, Sec. 4.1 specialised to two lists:
// returns the number of items of A among the first d items of merge(A, B),
// ties taken from A (stable).  32-ary: each round all lanes probe positions
// at an odd stride (distinct banks), a ballot narrows the range 32-fold.
// ---------------------------------------------------------------------------
// `lo0` / `hi0` narrow the search when a bracket is known: the co-rank of
// d + m lies within [co-rank of d, co-rank of d + m] of the block before it.
template <typename KeyT>
__device__ __forceinline__ int warp_corank(const KeyT* A, int lenA, const KeyT* B, int lenB,
                                           int d, int lane, int lo0 = 0, int hi0 = 0x7fffffff) {
  int lo = d - lenB > lo0 ? d - lenB : lo0;
  int hi = d < lenA ? d : lenA;
  hi = hi < hi0 ? hi : hi0;
  while (hi > lo) {
    const int step = ((hi - lo + 31) >> 5) | 1;
    const int i = lo + lane * step;
    bool p = true;                                 // positions >= hi count as "true"
    if (i < hi) p = A[i] > B[d - 1 - i];           // A[i] comes after B[d-1-i]
    const unsigned bal = __ballot_sync(0xffffffffu, p);
    const int f = __ffs(bal) - 1;                  // first "true" probe, -1 if none
    const int top = lo + f * step;
    const int nlo = (f <= 0) ? (f == 0 ? lo : lo + 31 * step + 1) : top - step + 1;
    hi = (f < 0) ? hi : (top < hi ? top : hi);
    lo = nlo;
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
// stride >= 32 inside registers, transposes through the padded scratch to the
// blocked layout (items 32*lane .. 32*lane+31 in one lane), runs the five
// half-cleaners of stride < 32 inside registers, flipping the direction of the
// strides of 16 bytes and more by lane bits, and stores 16-byte chunks whose
// position in the row is XOR-permuted by the lane: every shared-memory access
// of the warp is conflict-free whatever the data.
// ---------------------------------------------------------------------------

// Register k of lane l receives C[32k + l]: A[32k + l] when that is below X,
// B[1023 - 32k - l] when it is at or above 1024 - Y, a pad in between.  The A
// and B halves of a register are fetched by two predicated loads, so each
// load instruction touches consecutive words only.
template <typename KeyT>
__device__ __forceinline__ void warp_load_bitonic(const KeyT* A, int X, const KeyT* B, int Y,
                                                  KeyT (&v)[32], int lane) {
  const KeyT* pa = A + lane;                         // C[32k+lane] = A[32k+lane]
  const KeyT* pb = B + (kBlockItems - 1 - lane);     // C[32k+lane] = B[1023-32k-lane]
  const int xa = X - lane;                           // 32k + lane < X  <=>  32k < xa
  const int xb = kBlockItems - Y - lane;             // 32k + lane >= 1024 - Y  <=>  32k >= xb
  if (X + Y == kBlockItems) {                        // full block: no pads, xa == xb
#pragma unroll
    for (int k = 0; k < 32; ++k) lds_pair(v[k], pa + 32 * k, pb - 32 * k, 32 * k, xa);
    return;
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    KeyT t = key_pad<KeyT>();
    lds_if_lt(t, pa + 32 * k, 32 * k, xa);
    lds_if_ge(t, pb - 32 * k, 32 * k, xb);
    v[k] = t;
  }
}

// Flip mask of a lane: the in-row XOR that makes its 16-byte chunk stores hit
// distinct banks within each quarter-warp (a multiple of the chunk size).
template <typename KeyT>
__device__ __forceinline__ int flip_mask(int lane) {
  constexpr int E = Vec16<KeyT>::E;
  return (lane & (32 / E - 1)) * E;
}

// Pieces of the warp's bitonic networks over 1024 items, 32 per lane.  In the
// striped layout register k of lane l holds item 32k + l (row k, column l); in
// the blocked layout lane l holds row l, item 32l + j in register j.

// Half-cleaners of register distance D, D/2, .., 1 (strides 32D .. 32 of the
// striped layout), ascending.
template <int D, typename KeyT, typename M>
__device__ __forceinline__ void striped_stages(KeyT (&v)[32], const M& c) {
#pragma unroll
  for (int s = D; s >= 1; s >>= 1) {
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if ((k & s) == 0) cas_mix(v[k], v[k + s], pair_ordinal(k, s), c);
  }
}

// Striped -> blocked through `out` (16-byte aligned, 32 * nr items): row k is
// stored with its 16-byte chunks XOR-swizzled by k & 7 (item 32k + l at word
// 32k + (l ^ E*(k & 7))), so the scalar row stores and the 16-byte row loads
// are both conflict-free.  Rows at or above nr are not stored; lanes at or
// above nr receive pads.
template <typename KeyT>
__device__ __forceinline__ void striped_to_blocked(KeyT (&v)[32], KeyT* out, int nr, int lane) {
  using V = Vec16<KeyT>;
  constexpr int E = V::E;
#pragma unroll
  for (int k = 0; k < 32; ++k)
    if (k < nr) out[32 * k + (lane ^ (E * (k & 7)))] = v[k];
  __syncwarp();
  if (lane < nr) {
    const typename V::T* row = reinterpret_cast<const typename V::T*>(out + 32 * lane);
    const int sw = lane & 7;
#pragma unroll
    for (int ch = 0; ch < 32 / E; ++ch) V::unpack(row[ch ^ sw], &v[ch * E]);
  } else {
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = key_pad<KeyT>();
  }
  __syncwarp();
}

// Half-cleaners of stride 16 .. 1 inside the lane (blocked layout).  FLIP:
// the strides of 16 bytes and more run in the direction of the lane's
// flip_mask bit, leaving register j with item 32l + (j ^ flip_mask(l)) -- the
// layout warp_store_block writes out; otherwise all ascending.
template <bool FLIP, typename KeyT, typename M>
__device__ __forceinline__ void blocked_stages(KeyT (&v)[32], int lane, const M& c) {
  constexpr int E = Vec16<KeyT>::E;
  const int F = flip_mask<KeyT>(lane);
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const uint32_t f = (F & s) ? 1u : 0u;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if ((k & s) != 0) continue;
      if (FLIP && s >= E)
        cas_dir_mix(v[k], v[k + s], f, pair_ordinal(k, s), c);
      else
        cas_mix(v[k], v[k + s], pair_ordinal(k, s), c);   // F has no bit below E
    }
  }
}

// Runs the bitonic merge of the 1024 items in v (striped layout).  The
// striped -> blocked transpose goes through the block's own output region
// `out` (16-byte aligned, at least 32 * nr items): row k (items 32k .. 32k+31)
// is stored with its 16-byte chunks XOR-swizzled by k & 7, which keeps both
// the scalar row stores and the 16-byte row loads conflict-free without
// padding.  After the five half-cleaners of stride >= 32 the rows are ordered
// (every item of row k is <= every item of row k+1), so rows at or above
// nr = ceil(m / 32) hold only pads (or real all-ones keys, bit-identical to
// pads) and are neither stored nor loaded.  M: the kernel's compare-exchange mix.
template <typename M, typename KeyT>
__device__ __forceinline__ void warp_bitonic_1024(KeyT (&v)[32], KeyT* out, int nr, int lane) {
  const M c = mad_ones<M>();
  striped_stages<16>(v, c);                          // strides 512 .. 32
  striped_to_blocked(v, out, nr, lane);
  blocked_stages<true>(v, lane, c);                  // strides 16 .. 1, store layout
}
__device__ __forceinline__ void sts_addr(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_addr(uint32_t addr, uint64_t v) {
  asm volatile("st.shared.b64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void sts128(uint32_t addr, const uint32_t* v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]),
               "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ void sts128(uint32_t addr, const uint64_t* v) {
  asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(v[0]), "l"(v[1]) : "memory");
}

// 16-byte store when a <= b (signed), compare and store in one predicate.
__device__ __forceinline__ void sts128_if_le(uint32_t addr, const uint32_t* v, int a, int b) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.le.s32 q, %5, %6;\n\t@q st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n\t}\n" ::"r"(
          addr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(a), "r"(b)
      : "memory");
}
__device__ __forceinline__ void sts128_if_le(uint32_t addr, const uint64_t* v, int a, int b) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.le.s32 q, %3, %4;\n\t@q st.shared.v2.b64 [%0], {%1, %2};\n\t}\n" ::"r"(
          addr),
      "l"(v[0]), "l"(v[1]), "r"(a), "r"(b)
      : "memory");
}

// Stores the sorted block: register j of the lane holds item 32*lane + (j ^ F),
// F = flip_mask(lane).  `out` must be 16-byte aligned.  Items go out in 16-byte
// chunks (chunk c of the lane lands at chunk c ^ (F / E) of its row); for a
// short block the chunks wholly below m are stored this way and the one chunk
// that straddles m item by item (by a single lane).  `xout` undoes the float
// transform on the way out.
template <typename KeyT>
__device__ __forceinline__ void warp_store_block(KeyT* out, int m, KeyT (&v)[32], int lane,
                                                 bool xout) {
  constexpr int E = Vec16<KeyT>::E;
  constexpr int SZ = (int)sizeof(KeyT);
  if (xout) {
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = (KeyT)ordered_to_f32((uint32_t)v[j]);
  }
  const int F = flip_mask<KeyT>(lane);
  const uint32_t row = smem_u32addr(out + 32 * lane);
  const int room = m - 32 * lane;                    // items of this row below m
#pragma unroll
  for (int c = 0; c < 32 / E; ++c) {
    const int pos = (c * E) ^ F;                      // item offset of the chunk in the row
    sts128_if_le(row + (uint32_t)(pos * SZ), &v[c * E], pos + E, room);
  }
  if (m < kBlockItems && (m % E) != 0) {
#pragma unroll
    for (int c = 0; c < 32 / E; ++c) {
      const int pos = (c * E) ^ F;
#pragma unroll
      for (int w = 0; w < E; ++w)
        if (pos < room && pos + E > room && pos + w < room)
          sts_addr(row + (uint32_t)((pos + w) * SZ), v[c * E + w]);
    }
  }
}

// `out` is 16-byte aligned; the warp may use out[0, 32 * ceil((X + Y) / 32))
// as transpose space, so up to 31 items past the block's end must be free.
// M: the calling kernel's compare-exchange mix.
// INPLACE: `out` may overlap A and B (a merge of two adjacent sequences back
// into their own span); the warp then synchronises between its loads and the
// first store.
template <typename KeyT, typename M, bool INPLACE = false>
__device__ __forceinline__ void warp_merge_block(const KeyT* A, int X, const KeyT* B, int Y,
                                                 KeyT* out, int lane, bool xout) {
  KeyT v[32];
  warp_load_bitonic(A, X, B, Y, v, lane);
  if constexpr (INPLACE) __syncwarp();
  warp_bitonic_1024<M>(v, out, (X + Y + 31) >> 5, lane);
  warp_store_block<KeyT>(out, X + Y, v, lane, xout);
}

// ---------------------------------------------------------------------------
// Warp merge of a small block (X + Y = m <= 32 R items, R in {1, 2, 4, 8}):
// the same bitonic merge of C = A ascending ++ pads ++ B descending, over
// 32 R items instead of 1024.  Register k of lane l holds C[32k + l]; the
// half-cleaners of stride >= 32 run between registers, those of stride < 32
// between lanes through shuffles (one shuffle and a min or max per register),
// and register k is stored to out[32k + l].  Every shared-memory access is 32
// consecutive items: conflict-free.  A merge tree's node ends in such a block
// whenever its size lies just above a multiple of 1024 -- on random inputs
// about half of a tile's nodes -- and this network costs a fraction of the
// 1024-item one.  `out` receives exactly m items (no transpose space).
// ---------------------------------------------------------------------------
constexpr int kSmallBlockMax = 256;

template <int R, typename KeyT>
__device__ __forceinline__ void warp_merge_small_r(const KeyT* A, int X, const KeyT* B, int Y,
                                                   KeyT* out, int lane, bool xout) {
  constexpr int n = 32 * R;
  const int m = X + Y;
  const KeyT* pa = A + lane;                         // C[32k+lane] = A[32k+lane]
  const KeyT* pb = B + (n - 1 - lane);               // C[32k+lane] = B[n-1-32k-lane]
  const int xa = X - lane;                           // 32k + lane < X  <=>  32k < xa
  const int xb = n - Y - lane;                       // 32k + lane >= n - Y  <=>  32k >= xb
  KeyT v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    KeyT t = key_pad<KeyT>();
    lds_if_lt(t, pa + 32 * k, 32 * k, xa);
    lds_if_ge(t, pb - 32 * k, 32 * k, xb);
    v[k] = t;
  }
#pragma unroll
  for (int s = R / 2; s >= 1; s >>= 1) {             // strides 16R .. 32: between registers
#pragma unroll
    for (int k = 0; k < R; ++k)
      if ((k & s) == 0) cas(v[k], v[k + s]);
  }
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {                // strides 16 .. 1: between lanes
    const bool upper = (lane & s) != 0;              // the pair's larger index keeps the max
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const KeyT y = __shfl_xor_sync(0xffffffffu, v[k], s);
      v[k] = upper ? kmax(v[k], y) : kmin(v[k], y);
    }
  }
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int idx = 32 * k + lane;
    if (idx < m) out[idx] = xout ? (KeyT)ordered_to_f32((uint32_t)v[k]) : v[k];
  }
}

// Merges A[0, X) and B[0, Y) (X + Y <= kSmallBlockMax) into out[0, X + Y)
// with the smallest network that holds them.
template <typename KeyT>
__device__ __forceinline__ void warp_merge_small(const KeyT* A, int X, const KeyT* B, int Y,
                                                 KeyT* out, int lane, bool xout) {
  const int m = X + Y;
  if (m <= 32) warp_merge_small_r<1>(A, X, B, Y, out, lane, xout);
  else if (m <= 64) warp_merge_small_r<2>(A, X, B, Y, out, lane, xout);
  else if (m <= 128) warp_merge_small_r<4>(A, X, B, Y, out, lane, xout);
  else warp_merge_small_r<8>(A, X, B, Y, out, lane, xout);
}

// Merges A[0, X) and B[0, Y) (X + Y <= 1024, any shared-memory offsets) into
// out[0, X + Y) with the register-and-shuffle network of the smallest power
// of two that holds them.  `out` may overlap A and B: every lane has loaded
// all of its items before the first shuffle completes, and the stores follow
// the shuffles.
template <typename KeyT>
__device__ __forceinline__ void warp_merge_any(const KeyT* A, int X, const KeyT* B, int Y,
                                               KeyT* out, int lane, bool xout) {
  const int m = X + Y;
  if (m <= kSmallBlockMax) warp_merge_small<KeyT>(A, X, B, Y, out, lane, xout);
  else if (m <= 512) warp_merge_small_r<16>(A, X, B, Y, out, lane, xout);
  else warp_merge_small_r<32>(A, X, B, Y, out, lane, xout);
}

// ---------------------------------------------------------------------------
// One CTA merge level with a barrier after it (used by the base case, whose
// blocks are all full).  Sequence q (q < 32) of `src` is described by lane
// q's (off, len); sequences (2p, 2p+1) are merged into `dst`, pair outputs
// packed in pair order, 16-byte aligned.  Work items are the 1024-item output
// blocks of every pair, dealt to the warps round-robin.  next_seq() gives the
// descriptors of the outputs.
// ---------------------------------------------------------------------------
template <typename KeyT, typename M>
__device__ __forceinline__ void cta_merge_level(const KeyT* src, KeyT* dst, int my_off, int my_len,
                                                int nseq, int warp, int nwarps, int lane,
                                                bool xout) {
  constexpr int E = Vec16<KeyT>::E;
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
      const int a1 = (d0 + m == L) ? a_len : warp_corank(A, a_len, B, b_len, d0 + m, lane, a0, a0 + m);
      const int X = a1 - a0;
      warp_merge_block<KeyT, M>(A + a0, X, B + (d0 - a0), m - X, dst + outoff + d0, lane, xout);
    }
    outoff += (L + E - 1) / E * E;
  }
}

// Descriptors of the pair outputs of a level: lane p gets (packed offset, length).
template <typename KeyT>
__device__ __forceinline__ void next_seq(int& my_off, int& my_len, int nseq, int lane) {
  constexpr int E = Vec16<KeyT>::E;
  const int l0 = __shfl_sync(0xffffffffu, my_len, (2 * lane) & 31);
  const int l1 = __shfl_sync(0xffffffffu, my_len, (2 * lane + 1) & 31);
  int len = 0;
  if (2 * lane < nseq) len = l0 + ((2 * lane + 1 < nseq) ? l1 : 0);
  const int span = (len + E - 1) / E * E;
  int incl = span;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  my_off = incl - span;
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

// Waits for phase `parity` of the barrier (each try_wait may suspend the
// thread for up to 100 us), giving up after `max_cycles` SM clocks (by
// default about two seconds) or 2^26 tries; returns false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  long long max_cycles = 4000000000ll) {
  const uint32_t addr = smem_u32addr(bar);
  const long long t0 = clock64();
  for (long long it = 0; it < (1ll << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity), "r"(100000u)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > max_cycles) break;
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

// Makes this thread's generic-proxy shared-memory writes visible to TMA.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy of `bytes` (multiple of 16, 16-byte aligned) from this CTA's
// shared memory to global memory; waits until the copy has read its source,
// after which the shared memory may be reused or released (the global writes
// complete on their own, before the grid completes).
__device__ __forceinline__ void bulk_s2g_and_wait(void* dst_gmem, const void* src_smem,
                                                  unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(smem_u32addr(src_smem)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void set_device_error(int* err, int code) {
  if (err) atomicCAS(err, kDevOk, code);
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch (sm_90 and later).  The sort's kernels after
// the base case are launched with programmatic stream serialization: a grid
// may be scheduled once every CTA of the kernel before it has started, so its
// CTAs become resident while that kernel's last wave drains.
// griddep_wait() then blocks until the previous grid has completed and its
// memory is visible; every such kernel calls it before its first global
// memory access (reads and writes alike).  For a normal launch both are
// no-ops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace mms
