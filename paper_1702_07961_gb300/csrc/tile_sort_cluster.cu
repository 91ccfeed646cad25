// tile_sort_cluster.cu -- the base case over runs of CL * 8192 4-byte keys
// (Sec. 4.3 "Internal Memory Sort", with the internal memory of a
// thread-block cluster instead of one CTA).
//
// A cluster of CL CTAs (CL = 2, 4 or 8) sorts one run.  Each CTA first sorts
// its 8192-key tile in its own shared memory exactly as the one-CTA base case
// does (tile_sort.cuh), then the cluster merges the CL sorted tiles in
// log2(CL) further levels through distributed shared memory.  At level l
// (groups of g = 2^l CTAs) the CTAs of a group hold two sorted runs of g/2
// tiles each, A and B, as consecutive 8192-key chunks; CTA j of the group
// produces items [8192 j, 8192 (j + 1)) of merge(A, B):
//   1. warps 0 and 1 find the co-ranks of the slice's two ends (the merge-path
//      search of Sec. 4.1 specialised to two lists, reading the peers' chunks);
//   2. the CTA copies its slice's two input pieces from the peers' shared
//      memory into its free buffer as 16-byte words;
//   3. after a cluster barrier (no CTA reads a peer's chunk any more) the CTA
//      merges the two pieces with the block merge of the CTA levels into its
//      chunk buffer, which then holds the slice.
// The slices of the last level are the run's 8192-key chunks in order; each CTA
// writes its own with one bulk store.  Every key is read from HBM once and
// written once, as in the one-CTA base case, and the levels the cluster adds
// are levels the merge rounds no longer run: a sort of 10^8 keys from runs of
// 32768 needs 12 merge levels instead of 14.  On GB300 a cluster level costs
// more than the merge-round level it saves (about 0.18 ms against 0.13 ms per
// 10^8 keys), so this base case is an option (mms_options.base_items), not the
// default.
#include "tile_sort.cuh"

namespace mms {

namespace {

constexpr int kCT = 8 * kBlockItems;          // keys per CTA tile (8 warps)
constexpr int kLogCT = 13;
static_assert((1 << kLogCT) == kCT, "tile size");
// 16-byte words one thread copies per level: a slice's two pieces span at most
// kCT + 2 * 6 keys once rounded out to whole words.
constexpr int kStageIters = ((kCT + 16) / 4 + 255) / 256;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}

// Barrier over every thread of the cluster: shared-memory writes of any CTA of
// the cluster before it are visible to every CTA's reads after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster
// (cta_addr: a shared::cta address of this CTA), and loads through it.
__device__ __forceinline__ uint32_t map_cluster(uint32_t cta_addr, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(cta_addr), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_cluster_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// A sorted run of the cluster: consecutive chunks of kCT keys in CTAs c0,
// c0 + 1, ..., each at the same offset of its shared memory (`buf`, this
// CTA's shared::cta address of the chunk buffer).
struct ChunkRun {
  uint32_t buf;
  unsigned c0;
  __device__ __forceinline__ uint32_t at(int i) const {
    return ld_cluster_u32(map_cluster(buf + 4u * (unsigned)(i & (kCT - 1)), c0 + (i >> kLogCT)));
  }
  // 16-byte word w of the run (keys 4w .. 4w + 3; never straddles two chunks).
  __device__ __forceinline__ uint4 word(int w) const {
    return ld_cluster_v4(
        map_cluster(buf + 16u * (unsigned)(w & (kCT / 4 - 1)), c0 + (w >> (kLogCT - 2))));
  }
};

// Items of A among the first d items of merge(A, B), ties taken from A: the
// 32-ary search of warp_corank over runs spread across the cluster.  The
// predicate A[i] > B[d - 1 - i] is false then true along i; each round the
// lanes probe 32 positions of the remaining range and a ballot narrows it.
__device__ __forceinline__ int cluster_corank(const ChunkRun& A, int lenA, const ChunkRun& B,
                                              int lenB, int d, int lane) {
  int lo = d - lenB > 0 ? d - lenB : 0;
  int hi = d < lenA ? d : lenA;
  while (hi > lo) {
    const int step = ((hi - lo + 31) >> 5) | 1;
    const int i = lo + lane * step;
    bool p = true;                                 // positions >= hi count as "true"
    if (i < hi) p = A.at(i) > B.at(d - 1 - i);
    const unsigned bal = __ballot_sync(0xffffffffu, p);
    const int f = __ffs(bal) - 1;                  // first "true" probe, -1 if none
    const int top = lo + f * step;
    const int nlo = (f <= 0) ? (f == 0 ? lo : lo + 31 * step + 1) : top - step + 1;
    hi = (f < 0) ? hi : (top < hi ? top : hi);
    lo = nlo;
  }
  return lo;
}

// Keys of the run of g/2 chunks that starts at chunk c0 (rank in the cluster),
// for the tile starting at sbase of a cluster over in[0, n).
__device__ __forceinline__ int run_items(long long n, long long sbase, unsigned c0, unsigned half) {
  const long long r = n - (sbase + (long long)c0 * kCT);
  const long long cap = (long long)half * kCT;
  return r <= 0 ? 0 : (int)(r >= cap ? cap : r);
}

// One cluster level (groups of 2^lv CTAs): on return `cur` holds this CTA's
// slice of its group's merged run (my_len keys; as floats when xout).  `fre`
// is the CTA's other buffer, s_co two ints of shared memory.
__device__ __forceinline__ void cluster_level(int lv, uint32_t* cur, uint32_t* fre, unsigned rank,
                                              long long n, long long sbase, int my_len, bool xout,
                                              int* s_co) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned g = 1u << lv, half = g >> 1, nb = rank & ~(g - 1);
  const int LA = run_items(n, sbase, nb, half), LB = run_items(n, sbase, nb + half, half);
  const ChunkRun A{smem_u32addr(cur), nb}, B{smem_u32addr(cur), nb + half};
  const int d0 = (int)(rank - nb) * kCT;           // this CTA's slice of merge(A, B)
  const int d1 = d0 + my_len;

  cluster_sync();                                  // every chunk of the level's input is in place
  if (warp < 2) {
    const int a = my_len > 0 ? cluster_corank(A, LA, B, LB, warp == 0 ? d0 : d1, lane) : 0;
    if (lane == 0) s_co[warp] = a;
  }
  __syncthreads();
  const int a0 = s_co[0], a1 = s_co[1];
  const int X = a1 - a0, Y = my_len - X, b0 = d0 - a0;
  // Pieces A[a0, a1) and B[b0, b0 + Y) as whole 16-byte words: A's to words
  // 0 .. na - 1 of fre, B's to words na .. na + nbw - 1, so that A[a0] lands at
  // fre[a0 % 4] and B[b0] at fre[4 na + b0 % 4].  The rounding reads at most 3
  // keys past a piece, inside its chunk's buffer (kTileSlack >= 3).
  const int wa0 = a0 >> 2, na = X > 0 ? ((a1 + 3) >> 2) - wa0 : 0;
  const int wb0 = b0 >> 2, nbw = Y > 0 ? ((b0 + Y + 3) >> 2) - wb0 : 0;
  // Three words in flight per thread at a time, then their stores.
  uint4* fw = reinterpret_cast<uint4*>(fre);
#pragma unroll
  for (int b = 0; b < kStageIters; b += 3) {
    uint4 w[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int q = (int)threadIdx.x + 256 * (b + j);
      if (b + j < kStageIters) {
        if (q < na) w[j] = A.word(wa0 + q);
        else if (q < na + nbw) w[j] = B.word(wb0 + q - na);
      }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int q = (int)threadIdx.x + 256 * (b + j);
      if (b + j < kStageIters && q < na + nbw) fw[q] = w[j];
    }
  }
  cluster_sync();                                  // no CTA reads a peer's chunk any more
  const int off = lane == 0 ? (a0 & 3) : 4 * na + (b0 & 3);
  const int len = lane == 0 ? X : Y;
  cta_merge_level<uint32_t, TileMix>(fre, cur, off, len, 2, warp, 8, lane, xout);
}

}  // namespace

// Base case over runs of CL * 8192 4-byte keys of in[0, n) into the same
// positions of out (in == out allowed: every CTA of a cluster has loaded its
// tile before the first cluster barrier, and clusters cover disjoint keys).
template <int CL, bool XIN, bool XOUT>
__global__ void __launch_bounds__(256, (MinBlocks<uint32_t, 8>::value))
    tile_sort_cluster_kernel(const uint32_t* __restrict__ in, uint32_t* out, long long n) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ int s_co[2];
  griddep_launch_dependents();                    // the first splitter may get resident early
  const unsigned rank = cluster_rank();
  const long long sbase = (long long)cluster_index() * CL * kCT;
  const long long base = sbase + (long long)rank * kCT;
  uint32_t v[32];
  tile_load<uint32_t, 8, XIN>(in, n, base, v);
  uint32_t* cur = tile_sort_smem<uint32_t, 8>(v, n, base, false, smem_raw);
  uint32_t* bufX = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* fre = (cur == bufX) ? bufX + kCT + kTileSlack : bufX;
  const long long rem = n - base;
  const int my_len = rem <= 0 ? 0 : (rem >= kCT ? kCT : (int)rem);
  // Every CTA runs every level (empty slices included): the cluster barriers
  // count all of the cluster's threads.
#pragma unroll
  for (int lv = 1; (1 << lv) <= CL; ++lv)
    cluster_level(lv, cur, fre, rank, n, sbase, my_len, XOUT && (2 << lv) > CL, s_co);
  cta_store_tile(cur, out + base, my_len);
}

template <int CL, bool XIN, bool XOUT>
static cudaError_t launch_cluster_t(const void* in, void* out, long long n, cudaStream_t s) {
  const size_t smem = tile_sort_smem_bytes(4, 8);
  auto k = tile_sort_cluster_kernel<CL, XIN, XOUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long R = (long long)CL * kCT;
  const long long clusters = (n + R - 1) / R;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * CL));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<const uint32_t*>(in), static_cast<uint32_t*>(out), n);
}

template <int CL>
static cudaError_t launch_cluster_cl(bool xin, bool xout, const void* in, void* out, long long n,
                                     cudaStream_t s) {
  if (xin && xout) return launch_cluster_t<CL, true, true>(in, out, n, s);
  if (xin) return launch_cluster_t<CL, true, false>(in, out, n, s);
  return launch_cluster_t<CL, false, false>(in, out, n, s);
}

cudaError_t launch_tile_sort_cluster(int cluster_ctas, bool xin, bool xout, const void* in,
                                     void* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  switch (cluster_ctas) {
    case 2: return launch_cluster_cl<2>(xin, xout, in, out, n, s);
    case 4: return launch_cluster_cl<4>(xin, xout, in, out, n, s);
    case 8: return launch_cluster_cl<8>(xin, xout, in, out, n, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mms
