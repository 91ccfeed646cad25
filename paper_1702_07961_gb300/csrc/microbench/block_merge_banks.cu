// block_merge_banks.cu -- bank-conflict control for the warp block merge
// (Sec. 4.2 block merging, Sec. 5.2 conflict-free shared-memory access).
//
// Not part of libmms.so.  A standalone program for reading shared-memory bank
// conflict counters under a profiler: every warp of every CTA holds two sorted
// 1024-key lists in shared memory and merges them `reps` times into 2048 keys,
// block by block (co-rank search, striped window load, bitonic network with the
// swizzled transpose, chunked store) -- the same device code the merge pass
// runs.  Variants:
//   full   -- the whole block merge;
//   loads  -- co-ranks and the window loads only;
//   corank -- the co-rank search only;
//   wsort  -- the tile sort's warp sort of 1024 keys (random keys only).
// On random keys each variant runs at reps = 0, 4 and 16; `full` then runs at
// reps = 0 and 16 on three more key sets: all keys equal, disjoint lists (every
// key of the first list below every key of the second), and interleaved lists
// (even and odd numbers), which move every block window to its extremes.
// reps = 0 leaves only the fill (global -> shared, 32 consecutive words per
// instruction) and the drain (shared -> global, the same), so counts that stay
// at the reps = 0 level as reps grows do not come from the block merge.  The
// program checks every merged output of `full` on the host and exits non-zero
// on a mismatch.
//
// Build and run (sm_103a):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -Iinclude \
//        -o block_merge_banks paper_1702_07961_gb300/csrc/microbench/block_merge_banks.cu
//   ./block_merge_banks
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../mms_common.cuh"
#include "../tile_sort.cuh"

using namespace mms;

namespace {

constexpr int kList = 1024;                 // keys per input list
constexpr int kWarps = 5;                   // warps per CTA
constexpr int kWarpWords = 4 * kList + 64;  // A, B, 2048-key output, slack (16-byte multiple)
enum Variant { kFull = 0, kLoads = 1, kCorank = 2, kWarpSort = 3 };

template <int V>
__global__ void __launch_bounds__(kWarps * 32) block_merge_banks(const uint32_t* in, uint32_t* out_g,
                                                                 int reps) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* A = reinterpret_cast<uint32_t*>(smem) + warp * kWarpWords;
  uint32_t* B = A + kList;
  uint32_t* out = A + 2 * kList;
  const size_t w = (size_t)blockIdx.x * kWarps + warp;
  const uint32_t* src = in + w * 2 * kList;
  for (int i = lane; i < kList; i += 32) {
    A[i] = src[i];
    B[i] = src[kList + i];
  }
  for (int i = lane; i < 2 * kList; i += 32) out[i] = 0;
  __syncwarp();
  uint32_t acc = 0;
  if constexpr (V == kWarpSort) {
    // The tile sort's warp sort of 1024 keys (x = A xor B, item 32j + lane in
    // register j), `reps` times, with its transposes in `out`; then stored.
    uint32_t v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = A[32 * j + lane] ^ B[32 * j + lane];
    for (int rep = 0; rep < reps; ++rep) warp_sort_1024(v, out, lane);
    if (reps > 0) warp_store_block<uint32_t>(out, kBlockItems, v, lane, false);
    __syncwarp();
    reps = 0;
  }
  for (int rep = 0; rep < reps; ++rep) {
    for (int d0 = 0; d0 < 2 * kList; d0 += kBlockItems) {
      if constexpr (V == kCorank) {
        acc += warp_corank(A, kList, B, kList, d0 + kBlockItems / 2, lane);
        continue;
      }
      const int a0 = (d0 == 0) ? 0 : warp_corank(A, kList, B, kList, d0, lane);
      const int a1 = (d0 + kBlockItems == 2 * kList)
                         ? kList
                         : warp_corank(A, kList, B, kList, d0 + kBlockItems, lane, a0, a0 + kBlockItems);
      const int X = a1 - a0;
      uint32_t v[32];
      warp_load_bitonic(A + a0, X, B + (d0 - a0), kBlockItems - X, v, lane);
      if constexpr (V == kLoads) {
#pragma unroll
        for (int j = 0; j < 32; ++j) acc += v[j];
        continue;
      }
      warp_bitonic_1024(v, out + d0, 32, lane);
      warp_store_block<uint32_t>(out + d0, kBlockItems, v, lane, false);
      __syncwarp();
    }
  }
  uint32_t* dst = out_g + w * 2 * kList;
  for (int i = lane; i < 2 * kList; i += 32) dst[i] = out[i] + acc;
}

template <int V>
bool run(const char* name, int ctas, const uint32_t* din, uint32_t* dout, int reps) {
  const size_t smem = (size_t)kWarps * kWarpWords * sizeof(uint32_t);
  cudaFuncSetAttribute(block_merge_banks<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  block_merge_banks<V><<<ctas, kWarps * 32, smem>>>(din, dout, reps);
  const cudaError_t e = cudaDeviceSynchronize();
  std::printf("%-11s reps=%-2d %s\n", name, reps, cudaGetErrorString(e));
  return e == cudaSuccess;
}

}  // namespace

// Fills the two sorted lists of every warp: 0 random, 1 all equal, 2 disjoint,
// 3 interleaved.
void fill(std::vector<uint32_t>& h, size_t lists, int kind) {
  std::mt19937 rng(1);
  for (size_t w = 0; w < lists; ++w) {
    uint32_t* a = h.data() + w * 2 * kList;
    uint32_t* b = a + kList;
    for (int i = 0; i < kList; ++i) {
      switch (kind) {
        case 0: a[i] = (uint32_t)rng(); b[i] = (uint32_t)rng(); break;
        case 1: a[i] = 7u; b[i] = 7u; break;
        case 2: a[i] = (uint32_t)i; b[i] = (uint32_t)(kList + i); break;
        default: a[i] = 2u * i; b[i] = 2u * i + 1u; break;
      }
    }
    std::sort(a, a + kList);
    std::sort(b, b + kList);
  }
}

bool check(const std::vector<uint32_t>& h, const uint32_t* dout, size_t lists, const char* name, int reps) {
  std::vector<uint32_t> got(h.size());
  cudaMemcpy(got.data(), dout, h.size() * 4, cudaMemcpyDeviceToHost);
  bool ok = true;
  for (size_t w = 0; w < lists && ok; ++w) {
    std::vector<uint32_t> want(h.begin() + w * 2 * kList, h.begin() + (w + 1) * 2 * kList);
    std::sort(want.begin(), want.end());
    ok = std::equal(want.begin(), want.end(), got.begin() + w * 2 * kList);
  }
  std::printf("full   reps=%-2d %-11s merged output %s\n", reps, name, ok ? "matches" : "MISMATCH");
  return ok;
}

// The warp-sort variant's output: each warp's x = A xor B, sorted, then zeros.
bool check_wsort(const std::vector<uint32_t>& h, const uint32_t* dout, size_t lists, int reps) {
  std::vector<uint32_t> got(h.size());
  cudaMemcpy(got.data(), dout, h.size() * 4, cudaMemcpyDeviceToHost);
  bool ok = true;
  for (size_t w = 0; w < lists && ok; ++w) {
    const uint32_t* a = h.data() + w * 2 * kList;
    std::vector<uint32_t> want(kList);
    for (int i = 0; i < kList; ++i) want[i] = a[i] ^ a[kList + i];
    std::sort(want.begin(), want.end());
    ok = std::equal(want.begin(), want.end(), got.begin() + w * 2 * kList);
    for (int i = kList; i < 2 * kList && ok; ++i) ok = got[w * 2 * kList + i] == 0u;
  }
  std::printf("wsort  reps=%-2d random      sorted output %s\n", reps, ok ? "matches" : "MISMATCH");
  return ok;
}

int main() {
  const int ctas = 2 * 152;
  const size_t lists = (size_t)ctas * kWarps;
  const size_t n = lists * 2 * kList;
  const char* names[4] = {"random", "equal", "disjoint", "interleaved"};
  std::vector<uint32_t> h(n);
  uint32_t *din = nullptr, *dout = nullptr;
  if (cudaMalloc(&din, n * 4) != cudaSuccess || cudaMalloc(&dout, n * 4) != cudaSuccess) return 1;
  bool ok = true;
  for (int kind = 0; kind < 4 && ok; ++kind) {
    fill(h, lists, kind);
    cudaMemcpy(din, h.data(), n * 4, cudaMemcpyHostToDevice);
    for (int reps : {0, 4, 16}) {
      if (kind > 0 && reps == 4) continue;
      ok = ok && run<kFull>(names[kind], ctas, din, dout, reps);
      if (ok && reps > 0) ok = check(h, dout, lists, names[kind], reps);
      if (kind == 0) {
        ok = ok && run<kLoads>("loads", ctas, din, dout, reps);
        ok = ok && run<kCorank>("corank", ctas, din, dout, reps);
        ok = ok && run<kWarpSort>("wsort", ctas, din, dout, reps);
        if (ok && reps > 0) ok = check_wsort(h, dout, lists, reps);
      }
    }
  }
  cudaFree(din);
  cudaFree(dout);
  return ok ? 0 : 1;
}
