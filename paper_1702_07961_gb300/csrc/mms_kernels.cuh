// mms_kernels.cuh -- host-side launchers of the three hot-path kernels and
// their tile geometry.  A tile is S = 1024 * tile_warps items; the base case
// sorts tiles of S keys and every merge round writes output tiles of S keys.
// Defaults: 8 warps (8192 keys) for 4-byte keys, 4 warps (4096 keys) for
// 8-byte keys, so that three CTAs' shared memory (two tile buffers each) fit
// in one SM.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace mms {

constexpr int kMaxFanout = 32;

// Compare-exchange pairs (of every 16 in a network stage) computed as one
// min and two multiply-adds instead of min and max, per kernel: the base
// case and the merge pass (plain pairs, pairs with a per-lane direction).
constexpr int kTileMadPairs = 6, kTileMadDirPairs = 12;
constexpr int kMergeMadPairs = 0, kMergeMadDirPairs = 12;
// The same for 64-bit keys (their selects as multiply-adds; see mms_common.cuh).
constexpr int kTileMad64Pairs = 0, kTileMad64DirPairs = 0;
constexpr int kMergeMad64Pairs = 6, kMergeMad64DirPairs = 0;

// Device error word values (the first word of a sort workspace).
constexpr int kDevOk = 0;
constexpr int kDevErrTimeout = 1;       // an mbarrier wait ran out of its bound
constexpr int kDevErrInternal = 2;      // a consistency check failed

// CTAs per SM the tile kernels are compiled for (register budget): three
// CTAs of 8 warps (4-byte keys) or of 4 warps (8-byte keys), whose shared
// memory (two tile buffers each, about 66 KB) fits three to an SM.
template <typename KeyT, int WARPS>
struct MinBlocks {
  static constexpr int value = 3;
};

// CTAs per SM the partition variant of the merge pass is compiled for: two
// (128 registers, no spills) measured faster on GB300 than three (80
// registers, about 650 bytes of spills): 10^8 u32 keys 18.4 against 14.7
// Gkeys/s.
constexpr int kPartitionMinBlocks = 2;

// Items of slack past a tile buffer: a partial block's transpose may use up
// to 31 items past the block's end.
constexpr int kTileSlack = 32;

inline int default_tile_warps(int key_bytes) { return key_bytes == 8 ? 4 : 8; }
inline bool valid_tile_warps(int key_bytes, int w) {
  return key_bytes == 8 ? (w == 2 || w == 4) : (w == 4 || w == 8);
}

size_t tile_sort_smem_bytes(int key_bytes, int warps);
size_t merge_pass_smem_bytes(int key_bytes, int warps, int K);

// Base case: sorts every tile of 1024 * tile_warps keys; in == out allowed.
// xin / xout: apply the float order transform on load / its inverse on store.
cudaError_t launch_tile_sort(int key_bytes, int tile_warps, bool xin, bool xout, const void* in,
                             void* out, long long n, cudaStream_t s);

// Base case over runs of cluster_ctas * 8192 4-byte keys (cluster_ctas 2, 4
// or 8): one thread-block cluster per run, each CTA sorting one 8192-key tile,
// then log2(cluster_ctas) merge levels across the cluster's shared memory.
// in == out allowed.
cudaError_t launch_tile_sort_cluster(int cluster_ctas, bool xin, bool xout, const void* in,
                                     void* out, long long n, cudaStream_t s);

// Base case of the key-value sort: 32-bit keys -> sorted tiles of 64-bit
// composites (ordered key << 32 | array position).
cudaError_t launch_tile_sort_composite(int tile_warps, bool xin, const void* keys32, void* out64,
                                       long long n, cudaStream_t s);

// Last step of the key-value sort: keys back from the sorted composites, and
// each value gathered from its original position.
cudaError_t launch_pairs_finalize(bool xout, const void* comp64, const void* vals_src,
                                  void* keys_out, void* vals_out, long long n, cudaStream_t s);

// Key-value sort of 8-byte keys as two stable 4-byte passes (low half, then
// high half): pass inputs, the high halves in pass-1 order, and the final
// permutation of keys and values.
cudaError_t launch_u64_pairs_split(const void* keys, const void* vals, void* lo, void* perm,
                                   void* kcopy, void* vcopy, long long n, cudaStream_t s);
cudaError_t launch_u64_pairs_hi(const void* kcopy, const void* perm, void* hi, long long n,
                                cudaStream_t s);
cudaError_t launch_u64_pairs_final(const void* kcopy, const void* vcopy, const void* perm,
                                   void* keys, void* vals, long long n, cudaStream_t s);

// Splitter: co-ranks of every output tile start (tiles of S items) of every
// group of K runs.  pdl as for launch_merge_pass.
cudaError_t launch_splitter(int key_bytes, long long S, const void* in, long long n,
                            long long run_len, int K, long long* table, cudaStream_t s,
                            bool pdl = false);

// One K-way merge round driven by the splitter table; output tiles of S
// items (a multiple of 1024, at most 1024 * tile_warps).  test_timeout: the
// test hook of mms_options.test_flags (every CTA's extra wait runs out).
// pdl: launch with programmatic stream serialization (the previous kernel on
// the stream is one of this library's).  partition: merge each tile with the
// heap-free partition variant instead of the CTA merge tree (default tile
// geometry only).
cudaError_t launch_merge_pass(int key_bytes, int tile_warps, long long S, bool xout, const void* in,
                              void* out, long long n, long long run_len, int K,
                              const long long* table, int* dev_err, cudaStream_t s,
                              bool test_timeout = false, bool pdl = false,
                              bool partition = false);

// Records the detail message mms_last_error_detail() returns on this thread.
void set_error_detail(const char* msg);

// Launches `kernel` on `s`, with programmatic stream serialization when `pdl`
// (the kernel must call griddep_wait() before its first global memory access;
// see mms_common.cuh).  Where the stream or device refuses the attribute, the
// launch is repeated without it.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  if (e != cudaSuccess && pdl && (e == cudaErrorNotSupported || e == cudaErrorInvalidValue)) {
    (void)cudaGetLastError();
    cfg.numAttrs = 0;
    e = cudaLaunchKernelEx(&cfg, kernel, args...);
  }
  return e;
}

// Output tiles of a round: every group of K runs (K * run_len items, the last
// group possibly short) is cut into tiles of S items, the last tile of every
// group possibly short.
__host__ __device__ inline long long tiles_per_group(long long S, long long run_len, int K) {
  return (run_len * K + S - 1) / S;
}
__host__ __device__ inline long long num_tiles(long long S, long long n, long long run_len, int K) {
  const long long G = run_len * K;
  const long long full = n / G;
  const long long rest = n - full * G;
  return full * tiles_per_group(S, run_len, K) + (rest + S - 1) / S;
}

}  // namespace mms
