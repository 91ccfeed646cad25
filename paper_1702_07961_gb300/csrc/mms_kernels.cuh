// mms_kernels.cuh -- host-side launchers of the three hot-path kernels and
// their fixed tile geometry.  Tile size S = 1024 * warps: 8 warps (8192 keys)
// for 4-byte keys, 4 warps (4096 keys) for 8-byte keys, so that two CTAs'
// shared memory (two tile buffers plus the per-warp transpose scratch) fit in
// one SM.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace mms {

constexpr int kTileWarps32 = 8;
constexpr int kTileWarps64 = 4;
constexpr int kMaxFanout = 32;

// Device error word values (the first word of a sort workspace).
constexpr int kDevOk = 0;
constexpr int kDevErrTimeout = 1;       // an mbarrier wait ran out of its bound
constexpr int kDevErrInternal = 2;      // a consistency check failed

inline int tile_warps(int key_bytes) { return key_bytes == 8 ? kTileWarps64 : kTileWarps32; }
inline long long tile_items(int key_bytes) { return 1024ll * tile_warps(key_bytes); }

size_t tile_sort_smem_bytes(int key_bytes, int warps);
size_t merge_pass_smem_bytes(int key_bytes, int warps);

// Base case: sorts every tile of tile_items(key_bytes) keys; in == out allowed.
// xin / xout: apply the float order transform on load / its inverse on store.
cudaError_t launch_tile_sort(int key_bytes, bool xin, bool xout, const void* in, void* out,
                             long long n, cudaStream_t s);

// Splitter: co-ranks of every output tile start of every group of K runs.
cudaError_t launch_splitter(int key_bytes, const void* in, long long n, long long run_len, int K,
                            long long* table, cudaStream_t s);

// One K-way merge round driven by the splitter table.
cudaError_t launch_merge_pass(int key_bytes, bool xout, const void* in, void* out, long long n,
                              long long run_len, int K, const long long* table, int* dev_err,
                              cudaStream_t s);

inline long long tiles_per_group(int key_bytes, long long run_len, int K) {
  return run_len * K / tile_items(key_bytes);
}
inline long long num_tiles(int key_bytes, long long n, long long run_len, int K) {
  const long long S = tile_items(key_bytes);
  const long long G = run_len * K;
  const long long full = n / G;
  const long long rest = n - full * G;
  return full * (G / S) + (rest + S - 1) / S;
}

}  // namespace mms
