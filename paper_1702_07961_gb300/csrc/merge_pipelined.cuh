// merge_pipelined.cuh -- launcher of the pipelined variant of a K-way merge
// round (merge_pipelined.cu).
#pragma once

#include <cuda_runtime.h>

namespace mms {

// One K-way merge round with persistent CTAs that pipeline their tiles: a
// producer warp plans and stages tile q + 1 while the merging warps merge
// tile q.  Same table, inputs and output as launch_merge_pass with the
// default tile geometry (S = 1024 * default_tile_warps(key_bytes)).
cudaError_t launch_merge_pipelined(int key_bytes, bool xout, const void* in, void* out, long long n,
                                   long long run_len, int K, const long long* table, int* dev_err,
                                   cudaStream_t s, bool pdl);

}  // namespace mms
