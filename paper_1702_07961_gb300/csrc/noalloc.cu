// noalloc.cu -- a sort entry point that allocates no device memory.
//
// Some callers cannot allocate device memory at the time they need a sort:
// a process whose device memory is owned by another allocator (a framework
// that reserves the whole GPU up front and must not be bypassed), or a
// service with a fixed memory budget that must not grow while it runs, or a
// plugin that may not call cudaMalloc because cudaMalloc can synchronise the
// device.  mms_sort_keys_noalloc serves them: its workspace is a file-scope
// __device__ array of fixed size, so the call itself never allocates.  The
// price is that every GPU that loads this library holds the array (about
// 4 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mms.h"

namespace {

// Largest sorts served: 2^20 keys of 4 bytes or 2^19 keys of 8 bytes (4 MiB
// of keys), whose workspace is 4 MiB + 257 rows of pivot table + status word.
constexpr size_t kNoAllocMaxKeys4 = MMS_NOALLOC_MAX_KEYS_4B;
constexpr size_t kNoAllocMaxKeys8 = MMS_NOALLOC_MAX_KEYS_8B;
constexpr size_t kNoAllocScratchBytes = (size_t(4) << 20) + (size_t(128) << 10);
constexpr int kMaxDevices = 64;

// The scratch itself: one copy per device, alive until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" mms_status mms_sort_keys_noalloc(mms_key_type kt, void* d_keys, size_t n,
                                            void* stream) {
  if (kt != MMS_KEY_U32 && kt != MMS_KEY_U64 && kt != MMS_KEY_F32) return MMS_ERR_INVALID_ARG;
  const size_t max_keys = (kt == MMS_KEY_U64) ? kNoAllocMaxKeys8 : kNoAllocMaxKeys4;
  if (n > max_keys) return MMS_ERR_INVALID_ARG;   // beyond the fixed scratch: rejected, nothing queued
  if (n <= 1) return MMS_OK;
  if (mms_sort_workspace_bytes(kt, n, 0) > kNoAllocScratchBytes) return MMS_ERR_INTERNAL;

  // Once per device, with that device current: the device address of this
  // device's copy of the array.  Host code may not use the array's name as an
  // address; only the address returned here is valid for kernels.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MMS_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || p == nullptr) return MMS_ERR_CUDA;
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  // The array keeps the previous call's contents: its status word must start
  // at zero.  The rest (ping-pong keys, pivot table) is fully overwritten.
  if (cudaMemsetAsync(scratch, 0, 256, (cudaStream_t)stream) != cudaSuccess) return MMS_ERR_CUDA;
  return mms_sort_keys_ex(kt, d_keys, n, scratch, kNoAllocScratchBytes, stream, nullptr);
}
