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
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mms.h"
#include "mms_kernels.cuh"

namespace {

// Largest sorts served: 2^20 keys of 4 bytes or 2^19 keys of 8 bytes (4 MiB
// of keys), whose workspace is 4 MiB + 257 rows of pivot table + status word.
constexpr size_t kNoAllocMaxKeys4 = MMS_NOALLOC_MAX_KEYS_4B;
constexpr size_t kNoAllocMaxKeys8 = MMS_NOALLOC_MAX_KEYS_8B;
constexpr size_t kNoAllocScratchBytes = (size_t(4) << 20) + (size_t(128) << 10);
constexpr int kMaxDevices = 64;

// The scratch itself: one copy per device, alive until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// The device address of the array, cached per device together with the CUDA
// context it was looked up in: a device reset creates a new primary context,
// and an address from the old one must not be used again.
struct ScratchAddr {
  CUcontext ctx;
  void* ptr;
};
std::mutex g_mu;
ScratchAddr g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
bool g_ctx_fn_looked_up = false;

// The current context, through the driver entry point the runtime hands out
// (the library does not link the driver library itself).  nullptr when the
// lookup fails; the cache then never matches and the address is looked up on
// every call, which is correct, only slower.
CUcontext current_context() {
  if (!g_ctx_fn_looked_up) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    g_ctx_fn_looked_up = true;
  }
  CUcontext c = nullptr;
  if (g_ctx_get_current == nullptr || g_ctx_get_current(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

mms_status fail_detail(mms_status s, const char* msg) {
  mms::set_error_detail(msg);
  return s;
}

// This device's address of the scratch array (set-up, with the device
// current: the first call on a device, and again after a device reset).
mms_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail_detail(MMS_ERR_CUDA, "mms_sort_keys_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_mu);
  const CUcontext ctx = current_context();
  ScratchAddr& e = g_scratch[dev];
  if (e.ptr == nullptr || ctx == nullptr || e.ctx != ctx) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess || p == nullptr)
      return fail_detail(MMS_ERR_CUDA, "mms_sort_keys_noalloc: cudaGetSymbolAddress failed");
    e.ptr = p;
    e.ctx = current_context();   // the lookup has made the device's context current
  }
  *out = e.ptr;
  return MMS_OK;
}

}  // namespace

extern "C" mms_status mms_sort_keys_noalloc(mms_key_type kt, void* d_keys, size_t n,
                                            void* stream) {
  if (kt != MMS_KEY_U32 && kt != MMS_KEY_U64 && kt != MMS_KEY_F32)
    return fail_detail(MMS_ERR_INVALID_ARG, "mms_sort_keys_noalloc: unknown key type");
  const size_t max_keys = (kt == MMS_KEY_U64) ? kNoAllocMaxKeys8 : kNoAllocMaxKeys4;
  if (n > max_keys)   // beyond the fixed scratch: rejected, nothing queued
    return fail_detail(MMS_ERR_INVALID_ARG,
                       "mms_sort_keys_noalloc: n above MMS_NOALLOC_MAX_KEYS_4B / _8B");
  if (n <= 1) return MMS_OK;
  if (mms_sort_workspace_bytes(kt, n, 0) > kNoAllocScratchBytes)
    return fail_detail(MMS_ERR_INTERNAL, "mms_sort_keys_noalloc: scratch smaller than the workspace");

  // Host code may not use the array's name as an address; only the address
  // looked up here is valid for kernels.
  void* scratch = nullptr;
  const mms_status st = scratch_address(&scratch);
  if (st != MMS_OK) return st;
  // The array keeps the previous call's contents; mms_sort_keys_ex clears the
  // status word of a caller's workspace first, and the rest (ping-pong keys,
  // pivot table) is fully overwritten.
  return mms_sort_keys_ex(kt, d_keys, n, scratch, kNoAllocScratchBytes, stream, nullptr);
}

extern "C" mms_status mms_noalloc_status(void* stream) {
  void* scratch = nullptr;
  const mms_status st = scratch_address(&scratch);
  if (st != MMS_OK) return st;
  return mms_workspace_status(scratch, kNoAllocScratchBytes, stream);
}
