// pairs.cu -- the key-value sort's own kernels.  Last step of the 4-byte
// key-value sort:  The sort itself runs on unique
// 64-bit composites (ordered 32-bit key << 32 | original array position), so
// equal keys keep their input order (stability) and every sorted composite
// names the position its value came from.  This kernel writes the keys back
// (undoing the float transform when asked) and gathers each value from a copy
// of the original values: keys and composites move coalesced, values by one
// gather per item.
#include "mms_common.cuh"
#include "mms_kernels.cuh"

namespace mms {

template <bool XOUT>
__global__ void __launch_bounds__(256)
    pairs_finalize_kernel(const uint64_t* __restrict__ comp, const uint32_t* __restrict__ vals_src,
                          uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                          long long n) {
  // 16-byte stores where both outputs lie on the 16-byte grid (keys and values
  // may start at any 4-byte offset), one item at a time otherwise.
  const bool vec = (((uintptr_t)keys_out | (uintptr_t)vals_out) & 15u) == 0;
  const long long nq = vec ? n / 4 : 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
    const ulonglong2 a = reinterpret_cast<const ulonglong2*>(comp)[2 * q];
    const ulonglong2 b = reinterpret_cast<const ulonglong2*>(comp)[2 * q + 1];
    const uint64_t c[4] = {a.x, a.y, b.x, b.y};
    uint32_t k[4], v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      k[i] = (uint32_t)(c[i] >> 32);
      if (XOUT) k[i] = ordered_to_f32(k[i]);
      v[i] = __ldg(vals_src + (uint32_t)c[i]);
    }
    reinterpret_cast<uint4*>(keys_out)[q] = make_uint4(k[0], k[1], k[2], k[3]);
    reinterpret_cast<uint4*>(vals_out)[q] = make_uint4(v[0], v[1], v[2], v[3]);
  }
  for (long long i = nq * 4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t c = comp[i];
    uint32_t k = (uint32_t)(c >> 32);
    if (XOUT) k = ordered_to_f32(k);
    keys_out[i] = k;
    vals_out[i] = vals_src[(uint32_t)c];
  }
}

cudaError_t launch_pairs_finalize(bool xout, const void* comp64, const void* vals_src,
                                  void* keys_out, void* vals_out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long quads = (n + 3) / 4;
  long long blocks = (quads + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  const auto* c = static_cast<const uint64_t*>(comp64);
  const auto* vs = static_cast<const uint32_t*>(vals_src);
  auto* ko = static_cast<uint32_t*>(keys_out);
  auto* vo = static_cast<uint32_t*>(vals_out);
  if (xout)
    pairs_finalize_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(c, vs, ko, vo, n);
  else
    pairs_finalize_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(c, vs, ko, vo, n);
  return cudaGetLastError();
}

// ---- key-value sorting of 8-byte keys -----------------------------------------
//
// Two stable passes of the 4-byte key-value sort, least significant half
// first (the textbook LSD composition of stable sorts): pass 1 sorts the
// items' positions by the low 32 key bits, pass 2 sorts the resulting
// position list by the high 32 key bits of the items it names.  Equal high
// halves keep pass 1's order, which is by (low half, position), so the final
// list is ordered by (key, position): the stable key order.  These kernels
// prepare the passes and apply the final permutation.

__global__ void __launch_bounds__(256)
    u64_split_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                     uint32_t* __restrict__ lo, uint32_t* __restrict__ perm,
                     uint64_t* __restrict__ kcopy, uint32_t* __restrict__ vcopy, long long n,
                     long long pos0) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t k = keys[i];
    lo[i] = (uint32_t)k;
    perm[i] = (uint32_t)(pos0 + i);
    kcopy[i] = k;
    vcopy[i] = vals[i];
  }
}

__global__ void __launch_bounds__(256)
    u64_hi_kernel(const uint64_t* __restrict__ kcopy, const uint32_t* __restrict__ perm,
                  uint32_t* __restrict__ hi, long long n, long long pos0) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    hi[i] = (uint32_t)(kcopy[(long long)perm[i] - pos0] >> 32);
}

__global__ void __launch_bounds__(256)
    u64_final_kernel(const uint64_t* __restrict__ kcopy, const uint32_t* __restrict__ vcopy,
                     const uint32_t* __restrict__ perm, uint64_t* __restrict__ keys,
                     uint32_t* __restrict__ vals, long long n, long long pos0) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long p = (long long)perm[i] - pos0;
    keys[i] = kcopy[p];
    vals[i] = vcopy[p];
  }
}

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_u64_pairs_split(const void* keys, const void* vals, void* lo, void* perm,
                                   void* kcopy, void* vcopy, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  u64_split_kernel<<<grid_for(n), 256, 0, s>>>(
      static_cast<const uint64_t*>(keys), static_cast<const uint32_t*>(vals),
      static_cast<uint32_t*>(lo), static_cast<uint32_t*>(perm), static_cast<uint64_t*>(kcopy),
      static_cast<uint32_t*>(vcopy), n, 0);
  return cudaGetLastError();
}

cudaError_t launch_u64_pairs_hi(const void* kcopy, const void* perm, void* hi, long long n,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  u64_hi_kernel<<<grid_for(n), 256, 0, s>>>(static_cast<const uint64_t*>(kcopy),
                                             static_cast<const uint32_t*>(perm),
                                             static_cast<uint32_t*>(hi), n, 0);
  return cudaGetLastError();
}

cudaError_t launch_u64_pairs_final(const void* kcopy, const void* vcopy, const void* perm,
                                   void* keys, void* vals, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  u64_final_kernel<<<grid_for(n), 256, 0, s>>>(
      static_cast<const uint64_t*>(kcopy), static_cast<const uint32_t*>(vcopy),
      static_cast<const uint32_t*>(perm), static_cast<uint64_t*>(keys),
      static_cast<uint32_t*>(vals), n, 0);
  return cudaGetLastError();
}

}  // namespace mms
