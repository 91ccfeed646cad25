// pairs.cu -- last step of the key-value sort.  The sort itself runs on unique
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
  const long long nq = n / 4;
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

}  // namespace mms
