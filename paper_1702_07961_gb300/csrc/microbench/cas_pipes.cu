// cas_pipes.cu -- throughput of compare-exchange forms on sm_103a: min and
// max on the ALU pipe, against the larger key computed as a + b - min(a, b)
// by integer multiply-adds on the FMA pipe, and mixes of the two.
//
// Not part of libmms.so.  Each thread runs `iters` times the five-stage
// in-register cascade of the block merge (strides 16 .. 1 over 32 registers,
// 80 compare-exchanges) on its own keys, with one of eight forms:
//   0  min + max
//   1  min + two multiply-adds (max = a + b - min)
//   2  per-lane direction: min + max + two selects
//   3  per-lane direction: min + max + four multiply-adds
//   4  per-lane direction: min + six multiply-adds
//   5  11 of 16 pairs as form 1, the rest as form 0 (the kernels' mix)
//   6  per-lane direction: 10 of 16 pairs as min + four multiply-adds, the
//      rest as form 2 (the kernels' mix)
//   7  per-lane direction: min + four multiply-adds for every pair
// The multiply-adds use a runtime 1 (blockDim.x >> 8 with 256 threads) so
// that they stay multiplies.  Every form is exact modulo 2^32: forms 0, 1, 5
// must give identical results, and so must forms 2, 3, 4, 6, 7; the program
// checks that and exits non-zero otherwise.
//
// Build and run (sm_103a):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o cas_pipes paper_1702_07961_gb300/csrc/microbench/cas_pipes.cu
//   ./cas_pipes
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

namespace {

__device__ __forceinline__ uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

template <int V>
__global__ void __launch_bounds__(256) cas_forms(const uint32_t* in, uint32_t* out, int iters) {
  uint32_t v[32];
  const uint32_t one = blockDim.x >> 8, m1 = 0u - one, m2 = m1 + m1;
  const uint32_t f = (threadIdx.x >> 2) & 1;   // per-lane direction (0/1)
  const bool fb = f != 0;
  for (int j = 0; j < 32; ++j) v[j] = in[(blockIdx.x * 256 + threadIdx.x) * 32 % 4096 + j] ^ threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if ((j & s) != 0) continue;
        const uint32_t a = v[j], b = v[j + s];
        const int i = (j & (s - 1)) | ((j >> 1) & ~(s - 1));   // ordinal of the pair in the stage
        if constexpr (V == 0) {
          v[j] = min(a, b);
          v[j + s] = max(a, b);
        }
        if constexpr (V == 1) {
          const uint32_t lo = min(a, b), sm = mad(a, one, b);
          v[j] = lo;
          v[j + s] = mad(lo, m1, sm);
        }
        if constexpr (V == 2) {
          const uint32_t lo = min(a, b), hi = max(a, b);
          v[j] = fb ? hi : lo;
          v[j + s] = fb ? lo : hi;
        }
        if constexpr (V == 3) {
          const uint32_t lo = min(a, b), hi = max(a, b), d = mad(lo, m1, hi), na = mad(f, d, lo);
          v[j] = na;
          v[j + s] = mad(na, m1, mad(lo, one, hi));
        }
        if constexpr (V == 4) {
          const uint32_t lo = min(a, b), sm = mad(a, one, b), hi = mad(lo, m1, sm);
          const uint32_t d = mad(lo, m1, hi), na = mad(f, d, lo);
          v[j] = na;
          v[j + s] = mad(na, m1, sm);
        }
        if constexpr (V == 5) {
          if (i % 3 != 2) {
            const uint32_t lo = min(a, b), sm = mad(a, one, b);
            v[j] = lo;
            v[j + s] = mad(lo, m1, sm);
          } else {
            v[j] = min(a, b);
            v[j + s] = max(a, b);
          }
        }
        if constexpr (V == 6) {
          if (i % 7 < 4 || i >= 14) {
            const uint32_t lo = min(a, b), sm = mad(a, one, b), d = mad(lo, m2, sm), na = mad(f, d, lo);
            v[j] = na;
            v[j + s] = mad(na, m1, sm);
          } else {
            const uint32_t lo = min(a, b), hi = max(a, b);
            v[j] = fb ? hi : lo;
            v[j + s] = fb ? lo : hi;
          }
        }
        if constexpr (V == 7) {
          const uint32_t lo = min(a, b), sm = mad(a, one, b), d = mad(lo, m2, sm), na = mad(f, d, lo);
          v[j] = na;
          v[j + s] = mad(na, m1, sm);
        }
      }
    }
  }
  uint32_t acc = 0;
  for (int j = 0; j < 32; ++j) acc = acc * 31 + v[j];
  out[blockIdx.x * 256 + threadIdx.x] = acc;
}

template <int V>
float run(const uint32_t* din, uint32_t* dout, int blocks, int iters, std::vector<uint32_t>& res) {
  cas_forms<V><<<blocks, 256>>>(din, dout, iters);             // warm-up
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a);
  cas_forms<V><<<blocks, 256>>>(din, dout, iters);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  res.resize((size_t)blocks * 256);
  cudaMemcpy(res.data(), dout, res.size() * 4, cudaMemcpyDeviceToHost);
  return ms;
}

}  // namespace

int main() {
  const int blocks = 152 * 3, iters = 2000;
  uint32_t *din = nullptr, *dout = nullptr;
  if (cudaMalloc(&din, 4096 * 4 + 32 * 4) != cudaSuccess) return 1;
  if (cudaMalloc(&dout, (size_t)blocks * 256 * 4) != cudaSuccess) return 1;
  std::vector<uint32_t> h(4096 + 32);
  uint32_t x = 12345u;
  for (auto& y : h) y = (x = x * 1664525u + 1013904223u);
  cudaMemcpy(din, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
  const double cas = (double)blocks * 256 * iters * 5 * 16;     // compare-exchanges per launch
  const char* names[8] = {"min + max", "min + 2 mad", "dir: min/max + 2 sel", "dir: min/max + 4 mad",
                          "dir: min + 6 mad", "mix 11/16 min + 2 mad", "dir: mix 10/16 min + 4 mad",
                          "dir: min + 4 mad"};
  std::vector<std::vector<uint32_t>> res(8);
  float t[8] = {run<0>(din, dout, blocks, iters, res[0]), run<1>(din, dout, blocks, iters, res[1]),
                run<2>(din, dout, blocks, iters, res[2]), run<3>(din, dout, blocks, iters, res[3]),
                run<4>(din, dout, blocks, iters, res[4]), run<5>(din, dout, blocks, iters, res[5]),
                run<6>(din, dout, blocks, iters, res[6]), run<7>(din, dout, blocks, iters, res[7])};
  for (int i = 0; i < 8; ++i)
    std::printf("%-28s %8.3f ms  %6.2f compare-exchanges / clk / SM at 2.07 GHz\n", names[i], t[i],
                cas / (t[i] * 1e-3) / 152 / 2.07e9);
  const bool same_plain = res[1] == res[0] && res[5] == res[0];
  const bool same_dir = res[3] == res[2] && res[4] == res[2] && res[6] == res[2] && res[7] == res[2];
  std::printf("plain forms identical: %s; per-lane-direction forms identical: %s\n",
              same_plain ? "yes" : "NO", same_dir ? "yes" : "NO");
  const cudaError_t e = cudaDeviceSynchronize();
  std::printf("%s\n", cudaGetErrorString(e));
  cudaFree(din);
  cudaFree(dout);
  return (e == cudaSuccess && same_plain && same_dir) ? 0 : 1;
}
