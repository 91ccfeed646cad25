// merge_pipelined.cu -- the pipelined variant of a K-way merge round (the
// paper's future work, Sec. 7: pipelining the merge).
//
// Persistent CTAs of WARPS merging warps and one producer warp.  A CTA takes
// the output tiles t = blockIdx.x + q * gridDim.x, q = 0, 1, ..., and keeps
// three tile buffers.  Tile q is staged into buffer s(q) = -q mod 3 and merged
// with s(q) and p(q) = 1 - q mod 3 as its two level buffers, so while the
// merging warps work on tile q the producer plans tile q + 1 and stages it into
// the third buffer.  Barriers (mbarriers in shared memory):
//   full[b]  -- two arrivals and the bulk copies' bytes: the producer's
//              expect-tx arrival as it starts the copies, and its arrival once
//              the node table and the plainly loaded items are written;
//   empty[b] -- one arrival: the merging warps release p(q) when tile q is
//              stored, which is the buffer tile q + 2 is staged into.
// The producer's k-th wait on empty[b] and the merging warps' wait on
// full[s(q)] take the parity of the phase they must observe
// (tests/test_pipeline_model.py replays the rotation).  The plan, the merge
// levels and the store are those of the CTA-tree merge (merge_tile.cuh).  Every
// wait is bounded; on a time-out the CTA records MMS_ERR_TIMEOUT and stops.
#include "merge_pipelined.cuh"
#include "merge_tile.cuh"

namespace mms {
namespace {

__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32addr(bar))
               : "memory");
}

// Barrier over the merging warps only (named barrier 1).
template <int NT>
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}
// The same barrier, returning whether any participating thread passed `v`.
template <int NT>
__device__ __forceinline__ bool consumers_any(bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((unsigned)v), "n"(NT)
      : "memory");
  return r != 0;
}

template <typename KeyT, int WARPS>
struct PipeGeom {
  static constexpr int kCtlInts = (int)(kMergeCtlBytes / sizeof(int));
  __host__ __device__ static constexpr size_t buf_bytes(int K) {
    return sizeof(KeyT) * (size_t)MergeGeom<KeyT, WARPS>::cap(K);   // a multiple of 16
  }
  // three buffers, six mbarriers (64 bytes), three control areas
  __host__ __device__ static constexpr size_t bytes(int K) {
    return 3 * buf_bytes(K) + 64 + 3 * kMergeCtlBytes;
  }
};

template <typename KeyT, int WARPS, bool XOUT>
__global__ void __launch_bounds__((WARPS + 1) * 32, 2)
    merge_pipelined_kernel(const KeyT* __restrict__ in, KeyT* __restrict__ out, long long n,
                           long long run_len, int K, const long long* __restrict__ table,
                           long long tpg, long long ntiles, int S, int* dev_err) {
  using P = PipeGeom<KeyT, WARPS>;
  constexpr int NT = WARPS * 32;                  // merging threads
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const size_t bb = P::buf_bytes(K);
  auto buf = [&](int b) { return reinterpret_cast<KeyT*>(smem_raw + (size_t)b * bb); };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + 3 * bb);
  uint64_t* empty = full + 3;
  int* ctls = reinterpret_cast<int*>(smem_raw + 3 * bb + 64);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 3; ++b) {
      mbar_init(&full[b], 2);
      mbar_init(&empty[b], 1);
    }
  }
  __syncthreads();
  griddep_wait();                                 // the pivot table and the runs: earlier kernels'
  griddep_launch_dependents();

  if (warp == WARPS) {
    // Producer: plan and stage tile q into s(q) once tile q - 2 has released it.
    unsigned empty_par = 0u;                      // bit b: parity of the next wait on empty[b]
    long long staged = 0;                         // tiles staged so far
    for (long long q = 0;; ++q) {
      const long long t = (long long)blockIdx.x + q * gridDim.x;
      if (t >= ntiles) break;
      const int b = (int)((3 - q % 3) % 3);
      if (q >= 2) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait_bounded(&empty[b], (empty_par >> b) & 1u);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        empty_par ^= 1u << b;
        if (!ok) {
          if (lane == 0) set_device_error(dev_err, kDevErrTimeout);
          break;
        }
      }
      const long long g = t / tpg, j = t % tpg;
      long long lo = 0, hi = 0;
      merge_tile_pivots(n, run_len, K, g, j, table + t * K, table + (t + 1) * K, S, lane, lo, hi);
      int* ctl = ctls + b * P::kCtlInts;
      merge_plan_warp<KeyT, WARPS>(in, n, run_len, K, g, j, lo, hi, S, buf(b), ctl, &full[b], lane);
      __syncwarp();
      if (lane == 0) {
        // A rejected plan started no copies and made no expect-tx arrival.
        if (ctl[kCtlNodeFields * 32 + 3]) mbar_arrive_plain(&full[b]);
        mbar_arrive_plain(&full[b]);              // publishes the node table and plain loads
      }
      staged = q + 1;
    }
    // Before the warp leaves, the copies it started have landed: the last two
    // staged tiles are the only ones whose full phase the merging warps may not
    // have awaited (if they stopped early), and no later staging reuses their
    // buffers, so their parities are unambiguous.  Bounded, like every wait.
    if (lane == 0) {
      for (long long q = staged - 2; q < staged; ++q)
        if (q >= 0) (void)mbar_wait_bounded(&full[(int)((3 - q % 3) % 3)], (unsigned)((q / 3) & 1));
    }
    __syncwarp();
    return;
  }

  // Merging warps: tile q with the level buffers s(q) and p(q).
  for (long long q = 0;; ++q) {
    const long long t = (long long)blockIdx.x + q * gridDim.x;
    if (t >= ntiles) break;
    const int b = (int)((3 - q % 3) % 3), p = (int)((4 - q % 3) % 3);
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait_bounded(&full[b], (unsigned)((q / 3) & 1));
    if (consumers_any<NT>(!ok)) {
      if (threadIdx.x == 0) set_device_error(dev_err, kDevErrTimeout);
      return;                                     // uniform over the merging warps
    }
    const int* ctl = ctls + b * P::kCtlInts;
    const long long g = t / tpg, j = t % tpg;
    if (ctl[kCtlNodeFields * 32 + 3]) {
      if (threadIdx.x == 0) set_device_error(dev_err, kDevErrInternal);
    } else {
      merge_levels<KeyT, WARPS>(buf(b), buf(p), ctl, out + g * run_len * K + j * S, XOUT,
                                []() { consumers_sync<NT>(); });
    }
    // The store has read the tile and every thread is past its last read of
    // either buffer: release p(q) (the buffer tile q + 2 is staged into).
    fence_proxy_async_smem();
    consumers_sync<NT>();
    if (threadIdx.x == 0) mbar_arrive_plain(&empty[p]);
  }
}

template <typename KeyT, int WARPS, bool XOUT>
cudaError_t launch_t(const void* in, void* out, long long n, long long run_len, int K,
                     const long long* table, int* dev_err, cudaStream_t s, bool pdl) {
  const size_t smem = PipeGeom<KeyT, WARPS>::bytes(K);
  auto k = merge_pipelined_kernel<KeyT, WARPS, XOUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long S = 1024ll * WARPS;
  const long long ntiles = num_tiles(S, n, run_len, K);
  if (ntiles <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long per_sm = 2;                     // CTAs an SM holds (three buffers each)
  const long long grid = ntiles < per_sm * sms ? ntiles : per_sm * sms;
  long long tpg = tiles_per_group(S, run_len, K);
  if (tpg > 0xFFFFFFFFll) tpg = 0xFFFFFFFFll;
  return launch_k(k, dim3((unsigned)grid), dim3((WARPS + 1) * 32), smem, s, pdl,
                  static_cast<const KeyT*>(in), static_cast<KeyT*>(out), n, run_len, K, table, tpg,
                  ntiles, (int)S, dev_err);
}

}  // namespace

cudaError_t launch_merge_pipelined(int key_bytes, bool xout, const void* in, void* out, long long n,
                                   long long run_len, int K, const long long* table, int* dev_err,
                                   cudaStream_t s, bool pdl) {
  if (n <= 0) return cudaSuccess;
  if (K < 2 || K > kMaxFanout) return cudaErrorInvalidValue;
  if (key_bytes == 4)
    return xout ? launch_t<uint32_t, 8, true>(in, out, n, run_len, K, table, dev_err, s, pdl)
                : launch_t<uint32_t, 8, false>(in, out, n, run_len, K, table, dev_err, s, pdl);
  return launch_t<uint64_t, 4, false>(in, out, n, run_len, K, table, dev_err, s, pdl);
}

}  // namespace mms
