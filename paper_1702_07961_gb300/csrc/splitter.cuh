// splitter.cuh -- parallel partitioning of a K-way merge round (Sec. 4.1),
// shared by the whole-array splitter and the segmented (batched) one.
//
// For every output tile j of every group of K sorted runs, one lane group
// (W >= K lanes, 32 / W groups per warp) finds the pivot indices c[r]
// (r < K): the number of items run r contributes to the group's first j*S
// outputs under the strict order (key, run, position).  That
// order makes the pivots unique even with repeated keys (the paper's
// non-overlap condition, read on the composite key) and equals a stable merge.
//
// Search (one lane per run, K <= 32): stride halving on regular samples.  At
// stride s the lane group holds the exact pivots d of the s-sample problem -- the
// items at positions s-1, 2s-1, ... of every run -- for rank floor(k/s).
// Halving s adds one candidate per run just above its pivot; the pivots of the
// s/2-sample problem for rank floor(2k/s) are then the floor(2k/s) smallest of
// (old selection expanded) + (candidates), found by dropping the largest items
// from the top with arg-max reductions over the lane group.  At s = 1 the sample problem is
// the whole problem.  About log2(k) rounds of two independent loads per lane.
// Positions past a run's end are padding items ordered after every real item
// (by run, then position).
#pragma once

#include "mms_common.cuh"
#include "mms_kernels.cuh"

namespace mms {

template <typename KeyT>
struct Item {
  KeyT key;
  bool pad;
};

template <typename KeyT, typename Idx>
__device__ __forceinline__ Item<KeyT> load_item(const KeyT* run, Idx len, Idx pos) {
  Item<KeyT> it;
  it.pad = pos >= len;
  it.key = it.pad ? KeyT(0) : run[pos];
  return it;
}

// a (run ra) strictly before b (run rb), ra != rb.
template <typename KeyT>
__device__ __forceinline__ bool before_cross(const Item<KeyT>& a, int ra, const Item<KeyT>& b,
                                             int rb) {
  if (a.pad != b.pad) return b.pad;
  if (!a.pad && a.key != b.key) return a.key < b.key;
  return ra < rb;
}

// Every reduction below runs over one lane group: the lanes of the mask gm
// (W consecutive lanes aligned to W; all of them execute the call).  A warp
// holds 32 / W groups, each working on its own output tile.
__device__ __forceinline__ uint32_t grp_max_u32(unsigned gm, uint32_t v) {
  return __reduce_max_sync(gm, v);
}
__device__ __forceinline__ uint32_t grp_min_u32(unsigned gm, uint32_t v) {
  return __reduce_min_sync(gm, v);
}

// Lanes with `cond` whose key equals the maximum key among them.
__device__ __forceinline__ unsigned lanes_with_max(unsigned gm, bool cond, uint32_t key) {
  const uint32_t mx = grp_max_u32(gm, cond ? key : 0u);
  return __ballot_sync(gm, cond && key == mx);
}
__device__ __forceinline__ unsigned lanes_with_max(unsigned gm, bool cond, uint64_t key) {
  const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
  const uint32_t mh = grp_max_u32(gm, cond ? hi : 0u);
  const bool c2 = cond && hi == mh;
  const uint32_t ml = grp_max_u32(gm, c2 ? lo : 0u);
  return __ballot_sync(gm, c2 && lo == ml);
}
__device__ __forceinline__ unsigned lanes_with_min(unsigned gm, bool cond, uint32_t key) {
  const uint32_t mn = grp_min_u32(gm, cond ? key : 0xffffffffu);
  return __ballot_sync(gm, cond && key == mn);
}
__device__ __forceinline__ unsigned lanes_with_min(unsigned gm, bool cond, uint64_t key) {
  const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
  const uint32_t mh = grp_min_u32(gm, cond ? hi : 0xffffffffu);
  const bool c2 = cond && hi == mh;
  const uint32_t ml = grp_min_u32(gm, c2 ? lo : 0xffffffffu);
  return __ballot_sync(gm, c2 && lo == ml);
}

// Lane holding the largest item among lanes with `cond` (runs compare by
// (pad, key, run)); -1 if none.  Lane numbers are the warp's.
template <typename KeyT>
__device__ __forceinline__ int grp_argmax(unsigned gm, bool cond, const Item<KeyT>& it) {
  if constexpr (sizeof(KeyT) == 4) {
    // One max over the keys with pads raised to the all-ones key, then the
    // lanes holding that maximum: a pad among them wins (pads come after
    // every real key, an all-ones real key included), else the highest lane
    // (the largest run index).  The pad ballot does not wait for the max.
    const uint32_t kk = cond ? (it.pad ? 0xffffffffu : (uint32_t)it.key) : 0u;
    const uint32_t mx = grp_max_u32(gm, kk);
    const unsigned padm = __ballot_sync(gm, cond && it.pad);
    const unsigned m = __ballot_sync(gm, cond && kk == mx);
    const unsigned mp = m & padm;
    return m ? 31 - __clz(mp ? mp : m) : -1;
  } else {
    const unsigned any = __ballot_sync(gm, cond);
    if (!any) return -1;
    const unsigned pads = __ballot_sync(gm, cond && it.pad);
    if (pads) return 31 - __clz(pads);
    return 31 - __clz(lanes_with_max(gm, cond, it.key));
  }
}

// grp_argmax when no lane of the group holds a pad: one max and one ballot
// (4-byte keys), or the two-word maximum (8-byte keys).
template <typename KeyT>
__device__ __forceinline__ int grp_argmax_real(unsigned gm, bool cond, KeyT key) {
  if constexpr (sizeof(KeyT) == 4) {
    const uint32_t mx = grp_max_u32(gm, cond ? (uint32_t)key : 0u);
    const unsigned m = __ballot_sync(gm, cond && (uint32_t)key == mx);
    return m ? 31 - __clz(m) : -1;
  } else {
    if (!__ballot_sync(gm, cond)) return -1;
    return 31 - __clz(lanes_with_max(gm, cond, key));
  }
}

template <typename KeyT>
__device__ __forceinline__ int grp_argmin(unsigned gm, bool cond, const Item<KeyT>& it) {
  const unsigned any = __ballot_sync(gm, cond);
  if (!any) return -1;
  const unsigned reals = __ballot_sync(gm, cond && !it.pad);
  if (!reals) return __ffs(any) - 1;
  return __ffs(lanes_with_min(gm, cond && !it.pad, it.key)) - 1;
}

template <typename KeyT>
__device__ __forceinline__ Item<KeyT> shfl_item(unsigned gm, const Item<KeyT>& it, int src) {
  Item<KeyT> o;
  o.key = __shfl_sync(gm, it.key, src);
  o.pad = __shfl_sync(gm, (int)it.pad, src) != 0;
  return o;
}

// The search itself: the lanes of the group (lane gb + r on run r, act for
// r < K) return the number of items each run contributes to the first k of
// the K runs' merge under the order (key, run, position).  `run` and `rlen`
// are the lane's run and its length (rlen = 0 when !act); the runs may lie in
// global or in shared memory.  Arguments other than run / rlen / act are
// uniform over the lane group; every lane of it must call.
// UNSWITCH: one drop loop per arg-max form (no pad test inside the loop);
// measured faster in the splitter kernel (splitter_row), slower inside the
// much larger partition merge kernel, which takes the default single loop.
template <typename KeyT, typename Idx, bool UNSWITCH = false>
__device__ __forceinline__ Idx multiseq_pivot(const KeyT* run, Idx rlen, bool act, int K, Idx k,
                                              unsigned gm) {
  const int lane = threadIdx.x & 31;
  Idx d = 0;                  // selected samples of this run at the current stride
  Item<KeyT> e{KeyT(0), false};  // the d-th sample (position d*s-1) when d >= 1
  const int T = 64 - __clzll((long long)k);
  bool pad_prev = true;       // the previous level had a pad candidate (so e may be a pad)
  for (int lev = T; lev >= 1; --lev) {
    const int sh = lev - 1;                     // s2 = 2^sh
    const Idx kp = k >> sh;
    const Idx dd = 2 * d;
    Item<KeyT> o = load_item(run, rlen, ((dd + 1) << sh) - 1);
    Item<KeyT> z{KeyT(0), false};
    if (d >= 1) z = load_item(run, rlen, ((dd - 1) << sh) - 1);
    // The largest selected item (lane mz's e) needs none of the new loads:
    // its reduction overlaps them.  e is a pad only if the previous level had
    // a pad candidate.
    const bool hasZ = act && d >= 1;
    const int mz = pad_prev ? grp_argmax(gm, hasZ, e) : grp_argmax_real(gm, hasZ, e.key);
    Item<KeyT> zmax{KeyT(0), false};
    if (mz >= 0) zmax = pad_prev ? shfl_item(gm, e, mz) : Item<KeyT>{__shfl_sync(gm, e.key, mz), false};
    // Pads at this level: o is a lane's highest position, so when no o is a
    // pad, no item of the level is (e, z and any deeper item lie below o).
    const bool any_pad = __any_sync(gm, act && o.pad);
    // Items to drop: (sum of the lanes' 2d + 1) - kp.  The lanes hold the
    // pivots of rank k >> lev, so the d sum to k >> (sh + 1) and the count is
    // K minus the low bit of kp: K - 1 or K, with no reduction.
    const Idx jrem = (Idx)K - (kp & 1);
    Idx cnt = dd + 1;

    // Candidates above every selected item are dropped first, in one step.
    bool above = act;
    if (mz >= 0) {
      if (any_pad) {
        above = act && (lane == mz || before_cross(zmax, mz, o, lane));
      } else {                                  // no pads: keys, then runs
        above = act && (lane == mz || zmax.key < o.key || (zmax.key == o.key && mz < lane));
      }
    }
    const unsigned abovem = __ballot_sync(gm, above);
    const Idx u = __popc(abovem);
    Idx pops;
    if (u <= jrem) {
      if (above) cnt = dd;
      pops = jrem - u;
    } else {                                    // keep only the smallest candidate
      const int mn = grp_argmin(gm, above, o);
      if (above && lane != mn) cnt = dd;
      pops = 0;
    }
    // Remaining drops one at a time from the largest current top.  The first
    // needs no reduction: the largest top is lane mz's e (every candidate
    // above it was dropped, mz's own included), and mz then falls back to z.
    Item<KeyT> top = (cnt == dd + 1) ? o : e;
    if (mz >= 0 && pops > 0) {                  // uniform over the group
      if (lane == mz) {
        cnt = dd - 1;                           // d >= 1 on lane mz, so cnt >= 1
        top = z;
      }
      pops -= 1;
    }
    auto drop = [&](int w) {
      if (lane == w) {
        cnt -= 1;
        if (cnt >= 1) {
          if (cnt == dd)
            top = e;
          else if (cnt == dd - 1)
            top = z;
          else
            top = load_item(run, rlen, (cnt << sh) - 1);
        }
      }
    };
    if constexpr (UNSWITCH) {
      if (any_pad) {
        for (Idx p = 0; p < pops; ++p) drop(grp_argmax(gm, act && cnt >= 1, top));
      } else {
        for (Idx p = 0; p < pops; ++p) drop(grp_argmax_real(gm, act && cnt >= 1, top.key));
      }
    } else {
      for (Idx p = 0; p < pops; ++p)
        drop(any_pad ? grp_argmax(gm, act && cnt >= 1, top)
                     : grp_argmax_real(gm, act && cnt >= 1, top.key));
    }
    d = cnt;
    e = top;
    pad_prev = any_pad;
  }
  return d;
}

// Pivots of output tile j of group g, found by one lane group of W >= K lanes
// (gm: its lanes, gb: its first lane; lane gb + r handles run r): row[r]
// receives the number of items of run r among the group's first j * S
// outputs.  Arguments are uniform over the lane group.  Idx is the type of
// the counts and positions of the search: int when n < 2^30 (every position
// probed stays below 2n), long long otherwise.
template <typename KeyT, int W, typename Idx = long long>
__device__ __forceinline__ void splitter_row(const KeyT* __restrict__ in, long long n,
                                             long long run_len, int K, long long S, long long g,
                                             long long j, long long* __restrict__ row,
                                             unsigned gm, int gb) {
  const int lane = threadIdx.x & 31;
  const int rr = lane - gb;                     // run of this lane
  const bool act = rr < K;
  const long long rstart = g * run_len * K + (long long)rr * run_len;
  long long rlen64 = n - rstart;
  rlen64 = rlen64 < 0 ? 0 : (rlen64 > run_len ? run_len : rlen64);
  const Idx rlen = act ? (Idx)rlen64 : Idx(0);
  const KeyT* run = in + (act ? rstart : 0);
  const Idx d = multiseq_pivot<KeyT, Idx, true>(run, rlen, act, K, (Idx)(j * S), gm);
  if (act) row[rr] = d;
}

}  // namespace mms
