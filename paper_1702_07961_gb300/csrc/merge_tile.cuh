// merge_tile.cuh -- the CTA body of one K-way merge round (Sec. 4.2 "I/O
// Efficient Merging", Sec. 5.1 I/O analysis), shared by the whole-array merge
// pass and the segmented (batched) merge pass.
//
// One CTA produces one output tile of S = 1024 * WARPS items of its group of K
// runs.  The splitter table gives, for the tile's start and end, the pivot in
// every run (Sec. 4.1), so the tile's inputs are K contiguous segments whose
// lengths sum to S.  The CTA:
//   1. stages the K segments into shared memory with 1-D TMA bulk copies
//      (cp.async.bulk between 16-byte boundaries, one mbarrier; plain loads
//      only where a boundary would lie past the end of the array), so every
//      input byte is read from HBM once;
//   2. merges them along a binary merge tree of ceil(log2 K') levels, K' <= K
//      the runs the group holds (the paper's minBlockHeap has the same
//      levels), one level at a time: every
//      tree node of the level (a pair of sequences) is cut into 1024-item
//      output blocks, the blocks of the level are dealt to the warps (its
//      full-size blocks first, then the small last blocks of its nodes,
//      which a smaller network merges), and a CTA barrier separates the
//      levels.  A node's output is written into the
//      span its segments were staged in, alternating between two buffers by
//      level; every segment span carries 32 items of slack so that a node's
//      last, partial block can use its output region as transpose space.
//      Each block is merged by the conflict-free warp bitonic block merge;
//   3. writes the tile with one TMA bulk store, so every output byte is
//      written once: 2 * S * sizeof(key) bytes of HBM traffic per tile.
#pragma once

#include "mms_common.cuh"
#include "mms_kernels.cuh"
#include "splitter.cuh"

namespace mms {

// Control area after a merge CTA's mbarrier: the merge-tree node table (10
// fields x 32 nodes) and four scalars, written by warp 0 for the whole CTA.
constexpr int kCtlNodeFields = 10;
constexpr int kCtlScalars = 8;
constexpr size_t kMergeCtlBytes = sizeof(int) * (kCtlNodeFields * 32 + kCtlScalars);

// Shared-memory geometry of a merge CTA for fanout K.  X: the staged
// segments, each at a 16-byte aligned span start R_r (up to 2E-2 items of
// alignment slack and 32 items of transpose slack per segment), and the odd
// tree levels' inputs; Y: the same spans, one buffer per level parity.
template <typename KeyT, int WARPS>
struct MergeGeom {
  static constexpr int E = Vec16<KeyT>::E;
  static constexpr int S = WARPS * kBlockItems;
  static constexpr int kSlack = 32;
  __host__ __device__ static constexpr int cap(int K) { return S + K * (2 * E + kSlack) + E; }
  // control block: mbarrier (16 bytes with padding), then the node table
  __host__ __device__ static constexpr size_t bytes(int K) {
    return sizeof(KeyT) * 2 * (size_t)cap(K) + 16 + kMergeCtlBytes;
  }
  // The partition variant adds its pivot rows after the control area: row b
  // (b <= WARPS) holds, per segment, the items of the tile's first 1024 b
  // outputs.
  static constexpr size_t kRowBytes = sizeof(int) * 32 * (WARPS + 1);
  __host__ __device__ static constexpr size_t bytes_partition(int K) { return bytes(K) + kRowBytes; }
};

inline size_t merge_pass_smem_bytes_impl(int key_bytes, int warps, int K, bool partition = false) {
  if (key_bytes == 4) {
    switch (warps) {
      case 4: return partition ? MergeGeom<uint32_t, 4>::bytes_partition(K) : MergeGeom<uint32_t, 4>::bytes(K);
      case 8: return partition ? MergeGeom<uint32_t, 8>::bytes_partition(K) : MergeGeom<uint32_t, 8>::bytes(K);
    }
  } else {
    switch (warps) {
      case 2: return partition ? MergeGeom<uint64_t, 2>::bytes_partition(K) : MergeGeom<uint64_t, 2>::bytes(K);
      case 4: return partition ? MergeGeom<uint64_t, 4>::bytes_partition(K) : MergeGeom<uint64_t, 4>::bytes(K);
    }
  }
  return 0;
}

// Segment bounds of the tile in run `lane` (lanes < K): from the pivot rows,
// or the run's ends for a group's first / last tile.  Warp 0 issues these
// loads first thing, so they are in flight across the CTA's setup.
__device__ __forceinline__ void merge_tile_pivots(long long n, long long run_len, int K,
                                                  long long g, long long j,
                                                  const long long* __restrict__ lo_row,
                                                  const long long* __restrict__ hi_row, int S,
                                                  int lane, long long& lo, long long& hi) {
  const long long gstart = g * run_len * K;
  const long long grest = n - gstart;
  const long long gsize = grest < run_len * K ? grest : run_len * K;
  long long rlen = n - (gstart + (long long)lane * run_len);
  rlen = rlen < 0 ? 0 : (rlen > run_len ? run_len : rlen);
  lo = 0;
  hi = 0;
  if (lane < K) {
    lo = (j == 0) ? 0 : lo_row[lane];
    hi = ((j + 1) * S < gsize) ? hi_row[lane] : rlen;   // not the group's last tile
  }
}

// Plans output tile j of group g, whose segment bounds in run `lane` are lo
// and hi (from merge_tile_pivots), and stages its segments into `stage`: one
// warp, one lane per run and one per merge-tree node.  Starts the bulk copies
// on `bar`, loads the items no bulk copy covers, and writes the node table and
// the scalars (levels, nodes, tile size, error) into `ctl`; the caller's CTA
// barrier publishes the plain loads and the table, the barrier's phase the
// copies.  On segment bounds that fail their check, ctl's error scalar is set
// and nothing is staged.
// `part` splits the work between two warps that both call this with the same
// bounds: bit 0 stages the segments (and writes the tile size and error
// scalars), bit 1 writes the node table (and the level and node counts).  The
// two halves need only the segment lengths and spans, which both compute, so a
// CTA can start the copies and build the table at the same time.
template <typename KeyT, int WARPS>
__device__ __forceinline__ void merge_plan_warp(const KeyT* __restrict__ in, long long n,
                                                long long run_len, int K, long long g,
                                                long long j, long long lo, long long hi, int S,
                                                KeyT* stage, int* ctl, uint64_t* bar, int lane,
                                                int part = 3) {
  using G = MergeGeom<KeyT, WARPS>;
  constexpr int E = G::E;
  const long long gstart = g * run_len * K;
  const long long grest = n - gstart;
  const long long gsize = grest < run_len * K ? grest : run_len * K;
  const bool act = lane < K;
  const long long rstart = gstart + (long long)lane * run_len;
  long long rlen = n - rstart;
  rlen = rlen < 0 ? 0 : (rlen > run_len ? run_len : rlen);
  // The pivot rows must describe segments inside their runs whose lengths
  // sum to this tile's size; anything else would overrun the staging buffer.
  // Each segment is checked against S first, so the sum fits 32 bits.
  const long long want = (gsize - j * S) < S ? (gsize - j * S) : S;
  const bool bad_seg = act && (lo < 0 || hi < lo || hi > rlen || hi - lo > S);
  const int len32 = (act && !bad_seg) ? (int)(hi - lo) : 0;
  const int sum = (int)__reduce_add_sync(0xffffffffu, (unsigned)len32);
  const bool bad = __any_sync(0xffffffffu, bad_seg) || sum != want || K > kMaxFanout || K < 2 ||
                   S > G::S || S < kBlockItems || (smem_u32addr(stage) & 15u) != 0;
  if (lane == 0 && (part & 1)) {
    ctl[kCtlNodeFields * 32 + 2] = (int)want;
    ctl[kCtlNodeFields * 32 + 3] = bad ? 1 : 0;
  }
  if (!bad) {
    const long long gsrc = rstart + lo;              // first item, index into `in`
    const int len = act ? (int)(hi - lo) : 0;
    // `in` itself may sit off the 16-byte grid (a segment of a batch): the
    // bulk copies align on absolute addresses.
    const int in_mis = (int)(((uintptr_t)in / sizeof(KeyT)) & (E - 1));
    const int head = act ? (int)((in_mis + gsrc) % E) : 0;   // items copied before the segment
    const int span = (head + len + E - 1) / E * E + G::kSlack;   // staged span + transpose slack
    // One scan over (span, len) packed into 16-bit halves: both totals stay
    // below 2^16 (the spans sum to at most the buffer capacity).
    static_assert(G::cap(kMaxFanout) < (1 << 16), "packed span scan needs cap < 2^16");
    int incl = span | (len << 16);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    const int R = (incl & 0xFFFF) - span;            // span start of segment `lane`
    const int lpre = (incl >> 16) - len;             // items in segments before `lane`
    // Bulk part: from gsrc - head to the first 16-byte boundary (of absolute
    // addresses) at or past the segment's end.  The span rounds up to that
    // boundary, so the few items past the segment land in its own span and
    // are never read.  Where that boundary lies past the end of `in`, the
    // copy stops at the last boundary inside the segment and plain loads
    // fetch the rest (at most one tile per pass).
    const long long bulk_lo = gsrc - head;
    const long long bulk_up = (in_mis + gsrc + len + E - 1) / E * E - in_mis;
    const long long bulk_hi = bulk_up <= n ? bulk_up : (in_mis + gsrc + len) / E * E - in_mis;
    const unsigned bulk_bytes = (act && len > 0 && bulk_hi > bulk_lo)
                                    ? (unsigned)((bulk_hi - bulk_lo) * sizeof(KeyT))
                                    : 0u;
    // Items no bulk copy covers, one segment at a time, consecutive lanes ->
    // consecutive words.
    auto plain_tail = [&]() {
      for (int r = 0; r < K; ++r) {
        const long long s_src = __shfl_sync(0xffffffffu, gsrc, r);
        const int s_len = __shfl_sync(0xffffffffu, len, r);
        const int s_off = __shfl_sync(0xffffffffu, R + head, r);
        const long long s_bhi = __shfl_sync(0xffffffffu, bulk_hi, r);
        const long long s_blo = __shfl_sync(0xffffffffu, bulk_lo, r);
        const long long from = (s_bhi > s_blo) ? s_bhi : s_src;   // first item not bulk-copied
        const long long e = from + lane;
        if (e < s_src + s_len) stage[s_off + (int)(e - s_src)] = in[e];
      }
    };
    if (part & 1) {
      const unsigned total = __reduce_add_sync(0xffffffffu, bulk_bytes);
      if (lane == 0) mbar_arrive_expect_tx(bar, total);
      __syncwarp();
      if (bulk_bytes) bulk_g2s(stage + R, in + bulk_lo, bulk_bytes, bar);
      if (__any_sync(0xffffffffu, act && len > 0 && bulk_hi < gsrc + len)) plain_tail();
    }
    if (!(part & 2)) return;
    // Merge-tree nodes, one per lane, in level order: node (level l >= 1,
    // pair q) merges child A = segments [q*2^l, q*2^l + 2^(l-1)) and child
    // B = the rest of [q*2^l, (q+1)*2^l) (segments past the group's runs are
    // empty).
    // The tree spans the group's runs that exist: the last group of a round
    // (or a round's only group) may hold fewer than K, and empty leaves would
    // add levels that only copy.  At least two leaves, so that the tile is
    // always merged into span start 0.
    const int kruns = __popc(__ballot_sync(0xffffffffu, act && rlen > 0));
    int nl = 0, nnodes = 0, c_level = 0, c_pair = 0;
    {
      int cnt = kruns > 2 ? kruns : 2, idx = 0;
      for (int l = 1; cnt > 1; ++l) {
        const int pairs = (cnt + 1) >> 1;
        if (lane >= idx && lane < idx + pairs) {
          c_level = l;
          c_pair = lane - idx;
        }
        idx += pairs;
        cnt = pairs;
        nl = l;
      }
      nnodes = idx;
    }
    const bool is_node = lane < nnodes;
    const int first = c_pair << c_level;             // first segment of the node
    const int mid = first + (1 << (c_level > 0 ? c_level - 1 : 0));
    const int last = first + (1 << c_level);
    auto seg_pre = [&](int sg) {                     // items in segments [0, sg)
      const int ss = sg < K ? sg : K;
      const int v = __shfl_sync(0xffffffffu, lpre, ss & 31);
      return ss >= K ? (int)want : v;
    };
    const int pf = seg_pre(first), pm = seg_pre(mid), pl = seg_pre(last);
    const int rf = __shfl_sync(0xffffffffu, R, first & 31);
    const int hf = __shfl_sync(0xffffffffu, head, first & 31);
    const int rm = __shfl_sync(0xffffffffu, R, mid & 31);
    const int hm = __shfl_sync(0xffffffffu, head, mid & 31);
    const int lenA = is_node ? pm - pf : 0;
    const int lenB = is_node ? pl - pm : 0;
    const int nb = (lenA + lenB + kBlockItems - 1) / kBlockItems;
    // A node's last block is "small" when it holds at most kSmallBlockMax
    // items; it is merged by the small network, after every full-size block
    // of its level, so that the level's big blocks are dealt first and the
    // cheap ones fill in.  Work items of a level: its nodes' big blocks in
    // node order, then its small blocks in node order; levels follow each
    // other.  Inclusive scans over the nodes (lanes, in level order) of the
    // big and the small block counts give every node its first big item and
    // its small item: with n0 / n1 the first / last node of the node's level,
    //   first big item = big blocks before the node + small blocks before n0,
    //   small item     = big blocks up to n1 + small blocks before the node.
    const int tail = lenA + lenB - (nb - 1) * kBlockItems;
    const int small = (nb > 0 && tail <= kSmallBlockMax) ? 1 : 0;
    const int nbig = nb - small;
    int sbig = nbig, ssm = small;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, sbig, o);
      const int y = __shfl_up_sync(0xffffffffu, ssm, o);
      if (lane >= o) {
        sbig += x;
        ssm += y;
      }
    }
    const unsigned same_level = __match_any_sync(0xffffffffu, is_node ? c_level : -1);
    const int n0 = __ffs(same_level) - 1, n1 = 31 - __clz(same_level);
    const int small_before_n0 = __shfl_sync(0xffffffffu, ssm - small, n0);
    const int big_upto_n1 = __shfl_sync(0xffffffffu, sbig, n1);
    const int small_upto_n1 = __shfl_sync(0xffffffffu, ssm, n1);
    ctl[0 * 32 + lane] = lenA;
    ctl[1 * 32 + lane] = lenB;
    ctl[2 * 32 + lane] = (c_level == 1) ? rf + hf : rf;                     // staged segment
    ctl[3 * 32 + lane] = (mid < K) ? ((c_level == 1) ? rm + hm : rm) : 0;   // vs. child output
    ctl[4 * 32 + lane] = rf;                                                // output span
    ctl[5 * 32 + lane] = (sbig - nbig) + small_before_n0;                  // first big item
    ctl[6 * 32 + lane] = nb;
    ctl[7 * 32 + lane] = is_node ? c_level : 0;
    ctl[8 * 32 + lane] = small ? big_upto_n1 + (ssm - small) : -1;         // small item
    ctl[9 * 32 + lane] = big_upto_n1 + small_upto_n1;                      // end of the level
    if (lane == 0) {
      ctl[kCtlNodeFields * 32 + 0] = nl;
      ctl[kCtlNodeFields * 32 + 1] = nnodes;
    }
  }
}

// Merges a staged tile level by level and writes it to dstg: run by the
// WARPS merging warps (threads 0 .. 32 * WARPS - 1).  bufX holds the staged
// segments, bufY is the other level buffer; `ctl` is the tile's node table.
// sync() is a barrier over exactly the merging warps; the caller has made the
// staged data and the table visible to them.
template <typename KeyT, int WARPS, typename Sync>
__device__ __forceinline__ void merge_levels(KeyT* bufX, KeyT* bufY, const int* ctl,
                                             KeyT* __restrict__ dstg, bool xout, Sync sync) {
  constexpr int E = Vec16<KeyT>::E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = ctl[kCtlNodeFields * 32 + 0];
  const int nnodes = ctl[kCtlNodeFields * 32 + 1];
  const long long want = ctl[kCtlNodeFields * 32 + 2];
  const bool is_node = lane < nnodes;
  const int c_lenA = ctl[0 * 32 + lane], c_lenB = ctl[1 * 32 + lane];
  const int c_offA = ctl[2 * 32 + lane], c_offB = ctl[3 * 32 + lane];
  const int c_out = ctl[4 * 32 + lane], c_first = ctl[5 * 32 + lane];
  const int c_nb = ctl[6 * 32 + lane], c_level = ctl[7 * 32 + lane];
  const int c_small = ctl[8 * 32 + lane], c_end = ctl[9 * 32 + lane];
  const int c_nbig = c_nb - (c_small >= 0 ? 1 : 0);

  // Level by level: the big blocks of the level's nodes, then their small
  // last blocks, are dealt to the warps round-robin; a barrier ends the level.
  for (int lv = 1; lv <= nl; ++lv) {
    const unsigned lvm = __ballot_sync(0xffffffffu, is_node && c_level == lv);
    const int n0 = __ffs(lvm) - 1, n1 = 31 - __clz(lvm);
    const int it0 = __shfl_sync(0xffffffffu, c_first, n0);
    const int it1 = __shfl_sync(0xffffffffu, c_end, n0);
    const int big_end = __shfl_sync(0xffffffffu, c_first + c_nbig, n1);
    const KeyT* src = (lv & 1) ? bufX : bufY;           // level lv reads level lv-1's buffer
    KeyT* dst = (lv & 1) ? bufY : bufX;
    for (int item = it0 + warp; item < it1; item += WARPS) {
      int c, blk;
      if (item < big_end) {                            // a big block: the node whose range holds it
        const unsigned sel = __ballot_sync(0xffffffffu, is_node && c_first <= item && c_nbig > 0);
        c = 31 - __clz(sel);
        blk = item - __shfl_sync(0xffffffffu, c_first, c);
      } else {                                         // a small block: its node's last
        c = __ffs(__ballot_sync(0xffffffffu, is_node && c_small == item)) - 1;
        blk = __shfl_sync(0xffffffffu, c_nb, c) - 1;
      }
      const int lenA = __shfl_sync(0xffffffffu, c_lenA, c);
      const int lenB = __shfl_sync(0xffffffffu, c_lenB, c);
      const int offA = __shfl_sync(0xffffffffu, c_offA, c);
      const int offB = __shfl_sync(0xffffffffu, c_offB, c);
      const int outo = __shfl_sync(0xffffffffu, c_out, c);
      const KeyT* A = src + offA;
      const KeyT* B = src + offB;
      const int L = lenA + lenB;
      const int d0 = blk * kBlockItems;
      const int m = (L - d0) < kBlockItems ? (L - d0) : kBlockItems;
      if (lenA != 0 && lenB != 0) {
        const int a0 = warp_corank(A, lenA, B, lenB, d0, lane);
        const int a1 =
            (d0 + m == L) ? lenA : warp_corank(A, lenA, B, lenB, d0 + m, lane, a0, a0 + m);
        const int X = a1 - a0;
        if (m <= kSmallBlockMax)
          warp_merge_small<KeyT>(A + a0, X, B + (d0 - a0), m - X, dst + outo + d0, lane,
                                 xout && lv == nl);
        else
          warp_merge_block<KeyT, MergeMix>(A + a0, X, B + (d0 - a0), m - X, dst + outo + d0, lane,
                                 xout && lv == nl);
      } else {
        // One child is empty (a node over runs past the group's last, or a
        // tile that takes nothing from one side): the block is a copy, made
        // with 32 consecutive keys per access instead of a merge network.
        const KeyT* from = (lenB == 0 ? A : B) + d0;
        KeyT* to = dst + outo + d0;
        const bool xo = xout && lv == nl;
        for (int i = lane; i < m; i += 32) {
          const KeyT v = from[i];
          to[i] = xo ? (KeyT)ordered_to_f32((uint32_t)v) : v;
        }
      }
      __syncwarp();
    }
    sync();
  }
  // The root node's output is the tile, at span start 0 of the last level's buffer.
  const KeyT* res = (nl & 1) ? bufY : bufX;
  const int m = (int)want;
  const int body = (((uintptr_t)dstg & 15u) == 0) ? m / E * E : 0;   // off-grid: plain stores
  fence_proxy_async_smem();
  sync();
  if (threadIdx.x == 0 && body > 0) bulk_s2g_and_wait(dstg, res, (unsigned)(body * sizeof(KeyT)));
  for (int i = body + (int)threadIdx.x; i < m; i += WARPS * 32) dstg[i] = res[i];
}

// The heap-free variant of the merge (Sec. 7, future work: multiway merging
// driven by the parallel partitioning alone, with no merge tree shared by the
// CTA).  The tile's output is cut into 1024-item blocks, one per warp.
//   1. Warp b finds the pivots of block start 1024 b in every staged segment
//      with the splitter's own search (the multi-sequence selection of
//      Sec. 4.1, multiseq_pivot, here over shared memory), and writes them as
//      row b of `rows`; one CTA barrier publishes the rows.
//   2. The warp's block is then the merge of its K pieces (segment r from
//      row b to row b + 1), which the warp merges alone: pairs of pieces, then
//      pairs of their outputs, along the same binary tree over the runs as the
//      CTA tree, with no barrier between its levels.  The first level reads the
//      staged pieces and writes its outputs packed into the warp's own
//      1024-item region of bufY; later levels merge adjacent outputs back into
//      their own span.  Merges of at most 1024 items at any offset take the
//      register-and-shuffle network of the smallest power of two that holds
//      them (warp_merge_any); the last level, whose output is the whole block
//      at its 16-byte aligned start, takes the transposed 1024-item network.
// bufX holds the staged segments (the node table's level-1 entries give each
// segment's span), bufY receives the tile; the final store is the same as the
// tree's.
// A warp whose pivot rows do not describe pieces inside their segments that
// add up to its block records kDevErrInternal in dev_err and merges nothing,
// so every shared-memory access stays inside the warp's spans.
template <typename KeyT, int WARPS, typename Sync>
__device__ __forceinline__ void merge_partition_blocks(const KeyT* bufX, KeyT* bufY, const int* ctl,
                                                       int* rows, KeyT* __restrict__ dstg, bool xout,
                                                       int* dev_err, Sync sync) {
  constexpr int E = Vec16<KeyT>::E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = ctl[kCtlNodeFields * 32 + 0];       // levels of the tree over the runs (>= 1)
  const int want = ctl[kCtlNodeFields * 32 + 2];     // items of the tile
  const int nnodes = ctl[kCtlNodeFields * 32 + 1];
  const int nleaf = 1 << nl;                         // segments, empty past the group's runs
  // Segment r is child A (r even) or B (r odd) of level-1 node r / 2; the
  // node table lists nodes in level order, so only its level-1 entries give
  // segments (with 5 runs, say, nodes 0..2 are level 1 and segments 6, 7 are
  // empty).
  int seg_off = 0, seg_len = 0;
  {
    const int q = lane >> 1;
    if (lane < nleaf && q < nnodes && ctl[7 * 32 + q] == 1) {
      seg_off = ctl[(2 + (lane & 1)) * 32 + q];
      seg_len = ctl[(lane & 1) * 32 + q];
    }
  }
  const int nblk = (want + kBlockItems - 1) / kBlockItems;
  if (warp == 0) {
    rows[lane] = 0;
    rows[nblk * 32 + lane] = seg_len;
  } else if (warp < nblk) {
    const int k = warp * kBlockItems;
    int d;
    if (nleaf == 2) {
      // Two segments: the search is the merge-path co-rank (ties from the
      // lower run, as in the order of Sec. 4.1).
      const int o0 = __shfl_sync(0xffffffffu, seg_off, 0), l0 = __shfl_sync(0xffffffffu, seg_len, 0);
      const int o1 = __shfl_sync(0xffffffffu, seg_off, 1), l1 = __shfl_sync(0xffffffffu, seg_len, 1);
      const int a = warp_corank(bufX + o0, l0, bufX + o1, l1, k, lane);
      d = lane == 0 ? a : (lane == 1 ? k - a : 0);
    } else {
      d = multiseq_pivot<KeyT, int>(bufX + seg_off, seg_len, lane < nleaf, nleaf, k, 0xffffffffu);
    }
    rows[warp * 32 + lane] = d;
  }
  sync();
  bool rows_ok = true;
  if (warp < nblk) {
    const int r0 = rows[warp * 32 + lane], r1 = rows[(warp + 1) * 32 + lane];
    const int bm = (want - warp * kBlockItems) < kBlockItems ? (want - warp * kBlockItems) : kBlockItems;
    const bool bad = lane < nleaf && (r0 < 0 || r1 < r0 || r1 > seg_len);
    const int sum = (int)__reduce_add_sync(0xffffffffu, (lane < nleaf && !bad) ? (unsigned)(r1 - r0) : 0u);
    rows_ok = !__any_sync(0xffffffffu, bad) && sum == bm;
    if (!rows_ok && lane == 0) set_device_error(dev_err, kDevErrInternal);
  }
  if (warp < nblk && rows_ok) {
    KeyT* blk = bufY + warp * kBlockItems;
    const int r0 = rows[warp * 32 + lane];
    int off = seg_off + r0;                          // lane q: sequence q of the level (bufX
    int len = rows[(warp + 1) * 32 + lane] - r0;     // offsets at level 1, then blk offsets)
    if (lane >= nleaf) len = 0;
    for (int l = 1; l <= nl; ++l) {
      const int npairs = nleaf >> l;
      const int la = __shfl_sync(0xffffffffu, len, (2 * lane) & 31);
      const int lb = __shfl_sync(0xffffffffu, len, (2 * lane + 1) & 31);
      const int oa = __shfl_sync(0xffffffffu, off, (2 * lane) & 31);
      const int ob = __shfl_sync(0xffffffffu, off, (2 * lane + 1) & 31);
      const int olen = lane < npairs ? la + lb : 0;
      int incl = olen;                               // outputs packed in pair order
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
      }
      const int ooff = incl - olen;
      const KeyT* src = (l == 1) ? bufX : blk;
      const bool root = l == nl;
      const bool xo = xout && root;
      for (int p = 0; p < npairs; ++p) {
        const int a = __shfl_sync(0xffffffffu, la, p);
        const int b = __shfl_sync(0xffffffffu, lb, p);
        const int m = a + b;
        if (m == 0) continue;                        // uniform over the warp
        const KeyT* A = src + __shfl_sync(0xffffffffu, oa, p);
        const KeyT* B = src + __shfl_sync(0xffffffffu, ob, p);
        KeyT* out = blk + __shfl_sync(0xffffffffu, ooff, p);
        if (a == 0 || b == 0) {
          // One side empty: a copy at the first level; later levels hold
          // the items in place already (only the float transform remains).
          if (l == 1 || xo) {
            const KeyT* from = a ? A : B;
            for (int i = lane; i < m; i += 32) {
              const KeyT v = from[i];
              out[i] = xo ? (KeyT)ordered_to_f32((uint32_t)v) : v;
            }
          }
        } else if (root && m > kSmallBlockMax) {
          if (l == 1)
            warp_merge_block<KeyT, MergeMix, false>(A, a, B, b, out, lane, xo);
          else
            warp_merge_block<KeyT, MergeMix, true>(A, a, B, b, out, lane, xo);
        } else {
          warp_merge_any<KeyT>(A, a, B, b, out, lane, xo);
        }
        __syncwarp();
      }
      off = ooff;
      len = olen;
    }
  }
  const int body = (((uintptr_t)dstg & 15u) == 0) ? want / E * E : 0;   // off-grid: plain stores
  fence_proxy_async_smem();
  sync();
  if (threadIdx.x == 0 && body > 0) bulk_s2g_and_wait(dstg, bufY, (unsigned)(body * sizeof(KeyT)));
  for (int i = body + (int)threadIdx.x; i < want; i += WARPS * 32) dstg[i] = bufY[i];
}

// Merges output tile j (of S items, a multiple of 1024 and at most
// 1024 * WARPS) of group g of `in` (n items in sorted runs of run_len, K runs
// per group) into `out`: the CTA body of a merge round, one tile at a time.
// lo_row and hi_row are the pivot rows of the tile's start and end (read only
// when the tile is not its group's first / last).  `bar` is an initialised
// mbarrier of this CTA whose next phase completes with parity `phase`.
// `xout` undoes the float transform on the tile's last level.  Returns false,
// with the error recorded, when the CTA must stop (a pivot row fails its
// check or the staging wait ran out); the decision is uniform over the CTA.
// test_timeout (a test hook; bar[1] then holds an initialised mbarrier): once
// the staged data has arrived, thread 0 also waits on bar[1] for 16 bytes no
// copy delivers, with a limit of about a millisecond, so the CTA takes the
// time-out path with no copy in flight.
// PARTITION: merge with the heap-free variant above instead of the CTA tree
// (shared memory of MergeGeom::bytes_partition).
template <typename KeyT, int WARPS, bool PARTITION = false>
__device__ __forceinline__ bool merge_tile(const KeyT* __restrict__ in, KeyT* __restrict__ out,
                                           long long n, long long run_len, int K, long long g,
                                           long long j, const long long* __restrict__ lo_row,
                                           const long long* __restrict__ hi_row, bool xout,
                                           int* dev_err, unsigned char* smem_raw, uint64_t* bar,
                                           unsigned phase, int S, bool test_timeout = false) {
  using G = MergeGeom<KeyT, WARPS>;
  const int cap = G::cap(K);
  KeyT* bufX = reinterpret_cast<KeyT*>(smem_raw);
  KeyT* bufY = bufX + cap;
  int* ctl = reinterpret_cast<int*>(bar + 2);          // node table and scalars (see above)
  // Every thread is past the previous tile (whose store has read its shared
  // memory) before the staging copies overwrite the buffer.
  // Warp 0 stages the segments while warp 1 builds the node table.
  long long lo = 0, hi = 0;
  if ((threadIdx.x >> 5) < 2)
    merge_tile_pivots(n, run_len, K, g, j, lo_row, hi_row, S, threadIdx.x & 31, lo, hi);
  __syncthreads();
  if ((threadIdx.x >> 5) < 2)
    merge_plan_warp<KeyT, WARPS>(in, n, run_len, K, g, j, lo, hi, S, bufX, ctl, bar,
                                 threadIdx.x & 31, (threadIdx.x >> 5) == 0 ? 1 : 2);
  __syncthreads();
  if (ctl[kCtlNodeFields * 32 + 3] || (smem_u32addr(smem_raw) & 1023u) != 0) {
    if (threadIdx.x == 0) set_device_error(dev_err, kDevErrInternal);
    return false;                                      // uniform over the CTA
  }
  // One thread polls the staging barrier; the others wait at the CTA barrier
  // (no issue slots spent polling), which also orders the staged data and the
  // plainly loaded items before every warp's reads.
  bool ok = (threadIdx.x == 0) ? mbar_wait_bounded(bar, phase) : true;
  if (test_timeout && threadIdx.x == 0 && ok) {
    mbar_arrive_expect_tx(bar + 1, 16u);
    ok = mbar_wait_bounded(bar + 1, 0u, 2000000ll);
  }
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) set_device_error(dev_err, kDevErrTimeout);
    return false;
  }
  if constexpr (PARTITION)
    merge_partition_blocks<KeyT, WARPS>(bufX, bufY, ctl, ctl + kCtlNodeFields * 32 + kCtlScalars,
                                        out + g * run_len * K + j * S, xout, dev_err,
                                        []() { __syncthreads(); });
  else
    merge_levels<KeyT, WARPS>(bufX, bufY, ctl, out + g * run_len * K + j * S, xout,
                              []() { __syncthreads(); });
  return true;
}

}  // namespace mms
