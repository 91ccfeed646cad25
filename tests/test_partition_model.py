"""Host model of the heap-free partition merge's index arithmetic
(merge_partition_blocks in csrc/merge_tile.cuh; Sec. 7, future work).

The model replays, for random tiles, what every warp of the kernel does with
its indices: segment spans from the level-1 node table, the pivot rows of the
1024-item block starts (brute force here: the k smallest items in the order
(key, run, position) of Sec. 4.1), the pieces, and the warp's tree levels with
outputs packed into its block region and merged back into their own span.  It
checks every access against the rules the kernel relies on -- level-1 outputs
inside the warp's region, later merges reading two adjacent sequences and
writing exactly their span, the root's transpose space inside the region --
and that the block equals the sorted items of its ranks.  No GPU needed.
"""
import random

import numpy as np
import pytest

BLOCK = 1024
SMALL = 256


def order_key(item):
    key, run, pos = item
    return (key, run, pos)


def tree_levels(kruns):
    cnt, nl = max(kruns, 2), 0
    while cnt > 1:
        cnt = (cnt + 1) // 2
        nl += 1
    return nl


def node_table(lens):
    """The plan's merge-tree nodes in level order (lane = node), as the
    kernel's plan writes them: (level, lenA, lenB, first segment of A, of B)
    for the tree over the group's K' runs (at least two leaves)."""
    K = len(lens)
    pre = [0]
    for x in lens:
        pre.append(pre[-1] + x)
    seg_pre = lambda sg: pre[min(sg, K)]
    nodes, cnt, l = [], max(K, 2), 1
    while cnt > 1:
        pairs = (cnt + 1) // 2
        for q in range(pairs):
            first, mid, last = q << l, (q << l) + (1 << (l - 1)), (q + 1) << l
            nodes.append((l, seg_pre(mid) - seg_pre(first), seg_pre(last) - seg_pre(mid), first,
                          mid if mid < K else None))
        cnt, l = pairs, l + 1
    return nodes, l - 1


def segments_from_table(nodes, nl):
    """What merge_partition_blocks reads: segment r is child A (r even) or B
    (r odd) of level-1 node r / 2, taken only from level-1 entries."""
    nleaf = 1 << nl
    out = []
    for r in range(nleaf):
        q = r >> 1
        if q < len(nodes) and nodes[q][0] == 1:
            lvl, la, lb, fa, fb = nodes[q]
            out.append((fa if r % 2 == 0 else fb, la if r % 2 == 0 else lb))
        else:
            out.append((None, 0))
    return out


def replay_tile(segs, S):
    """segs: the tile's staged segments, one sorted key list per run of the group."""
    K = len(segs)
    nodes, nl = node_table([len(x) for x in segs])
    nleaf = 1 << nl
    assert nleaf <= 32
    seg = []
    for r, (src, ln) in enumerate(segments_from_table(nodes, nl)):
        if ln:
            assert src == r, "segment r comes from run r"
        seg.append(segs[r][:ln] if ln else [])
        if r < K:
            assert ln == len(segs[r]), "every run's segment is found"
    items = sorted(((k, r, p) for r in range(nleaf) for p, k in enumerate(seg[r])), key=order_key)
    want = len(items)
    assert want <= S
    nblk = (want + BLOCK - 1) // BLOCK
    # rows[b][r]: items of run r among the first 1024 b outputs (brute force)
    rows = []
    for b in range(nblk + 1):
        k = min(b * BLOCK, want)
        row = [0] * nleaf
        for (_, r, _) in items[:k]:
            row[r] += 1
        rows.append(row)
    out_tile = []
    for w in range(nblk):
        region = [None] * BLOCK
        # lane q: (is_in_X, offset, len); level-1 offsets are into the segment q
        seqs = [("X", q, rows[w][q], rows[w + 1][q] - rows[w][q]) for q in range(nleaf)]
        for l in range(1, nl + 1):
            npairs = nleaf >> l
            new = []
            ooff = 0
            for p in range(npairs):
                A, B = seqs[2 * p], seqs[2 * p + 1]
                a, b = A[3], B[3]
                m = a + b
                root = l == nl
                if l == 1:
                    av = seg[A[1]][A[2]:A[2] + a]
                    bv = seg[B[1]][B[2]:B[2] + b]
                else:
                    assert A[0] == "Y" and B[0] == "Y"
                    assert B[2] == A[2] + a, "later levels merge adjacent sequences"
                    assert A[2] == ooff, "and write them back into their own span"
                    av, bv = region[A[2]:A[2] + a], region[B[2]:B[2] + b]
                    assert None not in av and None not in bv
                assert 0 <= ooff and ooff + m <= BLOCK, "outputs stay in the warp's region"
                if m > 0:
                    if root and m > SMALL and a and b:
                        assert ooff == 0 and 32 * ((m + 31) // 32) <= BLOCK, "transpose space"
                    merged = sorted(av + bv)
                    region[ooff:ooff + m] = merged
                new.append(("Y", None, ooff, m))
                ooff += m
            seqs = new + [("Y", None, ooff, 0)] * (len(seqs) - npairs)
        blk = region[:seqs[0][3]]
        lo, hi = w * BLOCK, min((w + 1) * BLOCK, want)
        assert blk == [k for (k, _, _) in items[lo:hi]], "block = sorted items of its ranks"
        out_tile += blk
    assert out_tile == sorted(k for s in seg for k in s)


def random_tile(rng, K, S, dups):
    total = rng.randint(1, S)
    cuts = sorted(rng.randint(0, total) for _ in range(K - 1))
    lens = [b - a for a, b in zip([0] + cuts, cuts + [total])]
    hi = 6 if dups else 1 << 30
    return [sorted(rng.randint(0, hi) for _ in range(n)) for n in lens]


@pytest.mark.parametrize("K", [2, 3, 4, 5, 6, 7, 8, 11, 13, 16, 21, 32])
@pytest.mark.parametrize("dups", [False, True])
def test_partition_index_model_random_tiles(K, dups):
    rng = random.Random(1000 * K + dups)
    for _ in range(6):
        replay_tile(random_tile(rng, K, 8192, dups), 8192)


def test_partition_index_model_edge_tiles():
    rng = random.Random(5)
    S = 8192
    replay_tile([list(range(S))] + [[] for _ in range(7)], S)            # one full segment
    replay_tile([[] for _ in range(7)] + [list(range(S))], S)            # the last one only
    replay_tile([[i] * 1 for i in range(3)] + [[]] * 5, S)               # a tiny tile
    replay_tile([sorted(rng.randint(0, 9) for _ in range(1024)) for _ in range(8)], S)  # exact blocks
    replay_tile([[7] * 1000, [7] * 24, [7] * 1, [7] * 2048], S)          # all equal keys
    replay_tile([list(range(r, 32 * 256, 32)) for r in range(32)], S)    # K = 32 interleaved
