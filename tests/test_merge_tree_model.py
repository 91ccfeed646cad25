"""Host model of a merge CTA's tree (merge_tile.cuh: the node table of
merge_plan_warp and the level loop of merge_levels).

For a tile of K segments staged in buffer X (segment r at span start R_r plus
its alignment head), the plan builds a binary tree over the K' <= K runs the
group holds (at least two leaves): level l has ceil(count / 2) nodes, node q
merges child A = segments [q * 2^l, q * 2^l + 2^(l-1)) and child B = the rest
of [q * 2^l, (q + 1) * 2^l).  Level l reads the buffer level l - 1 wrote (X
for the leaves) and writes its outputs, each at the span start of its first
segment, into the other buffer.  The model replays the table and the levels
with real merges and checks, for every K and run count:
  * ceil(log2 max(K', 2)) levels; the root's output, at span start 0 of the
    last level's buffer, is the sorted tile;
  * within a level, no node writes (output plus up to 31 items of transpose
    slack) outside its own segments' spans, so nodes never overwrite each
    other or an input the level still reads.
"""
import math

import numpy as np
import pytest

SLACK = 32
E = 4


def node_table(K, kruns):
    cnt, idx, nodes, nl = max(kruns, 2), 0, [], 0
    level = 1
    while cnt > 1:
        pairs = (cnt + 1) >> 1
        for q in range(pairs):
            nodes.append((level, q))
        idx += pairs
        cnt = pairs
        nl = level
        level += 1
    return nl, nodes


def run_tree(segs, K, kruns):
    lens = [len(s) for s in segs] + [0] * (K - len(segs))
    heads = [(3 * r) % E for r in range(K)]                 # some alignment heads
    spans = [(h + n + E - 1) // E * E + SLACK for h, n in zip(heads, lens)]
    R = np.concatenate([[0], np.cumsum(spans)]).astype(int)
    size = int(R[-1])
    X = np.full(size, -1, dtype=np.int64)
    Y = np.full(size, -1, dtype=np.int64)
    for r in range(len(segs)):
        X[R[r] + heads[r]: R[r] + heads[r] + lens[r]] = segs[r]
    pre = np.concatenate([[0], np.cumsum(lens)]).astype(int)
    want = int(pre[-1])
    seg_pre = lambda sg: want if sg >= K else int(pre[sg])
    nl, nodes = node_table(K, kruns)
    for lv in range(1, nl + 1):
        src, dst = (X, Y) if lv & 1 else (Y, X)
        written = []
        for level, q in nodes:
            if level != lv:
                continue
            first = q << level
            mid = first + (1 << (level - 1))
            last = first + (1 << level)
            lenA = seg_pre(mid) - seg_pre(first)
            lenB = seg_pre(last) - seg_pre(mid)
            offA = R[first] + heads[first] if level == 1 else R[first]
            offB = ((R[mid] + heads[mid]) if level == 1 else R[mid]) if mid < K else 0
            A = src[offA: offA + lenA]
            B = src[offB: offB + lenB]
            merged = np.sort(np.concatenate([A, B]), kind="stable")
            out = R[first]
            end_of_spans = R[min(last, K)]
            L = lenA + lenB
            nr = -(-L // 32) * 32                           # transpose rows of the last, partial block
            assert out + max(L, nr) <= end_of_spans         # stays inside its own segments' spans
            written.append((out, out + max(L, nr)))
            dst[out: out + L] = merged
        written.sort()
        for (a0, a1), (b0, b1) in zip(written, written[1:]):
            assert a1 <= b0                                 # nodes of a level never overlap
    res = Y if nl & 1 else X
    return nl, res[:want]


@pytest.mark.parametrize("K", [2, 3, 4, 5, 7, 8, 16, 32])
def test_tree_over_the_runs_a_group_holds(K):
    rng = np.random.default_rng(K)
    for kruns in range(1, K + 1):
        for trial in range(5):
            lens = rng.integers(0, 300, kruns)
            segs = [np.sort(rng.integers(0, 1000, n)) for n in lens]
            nl, res = run_tree(segs, K, kruns)
            assert nl == math.ceil(math.log2(max(kruns, 2)))
            assert np.array_equal(res, np.sort(np.concatenate(segs)))


BLOCK = 1024
SMALL_MAX = 256


def block_items(levels, sizes):
    """The plan's numbering of a tile's work items (merge_plan_warp): per node
    (lanes in level order) its first big item, its small item (or -1) and its
    level's end, from inclusive scans of the big and small block counts."""
    n = len(sizes)
    nb = [-(-L // BLOCK) for L in sizes]
    small = [1 if (b > 0 and L - (b - 1) * BLOCK <= SMALL_MAX) else 0 for L, b in zip(sizes, nb)]
    nbig = [b - s for b, s in zip(nb, small)]
    sbig = np.cumsum(nbig)
    ssm = np.cumsum(small)
    first, sitem, end = [], [], []
    for q in range(n):
        same = [i for i in range(n) if levels[i] == levels[q]]
        n0, n1 = same[0], same[-1]
        first.append(int(sbig[q] - nbig[q] + ssm[n0] - small[n0]))
        sitem.append(int(sbig[n1] + ssm[q] - small[q]) if small[q] else -1)
        end.append(int(sbig[n1] + ssm[n1]))
    return nb, nbig, small, first, sitem, end


def test_level_items_deal_big_blocks_first_then_small_ones():
    """merge_levels' item -> (node, block) lookup over the plan's numbering:
    every block of every node of a level is one item of that level's range,
    exactly once; the level's full-size blocks come first, its small last
    blocks (at most 256 items) after them; the levels' ranges follow each
    other from 0."""
    rng = np.random.default_rng(11)
    for trial in range(400):
        K = int(rng.choice([2, 3, 4, 5, 8, 16, 32]))
        nl, nodes = node_table(K, int(rng.integers(1, K + 1)))
        levels = [lv for lv, _ in nodes]
        kind = trial % 4
        if kind == 0:        # sizes near multiples of 1024, as on random keys
            sizes = [int(max(0, BLOCK * rng.integers(0, 9) + rng.integers(-60, 60))) for _ in nodes]
        elif kind == 1:      # exact multiples (sorted or interleaved inputs)
            sizes = [int(BLOCK * rng.integers(0, 9)) for _ in nodes]
        else:
            sizes = [int(rng.integers(0, 8193)) for _ in nodes]
        nb, nbig, small, first, sitem, end = block_items(levels, sizes)
        start = 0
        for lv in range(1, nl + 1):
            lvn = [q for q in range(len(nodes)) if levels[q] == lv]
            n0, n1 = lvn[0], lvn[-1]
            it0, it1 = first[n0], end[n0]
            big_end = first[n1] + nbig[n1]
            assert it0 == start
            got = []
            for item in range(it0, it1):
                if item < big_end:
                    c = max(q for q in range(len(nodes)) if first[q] <= item and nbig[q] > 0)
                    blk = item - first[c]
                    assert not (small[c] and blk == nb[c] - 1)
                else:
                    cs = [q for q in range(len(nodes)) if sitem[q] == item]
                    assert len(cs) == 1
                    c = cs[0]
                    blk = nb[c] - 1
                    assert sizes[c] - blk * BLOCK <= SMALL_MAX
                assert levels[c] == lv
                got.append((c, blk))
            want = [(q, b) for q in lvn for b in range(nb[q])]
            assert sorted(got) == sorted(want) and len(set(got)) == len(got)
            start = it1
