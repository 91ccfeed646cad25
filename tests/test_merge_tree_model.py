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
