"""CPU model of the cluster base case's index arithmetic (tile_sort_cluster.cu).

The cluster of CL CTAs sorts one run of CL * 8192 keys (Sec. 4.3 with the
cluster's shared memory as the internal memory): each CTA sorts its 8192-key
chunk, then at level l every CTA of a group of 2^l produces its 8192-key slice
of the merge of the group's two halves.  This model replays, per level and per
CTA, the kernel's run lengths, slice bounds, co-ranks, 16-byte word copies
from the peers' chunk buffers and offsets of the staged pieces, and checks:
- every word read lies in a chunk of the piece's own run and inside the chunk
  buffer (8192 keys + 32 of slack), and the copies fit the loop's bound;
- the staged pieces hold exactly A[a0, a1) and B[b0, b0 + Y), whatever lies
  past the valid keys of a chunk (planted garbage);
- the slice plus the block merge's transpose space fits the chunk buffer;
- the chunks after the last level are the sorted run.
Brute force: the co-ranks come from a stable merge by lexsort, the expected
runs from numpy's sort.
"""
import numpy as np
import pytest

KCT = 8192          # keys per CTA tile
SLACK = 32          # kTileSlack: items of slack past a tile buffer
STAGE_ITERS = ((KCT + 16) // 4 + 255) // 256
GARBAGE = np.uint32(0xA5A5A5A5)


def corank(A, B, d):
    """Items of A among the first d items of the stable merge of A and B (ties from A)."""
    if d == 0:
        return 0
    vals = np.concatenate([A, B])
    side = np.concatenate([np.zeros(len(A), np.int64), np.ones(len(B), np.int64)])
    order = np.lexsort((side, vals))
    return int(np.count_nonzero(side[order[:d]] == 0))


def run_items(n, sbase, c0, half):
    r = n - (sbase + c0 * KCT)
    return 0 if r <= 0 else min(r, half * KCT)


def runs_sorted(keys, R):
    """Every run of R consecutive keys sorted on its own (the base case's output)."""
    return np.concatenate([np.sort(keys[i:i + R]) for i in range(0, len(keys), R)])


def model_cluster_sort(keys, CL):
    n = len(keys)
    out = np.empty_like(keys)
    for sbase in range(0, n, CL * KCT):
        clen = [max(0, min(KCT, n - (sbase + c * KCT))) for c in range(CL)]
        bufs = []
        for c in range(CL):
            b = np.full(KCT + SLACK, GARBAGE, np.uint32)
            lo = sbase + c * KCT
            b[:clen[c]] = np.sort(keys[lo:lo + clen[c]])
            bufs.append(b)
        lv = 1
        while (1 << lv) <= CL:
            g, half = 1 << lv, 1 << (lv - 1)
            new = []
            for rank in range(CL):
                nb = rank & ~(g - 1)
                LA, LB = run_items(n, sbase, nb, half), run_items(n, sbase, nb + half, half)
                A = np.concatenate([bufs[nb + j][:clen[nb + j]] for j in range(half)])
                B = np.concatenate([bufs[nb + half + j][:clen[nb + half + j]] for j in range(half)])
                assert len(A) == LA and len(B) == LB
                my_len = clen[rank]
                d0 = (rank - nb) * KCT
                d1 = d0 + my_len
                assert my_len == 0 or d1 <= LA + LB           # chunks before a non-empty one are full
                a0 = corank(A, B, d0) if my_len else 0
                a1 = corank(A, B, d1) if my_len else 0
                X, Y, b0 = a1 - a0, my_len - (a1 - a0), d0 - a0
                assert my_len == 0 or (0 <= X <= LA and 0 <= b0 and b0 + Y <= LB)
                wa0 = a0 >> 2
                na = ((a1 + 3) >> 2) - wa0 if X > 0 else 0
                wb0 = b0 >> 2
                nbw = ((b0 + Y + 3) >> 2) - wb0 if Y > 0 else 0
                assert na + nbw <= STAGE_ITERS * 256
                assert 4 * (na + nbw) <= KCT + SLACK
                fre = np.full(KCT + SLACK, GARBAGE, np.uint32)
                for q in range(na + nbw):
                    w, c0 = (wa0 + q, nb) if q < na else (wb0 + q - na, nb + half)
                    chunk = c0 + (w >> 11)
                    off = w & 2047
                    assert c0 <= chunk < c0 + half          # the word lies in the piece's own run
                    assert 4 * off + 4 <= KCT + SLACK       # and inside the chunk buffer
                    fre[4 * q:4 * q + 4] = bufs[chunk][4 * off:4 * off + 4]
                offA, offB = a0 & 3, 4 * na + (b0 & 3)
                assert np.array_equal(fre[offA:offA + X], A[a0:a1])
                assert np.array_equal(fre[offB:offB + Y], B[b0:b0 + Y])
                assert offA + X <= offB or Y == 0 or X == 0
                merged = np.sort(np.concatenate([fre[offA:offA + X], fre[offB:offB + Y]]))
                assert my_len + 31 <= KCT + SLACK          # block merges' transpose space
                nbuf = np.full(KCT + SLACK, GARBAGE, np.uint32)
                nbuf[:my_len] = merged
                new.append(nbuf)
            bufs = new
            lv += 1
        for c in range(CL):
            out[sbase + c * KCT:sbase + c * KCT + clen[c]] = bufs[c][:clen[c]]
    return out


@pytest.mark.parametrize("CL", [2, 4, 8])
@pytest.mark.parametrize("extra", [1, 4097, 3, 8191])
def test_cluster_levels_sort_any_tail(CL, extra):
    rng = np.random.default_rng(CL * 100 + extra)
    n = CL * KCT + (CL // 2) * KCT + extra            # one full cluster and a ragged one
    keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(model_cluster_sort(keys, CL), runs_sorted(keys, CL * KCT))


@pytest.mark.parametrize("kind", ["dups", "equal", "sorted", "reversed", "disjoint"])
def test_cluster_levels_structured_inputs(kind):
    CL = 4
    n = 2 * CL * KCT - 5
    rng = np.random.default_rng(7)
    if kind == "dups":
        keys = (rng.integers(0, 5, n)).astype(np.uint32)
    elif kind == "equal":
        keys = np.full(n, 42, np.uint32)
    elif kind == "sorted":
        keys = np.arange(n, dtype=np.uint32)
    elif kind == "reversed":
        keys = np.arange(n, dtype=np.uint32)[::-1].copy()
    else:                                              # each chunk above the previous one
        keys = np.concatenate([np.arange(KCT, dtype=np.uint32) + np.uint32(c * KCT)
                               for c in range(n // KCT + 1)])[:n][::-1].copy()
    assert np.array_equal(model_cluster_sort(keys, CL), runs_sorted(keys, CL * KCT))


def test_cluster_sizes_below_one_cluster():
    for n in [8193, 8192 + 4, 16384, 20000, 32767, 32768]:
        keys = np.random.default_rng(n).integers(0, 1000, n).astype(np.uint32)
        assert np.array_equal(model_cluster_sort(keys, 4), np.sort(keys))


def test_model_catches_a_short_word_range():
    """Planted mistake: rounding a piece's last word down instead of up loses keys."""
    A = np.arange(0, 20, 2, dtype=np.uint32)
    a0, a1 = 1, 7
    wa0 = a0 >> 2
    na_bad = (a1 >> 2) - wa0
    fre = np.full(64, GARBAGE, np.uint32)
    for q in range(na_bad):
        fre[4 * q:4 * q + 4] = A[4 * (wa0 + q):4 * (wa0 + q) + 4]
    assert not np.array_equal(fre[a0 & 3:(a0 & 3) + a1 - a0], A[a0:a1])
