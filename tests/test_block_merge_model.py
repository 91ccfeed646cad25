"""Host model of the warp block merge of the merge pass (mms_common.cuh:
warp_load_bitonic, warp_bitonic_1024 and warp_store_block) for 32-bit keys.

It replays the kernel's index maps -- the striped window load of A ascending
and B descending, the register cascade, the chunk-swizzled transpose, the
in-lane cascade whose strides of 16 bytes and more run in the direction of the
lane's flip-mask bit, and the 16-byte chunk stores XOR-permuted by the lane --
and checks that the block comes out as merge(A, B) for full and partial blocks
(pads past m are not stored), and that every warp-wide shared-memory access
touches 32 distinct banks, or 8 distinct 16-byte bank groups per quarter-warp.
The GPU parity tests check the kernel's bits; this pins the design.
"""
import numpy as np
import pytest

E = 4
LANES = 32
PAD = np.uint32(0xFFFFFFFF)


def flip_mask(lane):
    return (lane & (32 // E - 1)) * E


def window_load(A, B, banks):
    """Register k of lane l = C[32k + l], C = A ++ pads ++ reversed(B)."""
    X, Y = len(A), len(B)
    v = np.full((32, LANES), PAD, dtype=np.uint32)
    for k in range(32):
        a_words, b_words = [], []
        for lane in range(LANES):
            i = 32 * k + lane
            if i < X:
                v[k, lane] = A[i]
                a_words.append(i % 32)                    # A + i: consecutive words
            elif i >= 1024 - Y:
                j = 1023 - i
                v[k, lane] = B[j]
                b_words.append((1023 - i) % 32)           # B + 1023 - i: consecutive, descending
        for words in (a_words, b_words):                  # two predicated loads per register
            if words:
                banks.append(("window_load", words))
    return v


def cascade(x, dmax, dirs=None):
    """Half-cleaners of distance dmax .. 1 along axis 0; dirs(s) -> per-column
    bool array: True puts the larger key first."""
    x = x.copy()
    s = dmax
    while s >= 1:
        f = np.zeros(x.shape[1], dtype=bool) if dirs is None else dirs(s)
        for k in range(x.shape[0]):
            if k & s == 0:
                lo = np.minimum(x[k], x[k + s])
                hi = np.maximum(x[k], x[k + s])
                x[k] = np.where(f, hi, lo)
                x[k + s] = np.where(f, lo, hi)
        s //= 2
    return x


def block_merge_model(A, B, banks, flips=True):
    m = len(A) + len(B)
    nr = (m + 31) // 32
    v = window_load(A, B, banks)
    v = cascade(v, 16)                                    # strides 512 .. 32 (registers)
    buf = np.full(1024, 0, dtype=np.uint32)
    for k in range(nr):                                   # striped -> blocked, rows swizzled by k & 7
        words = []
        for lane in range(LANES):
            a = 32 * k + (lane ^ (E * (k & 7)))
            buf[a] = v[k, lane]
            words.append(a % 32)
        banks.append(("row_store", words))
    rows = np.full((LANES, 32), PAD, dtype=np.uint32)
    for ch in range(32 // E):
        groups = []
        for lane in range(nr):
            pos = ch ^ (lane & 7)
            rows[lane, E * ch: E * ch + E] = buf[32 * lane + E * pos: 32 * lane + E * pos + E]
            groups.append((lane // 8, pos))
        banks.append(("chunk_load", groups))
    F = np.array([flip_mask(l) if flips else 0 for l in range(LANES)])
    regs = cascade(rows.T, 16, lambda s: (F & s) != 0 if s >= E else np.zeros(LANES, bool))
    # register j of lane l now holds item 32l + (j ^ F[l]); chunk stores below m
    out = np.full(1024, 0xDEAD, dtype=np.uint32)
    for c in range(32 // E):
        groups = []
        for lane in range(LANES):
            pos = (c * E) ^ F[lane]
            if pos + E <= m - 32 * lane:
                out[32 * lane + pos: 32 * lane + pos + E] = regs[c * E: c * E + E, lane]
                groups.append((lane // 8, (pos // E)))
        banks.append(("chunk_store", groups))
    for lane in range(LANES):                             # the chunk straddling m, item by item
        room = m - 32 * lane
        for c in range(32 // E):
            pos = (c * E) ^ F[lane]
            if pos < room < pos + E:
                for w in range(E):
                    if pos + w < room:
                        out[32 * lane + pos + w] = regs[c * E + w, lane]
    return out[:m], out[m:]


@pytest.mark.parametrize("X,Y", [(512, 512), (1024, 0), (0, 1024), (300, 724), (700, 1), (5, 3),
                                 (0, 37), (400, 0), (17, 13)])
@pytest.mark.parametrize("kind", ["uniform", "dups"])
def test_block_merge_model_merges(X, Y, kind):
    rng = np.random.default_rng(X * 1000 + Y)
    hi = 2**32 if kind == "uniform" else 4
    A = np.sort(rng.integers(0, hi, X, dtype=np.uint64).astype(np.uint32))
    B = np.sort(rng.integers(0, hi, Y, dtype=np.uint64).astype(np.uint32))
    banks = []
    got, rest = block_merge_model(A, B, banks)
    assert np.array_equal(got, np.sort(np.concatenate([A, B])))
    assert np.all(rest == 0xDEAD)                         # nothing stored past m
    for kind_, access in banks:
        if kind_ in ("chunk_store", "chunk_load"):
            for q in range(4):
                groups = [g for quarter, g in access if quarter == q]
                assert len(set(groups)) == len(groups), (kind_, q, groups)
        else:
            assert len(set(access)) == len(access), (kind_, access)


def test_without_lane_flips_the_chunk_stores_conflict():
    """The flipped in-lane directions exist for the store: with every lane
    ascending the block still merges, but a quarter-warp's 16-byte stores all
    land in one bank group."""
    rng = np.random.default_rng(5)
    A = np.sort(rng.integers(0, 2**32, 600, dtype=np.uint64).astype(np.uint32))
    B = np.sort(rng.integers(0, 2**32, 424, dtype=np.uint64).astype(np.uint32))
    banks = []
    got, _ = block_merge_model(A, B, banks, flips=False)
    assert np.array_equal(got, np.sort(np.concatenate([A, B])))
    stores = [access for kind, access in banks if kind == "chunk_store"]
    assert any(len(set(g for quarter, g in access if quarter == 0)) < 8 for access in stores)
