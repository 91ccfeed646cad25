"""Host model of the tile sort's warp sort (tile_sort.cuh: warp_sort_1024 and
blocked_to_striped_rev, with the striped/blocked pieces of mms_common.cuh).

It replays, with numpy, the index maps the kernel uses -- the chunk-swizzled
row stores, the row loads that read the upper half of every block backwards,
the transposes, and the half-cleaner cascades -- and checks two things:
  * every merge level turns blocks whose halves are sorted into sorted blocks
    (the reversed read makes each block bitonic, so ascending cascades sort
    it), so the whole warp sort sorts any 1024 keys, duplicates included;
  * every shared-memory instruction of the transposes touches 32 distinct
    banks (32-bit keys) and every 16-byte chunk store of a quarter-warp hits
    8 distinct 16-byte bank groups: no bank conflicts by construction.
The kernel's last level runs its in-lane stages with per-lane directions that
leave each row XOR-permuted for the store; the model keeps rows ascending (the
same keys per row).  No GPU is involved; the GPU parity tests check the
kernel's bits.
"""
import numpy as np
import pytest

E = 4          # 32-bit keys per 16-byte chunk
LANES = 32


def swz_word(row, w):
    """Word of item (row, column w) in the transposed buffer: the row's 16-byte
    chunks are XOR-swizzled by row & 7."""
    return 32 * row + (w ^ (E * (row & 7)))


def blocked_to_striped_rev(blocked, R, banks=None):
    """blocked[l] = row l (32 keys).  Returns striped[k][l] as the kernel's
    register k of lane l, upper half of every block of R rows read backwards."""
    buf = np.empty(1024, dtype=blocked.dtype)
    # each lane stores its row as chunks ch at position ch ^ (lane & 7)
    for ch in range(32 // E):
        groups = []
        for lane in range(LANES):
            pos = ch ^ (lane & 7)
            buf[32 * lane + E * pos: 32 * lane + E * pos + E] = blocked[lane, E * ch: E * ch + E]
            groups.append((lane // 8, (32 * lane + E * pos) % 32 // E))
        if banks is not None:
            banks.append(("chunk_store", groups))
    striped = np.empty((32, LANES), dtype=blocked.dtype)
    for k in range(32):
        kq = k % R
        rev = kq >= R // 2
        src = k - kq + R - 1 - (kq - R // 2) if rev else k
        words = []
        for lane in range(LANES):
            w = 31 - lane if rev else lane
            a = swz_word(src, w)
            striped[k, lane] = buf[a]
            words.append(a % 32)
        if banks is not None:
            banks.append(("row_load", words))
    return striped


def striped_to_blocked(striped, banks=None):
    buf = np.empty(1024, dtype=striped.dtype)
    for k in range(32):
        words = []
        for lane in range(LANES):
            a = swz_word(k, lane)
            buf[a] = striped[k, lane]
            words.append(a % 32)
        if banks is not None:
            banks.append(("row_store", words))
    blocked = np.empty((LANES, 32), dtype=striped.dtype)
    for ch in range(32 // E):
        groups = []
        for lane in range(LANES):
            pos = ch ^ (lane & 7)
            blocked[lane, E * ch: E * ch + E] = buf[32 * lane + E * pos: 32 * lane + E * pos + E]
            groups.append((lane // 8, pos))
        if banks is not None:
            banks.append(("chunk_load", groups))
    return blocked


def half_cleaners(x, dmax):
    """Ascending half-cleaners of distance dmax .. 1 along axis 0 (registers of
    the striped layout, or the items of a row)."""
    x = x.copy()
    s = dmax
    while s >= 1:
        for k in range(x.shape[0]):
            if k & s == 0:
                lo = np.minimum(x[k], x[k + s])
                hi = np.maximum(x[k], x[k + s])
                x[k], x[k + s] = lo, hi
        s //= 2
    return x


def warp_sort_model(keys, banks=None):
    blocked = np.sort(keys.reshape(LANES, 32), axis=1)          # lane_sort32: each row ascending
    for R in (2, 4, 8, 16, 32):
        striped = blocked_to_striped_rev(blocked, R, banks)
        striped = half_cleaners(striped, R // 2)                 # strides 16R .. 32
        blocked = striped_to_blocked(striped, banks)
        blocked = half_cleaners(blocked.T, 16).T                 # strides 16 .. 1 inside the lane
    return blocked.reshape(-1)


@pytest.mark.parametrize("kind", ["uniform", "dups", "sorted", "reversed", "equal"])
def test_warp_sort_model_sorts(kind):
    rng = np.random.default_rng(7)
    if kind == "uniform":
        keys = rng.integers(0, 2**32, 1024, dtype=np.uint64).astype(np.uint32)
    elif kind == "dups":
        keys = rng.integers(0, 5, 1024).astype(np.uint32)
    elif kind == "sorted":
        keys = np.arange(1024, dtype=np.uint32)
    elif kind == "reversed":
        keys = np.arange(1024, dtype=np.uint32)[::-1].copy()
    else:
        keys = np.full(1024, 9, dtype=np.uint32)
    assert np.array_equal(warp_sort_model(keys), np.sort(keys))


def test_warp_sort_model_catches_a_missing_reversal():
    """Without the backwards read the blocks are not bitonic and the cascades
    fail: the reversal is what the sort rests on."""
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 2**32, 1024, dtype=np.uint64).astype(np.uint32)
    blocked = np.sort(keys.reshape(LANES, 32), axis=1)
    striped = blocked.copy()                                     # rows in order, no reversal
    striped = half_cleaners(striped, 1)
    rows = half_cleaners(striped.T, 16).T
    pairs = rows.reshape(16, 64)
    assert not all(np.all(p[1:] >= p[:-1]) for p in pairs)


def test_warp_sort_transposes_are_conflict_free():
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 2**32, 1024, dtype=np.uint64).astype(np.uint32)
    banks = []
    warp_sort_model(keys, banks)
    assert banks
    for kind, access in banks:
        if kind in ("chunk_store", "chunk_load"):
            # a 16-byte access is served per quarter-warp: 8 lanes, 8 distinct bank groups
            for q in range(4):
                groups = [g for quarter, g in access if quarter == q]
                assert len(groups) == 8 and len(set(groups)) == 8, (kind, q, groups)
        else:
            assert len(access) == 32 and len(set(access)) == 32, (kind, access)


def odd_even_pairs(n):
    """The lane network's compare-exchanges, in the loop order of lane_sort32
    (tile_sort.cuh): Batcher's odd-even merge sort, stage (p, k) comparing x
    and x + k for x = j + i, j from k mod p in steps of 2k, i < k, when both
    lie in the same block of 2p items."""
    out = []
    p = 1
    while p < n:
        k = p
        while k >= 1:
            j = k % p
            while j + k < n:
                for i in range(k):
                    x = j + i
                    if x + k < n and x // (2 * p) == (x + k) // (2 * p):
                        out.append((x, x + k))
                j += 2 * k
            k //= 2
        p *= 2
    return out


def batcher_recursive(lo, n):
    """Batcher's construction written recursively: sort both halves, then the
    odd-even merge (merge the even and the odd subsequences, then compare
    neighbours (2i-1, 2i))."""
    def merge(lo, n, r):
        step = 2 * r
        if step < n:
            yield from merge(lo, n, step)
            yield from merge(lo + r, n, step)
            for i in range(lo + r, lo + n - r, step):
                yield (i, i + r)
        else:
            yield (lo, lo + r)
    if n > 1:
        m = n // 2
        yield from batcher_recursive(lo, m)
        yield from batcher_recursive(lo + m, m)
        yield from merge(lo, n, 1)


def test_lane_network_is_batchers_odd_even_merge_sort():
    pairs = odd_even_pairs(32)
    assert len(pairs) == 191                       # (p^2 - p + 4) 2^(p-2) - 1 for n = 2^5
    assert sorted(pairs) == sorted(batcher_recursive(0, 32))
    # 0-1 principle, exhaustively for the 16-input network of the same loops
    p16 = odd_even_pairs(16)
    x = ((np.arange(1 << 16)[:, None] >> np.arange(16)) & 1).astype(np.uint8)
    for a, b in p16:
        lo, hi = np.minimum(x[:, a], x[:, b]), np.maximum(x[:, a], x[:, b])
        x[:, a], x[:, b] = lo, hi
    assert np.all(np.diff(x.astype(np.int8), axis=1) >= 0)
    # and random keys with many ties for the 32-input network
    rng = np.random.default_rng(3)
    y = rng.integers(0, 6, size=(20000, 32))
    for a, b in pairs:
        lo, hi = np.minimum(y[:, a], y[:, b]), np.maximum(y[:, a], y[:, b])
        y[:, a], y[:, b] = lo, hi
    assert np.all(np.diff(y, axis=1) >= 0)
