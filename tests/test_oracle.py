"""Pins for the CPU oracle: checks against facts the paper and the mathematics fix.

None of these compares the oracle with itself: brute-force enumeration of all
permutations for tiny n, the IEEE-754 totalOrder table, library routines
(numpy's stable sort) on the special cases that reduce to them, closed forms
(a permutation of 0..n-1 sorts to iota; the index payload then equals the
inverse permutation), and invariants of the partitioning (Sec. 4.1).  The last
test plants known mistakes in the oracle and checks that a pin catches each.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- brute force over all index permutations (definition of a stable sort) --

def brute_force_stable_perm(keys):
    """The unique index permutation that is non-decreasing and keeps equal keys
    in input order, found by enumerating every permutation (tiny n only)."""
    n = len(keys)
    found = []
    for p in itertools.permutations(range(n)):
        ok = True
        for a, b in zip(p, p[1:]):
            if keys[a] > keys[b] or (keys[a] == keys[b] and a > b):
                ok = False
                break
        if ok:
            found.append(p)
    assert len(found) == 1, "a stable sort order is unique"
    return np.array(found[0], dtype=np.uint64)


@pytest.mark.parametrize("n", range(0, 7))
def test_brute_force_all_permutations_small(n):
    for perm in itertools.permutations(range(n)):
        keys = np.array(perm, dtype=np.uint32)
        assert np.array_equal(oracle.argsort(keys), brute_force_stable_perm(list(perm)))


@pytest.mark.parametrize("n", range(1, 7))
def test_brute_force_words_with_repeats(n):
    """All 3^n words over {0,1,2}: stability decides among the equal keys."""
    for w in itertools.product(range(3), repeat=n):
        keys = np.array(w, dtype=np.uint32)
        assert np.array_equal(oracle.argsort(keys), brute_force_stable_perm(list(w)))


@pytest.mark.parametrize("n", [7, 8])
def test_all_permutations_sort_to_iota(n):
    """Every permutation of 0..n-1 sorts to iota, with the inverse permutation
    as index payload (closed form), for all n! inputs."""
    for perm in itertools.permutations(range(n)):
        keys = np.array(perm, dtype=np.uint32)
        k, v = oracle.sort(keys, synth.index_payload(n))
        assert np.array_equal(k, np.arange(n, dtype=np.uint32))
        inv = np.empty(n, dtype=np.uint32)
        inv[keys] = np.arange(n, dtype=np.uint32)
        assert np.array_equal(v, inv)


@pytest.mark.parametrize("n", [7, 8])
def test_all_words_stability(n):
    """All 3^n words: output non-decreasing, same multiset, and index payloads
    strictly increasing inside every run of equal keys."""
    for w in itertools.product(range(3), repeat=n):
        keys = np.array(w, dtype=np.uint32)
        k, v = oracle.sort(keys, synth.index_payload(n))
        assert np.all(k[1:] >= k[:-1])
        assert np.array_equal(np.bincount(k, minlength=3), np.bincount(keys, minlength=3))
        same = k[1:] == k[:-1]
        assert np.all(v[1:][same] > v[:-1][same])
        assert np.array_equal(keys[v], k)


# ---- library special cases -------------------------------------------------

@pytest.mark.parametrize("dtype,n", [(np.uint32, 200_000), (np.uint64, 100_000)])
def test_matches_numpy_stable_sort_integers(dtype, n):
    """For integer keys the order is numeric order, so numpy's stable argsort
    must produce the identical permutation (repeats included)."""
    keys = synth.uniform(n, 7, dtype) % dtype(5000)
    assert np.array_equal(oracle.argsort(keys), np.argsort(keys, kind="stable").astype(np.uint64))


def test_u64_high_word_decides():
    """Keys equal in the low word and different in the high word."""
    keys = (np.arange(64, dtype=np.uint64)[::-1] << np.uint64(32)) | np.uint64(7)
    k, _ = oracle.sort(keys)
    assert np.array_equal(k, np.sort(keys))


# ---- IEEE-754-2008 totalOrder (5.10) on binary32 bit patterns ----------------

def _load_total_order():
    rows = []
    with open(os.path.join(GOLDEN, "f32_total_order.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(int(line.split()[0], 16))
    return rows


TOTAL_ORDER_F32 = _load_total_order()  # IEEE 754-2008 clause 5.10, ascending


def test_f32_total_order_table():
    want = np.array(TOTAL_ORDER_F32, dtype=np.uint32)
    rng = np.random.default_rng(0)
    for _ in range(200):
        shuffled = rng.permutation(want).view(np.float32)
        k, _ = oracle.sort(shuffled)
        assert np.array_equal(k.view(np.uint32), want)
    f = want.view(np.float32)
    for i in range(len(want)):
        for j in range(len(want)):
            assert oracle.less(f, i, j) == (i < j)


def test_f32_finite_matches_numeric_order():
    """Away from NaN and signed zero, totalOrder is numeric order: compare with
    numpy's stable sort on the float values (a library routine)."""
    x = synth.normal_f32(50_000, 5)
    bits = x.view(np.uint32)
    x = x[~np.isnan(x) & (bits != 0x80000000)]
    assert np.array_equal(oracle.argsort(x), np.argsort(x, kind="stable").astype(np.uint64))


def test_f32_negative_zero_before_positive_zero_and_bits_kept():
    x = np.array([0.0, -0.0, 0.0, -0.0], dtype=np.float32)
    k, v = oracle.sort(x, synth.index_payload(4))
    assert list(k.view(np.uint32)) == [0x80000000, 0x80000000, 0, 0]
    assert list(v) == [1, 3, 0, 2]


# ---- closed forms at larger sizes --------------------------------------------

def test_permutation_closed_form():
    n = 1 << 18
    keys = synth.permutation(n, 3)
    k, v = oracle.sort(keys, synth.index_payload(n))
    assert np.array_equal(k, np.arange(n, dtype=np.uint32))
    inv = np.empty(n, dtype=np.uint32)
    inv[keys] = np.arange(n, dtype=np.uint32)
    assert np.array_equal(v, inv)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_interleaved_runs_closed_form(dtype):
    n, K = 1 << 15, 8
    keys = synth.interleaved(n, K, 32, dtype)
    k, _ = oracle.sort(keys)
    iota = np.arange(n, dtype=np.uint64)
    want = (iota << np.uint64(32)) | iota if np.dtype(dtype) == np.uint64 else iota.astype(np.uint32)
    assert np.array_equal(k, want)


def test_sortedness_zero_swaps_is_identity():
    keys = synth.sortedness(10_000, 0, 1)
    k, _ = oracle.sort(keys)
    assert np.array_equal(k, keys)


# ---- base case and merge round -------------------------------------------------

def test_tile_sort_each_tile_is_a_sorted_permutation_of_itself():
    keys = synth.uniform(10_000, 4)
    out, _ = oracle.tile_sort(keys, 1024)
    for s in range(0, 10_000, 1024):
        assert np.array_equal(out[s:s + 1024], np.sort(keys[s:s + 1024]))


def test_merge_pass_matches_numpy_per_group():
    run, K = 512, 4
    keys = synth.uniform(run * 11 + 100, 9)
    pre, _ = oracle.tile_sort(keys, run)
    out, _ = oracle.merge_pass(pre, run, K)
    for gs, ge in oracle.group_bounds(keys.shape[0], run, K):
        assert np.array_equal(out[gs:ge], np.sort(keys[gs:ge]))


# ---- partitioning (Sec. 4.1) ----------------------------------------------------

def _composite_rank_key(runs):
    """(key, run, pos) triples, the strict order under which pivots are unique."""
    return [(int(x), r, p) for r, run in enumerate(runs) for p, x in enumerate(run)]


@pytest.mark.parametrize("seed", range(30))
def test_corank_definition_brute_force(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 6))
    runs = [np.sort(rng.integers(0, 4, size=int(rng.integers(0, 7))).astype(np.uint32)) for _ in range(K)]
    items = sorted(_composite_rank_key(runs))
    for k in range(len(items) + 1):
        c = oracle.corank(runs, k)
        want = np.zeros(K, dtype=np.int64)
        for (_, r, _) in items[:k]:
            want[r] += 1
        assert np.array_equal(c, want)
        assert c.sum() == k
        # non-overlap: everything selected precedes everything not selected
        sel = [(int(runs[r][p]), r, p) for r in range(K) for p in range(c[r])]
        rest = [(int(runs[r][p]), r, p) for r in range(K) for p in range(c[r], len(runs[r]))]
        if sel and rest:
            assert max(sel) < min(rest)


def test_corank_distinct_values_closed_form():
    """With distinct values, c[r] = #{x in run r : x < v_k}, v_k the k-th smallest value."""
    rng = np.random.default_rng(1)
    vals = rng.permutation(4000).astype(np.uint32)
    runs = [np.sort(vals[i * 500:(i + 1) * 500]) for i in range(8)]
    allv = np.sort(vals)
    for k in [1, 17, 500, 1999, 3999]:
        thr = allv[k]
        want = np.array([np.sum(r < thr) for r in runs])
        assert np.array_equal(oracle.corank(runs, k), want)


def test_splitter_table_rows():
    run, K, S = 256, 4, 128
    keys = synth.uniform(run * 9 + 37, 2) % np.uint32(50)
    pre, _ = oracle.tile_sort(keys, run)
    tab = oracle.splitter_table(pre, run, K, S)
    t = 0
    for gs, ge in oracle.group_bounds(pre.shape[0], run, K):
        runs = [pre[s:min(s + run, ge)] for s in range(gs, gs + run * K, run)]
        runs = [r if r.size else np.zeros(0, np.uint32) for r in runs]
        for j in range((ge - gs + S - 1) // S):
            assert np.array_equal(tab[t], oracle.corank(runs, j * S))
            t += 1
    assert t == tab.shape[0]


# ---- planted mistakes: every one must trip a pin ----------------------------

def _pins_hold() -> bool:
    try:
        for w in itertools.product(range(3), repeat=5):
            keys = np.array(w, dtype=np.uint32)
            if not np.array_equal(oracle.argsort(keys), brute_force_stable_perm(list(w))):
                return False
        keys = synth.permutation(4096, 1)
        k, _ = oracle.sort(keys)
        if not np.array_equal(k, np.arange(4096, dtype=np.uint32)):
            return False
        k64 = (np.arange(64, dtype=np.uint64)[::-1] << np.uint64(32)) | np.uint64(7)
        if not np.array_equal(oracle.sort(k64)[0], np.sort(k64)):
            return False
        want = np.array(TOTAL_ORDER_F32, dtype=np.uint32)
        got, _ = oracle.sort(np.random.default_rng(0).permutation(want).view(np.float32))
        if not np.array_equal(got.view(np.uint32), want):
            return False
        return True
    except AssertionError:
        return False


def test_segmented_sort_closed_form_and_brute_force():
    """Batched sort: each segment of concatenated permutations sorts to its own
    iota (closed form) and the index payload becomes each segment's inverse
    permutation; tiny segments of words with repeats match brute force."""
    sizes = [0, 1, 5, 300, 0, 2, 4097]
    parts = [synth.permutation(n, 40 + i) for i, n in enumerate(sizes)]
    keys = np.concatenate(parts).astype(np.uint32)
    off = synth.offsets_of(sizes)
    vals = synth.index_payload(keys.size)
    k, v = oracle.segmented_sort(keys, off, vals)
    for i, n in enumerate(sizes):
        a, b = int(off[i]), int(off[i + 1])
        assert np.array_equal(k[a:b], np.arange(n, dtype=np.uint32))
        inv = np.empty(n, dtype=np.uint32)
        inv[parts[i]] = np.arange(n, dtype=np.uint32)
        assert np.array_equal(v[a:b] - np.uint32(a), inv)
    words = np.array([2, 0, 1, 0, 2, 1, 1, 0, 2], dtype=np.uint32)
    off = np.array([0, 4, 4, 9], dtype=np.int64)
    k, v = oracle.segmented_sort(words, off, np.arange(9, dtype=np.uint32))
    for a, b in [(0, 4), (4, 9)]:
        p = brute_force_stable_perm(list(words[a:b]))
        assert list(v[a:b]) == [a + i for i in p]
    # no item crosses a segment boundary
    assert sorted(k[:4].tolist()) == sorted(words[:4].tolist())


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5])
def test_planted_mistakes_are_caught(mutation):
    assert _pins_hold()
    with oracle.mutation(mutation):
        assert not _pins_hold(), f"planted mistake {mutation} went unnoticed"
    assert _pins_hold()


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_oracle_equals_the_serial_oracle(threads):
    """The CPU baseline's all-cores variant splits the same recursion into
    threads: it must return exactly the serial oracle's result."""
    for n, mod in [(0, 0), (1, 0), (65535, 7), (65537, 0), (300001, 1000), (1 << 20, 3)]:
        keys = synth.uniform(n, n + threads, np.uint32)
        if mod:
            keys = keys % np.uint32(mod)
        vals = synth.index_payload(n)
        a = oracle.sort(keys, vals)
        b = oracle.sort_parallel(keys, vals, threads)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    f = synth.normal_f32(200000, 5)
    assert np.array_equal(oracle.sort(f)[0].view(np.uint32), oracle.sort_parallel(f, None, threads)[0].view(np.uint32))
