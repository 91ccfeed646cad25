"""Host model of the splitter's search (splitter.cuh: splitter_row), checked
against brute force.

The kernel finds, for output rank k of a group of K sorted runs, how many
items each run contributes among the k smallest under the order (key, run,
position), by stride halving on regular samples: at stride s the lanes hold
the exact answer of the s-sample problem for rank floor(k/s); halving s adds
one candidate per run, and the largest items are dropped until the count is
floor(2k/s).  The model replays those steps one lane per run -- the same
probes, the same "drop every candidate above all selected items first" step,
the same pops from the largest top -- and checks:
  * the result equals brute force on small inputs with many duplicates;
  * every level drops K - 1 or K items: K minus the low bit of the level's
    rank, the closed form the kernel uses instead of a reduction;
  * every probed position lies below 2k, so for n < 2^30 the kernel's 32-bit
    counts and positions cannot overflow.
"""
import numpy as np
import pytest


PROBES = []


def item(run, pos):
    """(pad, key): positions past the run's end are pads, after every real item."""
    PROBES.append(pos)
    return (True, 0) if pos >= len(run) else (False, int(run[pos]))


def before(a, ra, b, rb):
    """Item a of run ra strictly before item b of run rb (ra != rb)."""
    if a[0] != b[0]:
        return b[0]
    if not a[0] and a[1] != b[1]:
        return a[1] < b[1]
    return ra < rb


def argmax(lanes, vals):
    """The lane with the largest item among `lanes` (pads first, then the
    largest key, ties to the highest lane), or -1."""
    if not lanes:
        return -1
    pads = [r for r in lanes if vals[r][0]]
    if pads:
        return max(pads)
    mx = max(vals[r][1] for r in lanes)
    return max(r for r in lanes if vals[r][1] == mx)


def argmin(lanes, vals):
    reals = [r for r in lanes if not vals[r][0]]
    if not reals:
        return min(lanes)
    mn = min(vals[r][1] for r in reals)
    return min(r for r in reals if vals[r][1] == mn)


def splitter_model(runs, k, drops):
    K = len(runs)
    d = [0] * K
    e = [(False, 0)] * K
    for lev in range(k.bit_length(), 0, -1):
        sh = lev - 1
        kp = k >> sh
        dd = [2 * x for x in d]
        o = [item(runs[r], ((dd[r] + 1) << sh) - 1) for r in range(K)]
        z = [item(runs[r], ((dd[r] - 1) << sh) - 1) if d[r] >= 1 else (False, 0) for r in range(K)]
        jrem = 2 * sum(d) + K - kp
        # the kernel's closed form: the lanes hold the pivots of rank k >> lev, so sum(d) = k >> lev
        assert sum(d) == k >> lev and jrem == K - (kp & 1)
        drops.append((jrem, K))
        cnt = [x + 1 for x in dd]
        mz = argmax([r for r in range(K) if d[r] >= 1], e)
        above = [mz < 0 or r == mz or before(e[mz], mz, o[r], r) for r in range(K)]
        u = sum(above)
        if u <= jrem:
            for r in range(K):
                if above[r]:
                    cnt[r] = dd[r]
            pops = jrem - u
        else:
            mn = argmin([r for r in range(K) if above[r]], o)
            for r in range(K):
                if above[r] and r != mn:
                    cnt[r] = dd[r]
            pops = 0
        top = [o[r] if cnt[r] == dd[r] + 1 else e[r] for r in range(K)]
        if mz >= 0 and pops > 0:
            # the kernel's first drop without a reduction: the largest top is
            # lane mz's e, whose own candidate the bulk step dropped
            assert argmax([r for r in range(K) if cnt[r] >= 1], top) == mz and cnt[mz] == dd[mz]
            cnt[mz] -= 1
            top[mz] = z[mz]
            pops -= 1
        for _ in range(pops):
            w = argmax([r for r in range(K) if cnt[r] >= 1], top)
            cnt[w] -= 1
            if cnt[w] >= 1:
                if cnt[w] == dd[w]:
                    top[w] = e[w]
                elif cnt[w] == dd[w] - 1:
                    top[w] = z[w]
                else:
                    top[w] = item(runs[w], (cnt[w] << sh) - 1)
        d, e = cnt, top
    return d


def brute(runs, k):
    order = sorted((int(v), r, p) for r, run in enumerate(runs) for p, v in enumerate(run))
    counts = [0] * len(runs)
    for _, r, _ in order[:k]:
        counts[r] += 1
    return counts


@pytest.mark.parametrize("K", [2, 3, 4, 5, 8])
@pytest.mark.parametrize("vals", [3, 1000])
def test_splitter_model_matches_brute_force(K, vals):
    rng = np.random.default_rng(K * 100 + vals)
    for trial in range(40):
        lens = rng.integers(0, 40, K)
        runs = [np.sort(rng.integers(0, vals, n)) for n in lens]
        total = int(sum(lens))
        for k in sorted({0, 1, total // 3, total // 2, total - 1, total} - {-1}):
            if k < 0:
                continue
            drops = []
            PROBES.clear()
            assert splitter_model(runs, k, drops) == brute(runs, k), (trial, lens, k)
            # every probe lies below 2k: the kernel's 32-bit variant (n < 2^30) cannot overflow
            assert all(0 <= p < 2 * k for p in PROBES), (k, max(PROBES, default=0))
            # every level drops K - 1 or K items (one warp reduction, exact modulo 2^32)
            assert all(K - 1 <= j <= K for j, _ in drops), drops


def test_splitter_model_equal_keys_follow_run_order():
    """All keys equal: the order falls back to (run, position), so the first
    runs are taken whole."""
    runs = [np.full(5, 7), np.full(3, 7), np.full(4, 7)]
    assert splitter_model(runs, 6, []) == [5, 1, 0]
    assert splitter_model(runs, 9, []) == [5, 3, 1]
