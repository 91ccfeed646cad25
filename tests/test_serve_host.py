"""Host logic of the serving loop (no GPU): the device arena's first-fit
allocator, launch-group formation, and the Poisson arrival process."""
import numpy as np
import pytest

from paper_1702_07961_gb300 import KEY_F32, KEY_U32, KEY_U64
from paper_1702_07961_gb300.serve import (DeviceArena, Request, finish_group, form_group,
                                          poisson_arrivals, summarize)


def test_arena_first_fit_and_merge():
    a = DeviceArena(10 * 256)
    x = a.alloc(100)          # rounds to 256
    y = a.alloc(700)          # 768
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 1024)
    assert a.bytes_used == 256 + 768 + 256
    assert a.alloc(10 * 256) is None
    a.free(y)
    assert a.alloc(512) == 256                # first fit reuses the hole
    a.free(x)
    a.free(256)
    a.free(z)
    assert a.bytes_used == 0 and a.free_list == [(0, 2560)]   # every block merged back


def test_arena_random_churn_never_overlaps():
    rng = np.random.default_rng(1)
    a = DeviceArena(1 << 20)
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            off = list(live)[rng.integers(len(live))]
            a.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 40000))
            off = a.alloc(n)
            if off is not None:
                live[off] = a.used[off]
        spans = sorted(live.items())
        for (o1, l1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + l1 <= o2
        assert sum(l for _, l in a.free_list) + a.bytes_used == a.size


def req(i, n, kt=KEY_U32, pairs=False):
    return Request(i, kt, np.zeros(n, dtype=np.uint32 if kt != KEY_U64 else np.uint64),
                   np.zeros(n, np.uint32) if pairs else None)


def test_group_coalesces_small_requests_of_one_class_in_fifo_order():
    q = [req(0, 1000), req(1, 2000, KEY_F32), req(2, 3000), req(3, 5 << 20), req(4, 4000),
         req(5, 100, pairs=True), req(6, 50)]
    g = form_group(q, small_max=1 << 20, batch_max=1 << 25, max_segments=64)
    assert [r.rid for r in g] == [0, 2, 4, 6]          # same class (u32, no values), small, in order


def test_group_caps_and_large_requests():
    q = [req(0, 6 << 20), req(1, 10)]
    assert [r.rid for r in form_group(q, 1 << 20, 1 << 25, 64)] == [0]      # large: alone
    q = [req(i, 1000) for i in range(10)]
    assert len(form_group(q, 1 << 20, 3500, 64)) == 3                      # item cap
    assert len(form_group(q, 1 << 20, 1 << 25, 4)) == 4                    # segment cap


def test_group_without_coalescing():
    """small_max = 0 (bench --small-max 0): every request is its own group."""
    q = [req(i, 1000) for i in range(5)]
    assert [r.rid for r in form_group(q, 0, 1 << 25, 64)] == [0]
    assert [r.rid for r in form_group(q[1:], 0, 1 << 25, 64)] == [1]


def test_poisson_arrivals_rate():
    t = poisson_arrivals(20000, 250.0, 3)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 20000 - 1 / 250.0) < 0.05 / 250.0 * 10
    gaps = np.diff(t)
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) < 0.05      # exponential gaps: CV = 1


def test_plan_cost_fit_skips_partial_last_rounds():
    """fit_plan_costs averages only rounds that merged K runs per group."""
    from paper_1702_07961_gb300.autotune import fit_plan_costs
    rows = []
    for key in ("u32", "u64"):
        for K in (2, 4, 8, 16, 32):
            # two full rounds at 1.0 + 0.1 ms, then a last round over 3 runs at 0.5 + 0.1 ms
            rows.append({"key": key, "n": 10**8, "K": K, "merge_pass_ms": [1.0, 1.0, 0.5],
                         "splitter_ms": [0.1, 0.1, 0.1], "runs_merged": [K, K, min(K, 3)]})
    got = fit_plan_costs(rows)
    # K = 2: every round merged 2 runs, the last included (0.6 ms); K >= 4: the last is left out
    assert got["u32"][0] == pytest.approx((1.1 + 1.1 + 0.6) / 3)
    for c in got["u32"][1:] + got["u64"][1:]:
        assert c == pytest.approx(1.1)


def test_nonzero_status_word_marks_the_group_failed():
    """A sort stopped on the device (workspace status word non-zero) must not be
    returned as a sorted result: every request of its launch group fails."""
    ok = [req(0, 10), req(1, 20)]
    finish_group(ok, 0, 1.5)
    assert all(r.finish == 1.5 and r.error is None for r in ok)
    timed_out = [req(2, 10), req(3, 30)]
    finish_group(timed_out, 1, 2.0)                 # the device's time-out word
    assert all(r.finish == 2.0 and "timed out" in r.error for r in timed_out)
    bad = [req(4, 10)]
    finish_group(bad, 2, 2.5)                       # a failed consistency check
    assert "consistency" in bad[0].error
    assert summarize(ok + timed_out + bad)["failed"] == 3
