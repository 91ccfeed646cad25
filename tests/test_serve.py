"""The serving loop on the GPU: a mix of requests of every key type, with and
without values, arriving faster than they are served.  Every result must
equal the oracle's stable sort of that request, and equal the same request
served alone (one plain whole-array sort at a time), bit for bit; the mix
must actually have been coalesced into batched launches and overlapped on
the device; and a tight memory budget must only delay requests."""
import numpy as np
import pytest

import oracle
import synth
from paper_1702_07961_gb300 import KEY_F32, KEY_U32, KEY_U64
from paper_1702_07961_gb300.serve import Request, SortServer, poisson_arrivals, serve_serial

pytestmark = pytest.mark.gpu

NP = {KEY_U32: np.uint32, KEY_U64: np.uint64, KEY_F32: np.float32}


def make_requests(count, seed, lo, hi, rate, big=()):
    sizes = list(synth.segment_sizes(count, lo, hi, seed)) + list(big)
    rng = np.random.default_rng(seed)
    arrivals = poisson_arrivals(len(sizes), rate, seed)
    reqs = []
    for i, n in enumerate(sizes):
        n = int(n)
        kt = int(rng.choice([KEY_U32, KEY_U64, KEY_F32]))
        if kt == KEY_F32:
            keys = synth.normal_f32(n, seed * 1000 + i)
        elif kt == KEY_U64:
            keys = synth.uniform(n, seed * 1000 + i, np.uint64) % np.uint64(1 << 40)
        else:
            keys = synth.uniform(n, seed * 1000 + i, np.uint32) % np.uint32(1000)   # many ties
        vals = synth.uniform(n, seed * 2000 + i, np.uint32) if rng.random() < 0.5 else None
        reqs.append(Request(i, kt, keys, vals, float(arrivals[i])))
    return reqs


def outputs(r):
    k = r.out_keys.numpy().view(NP[r.kt])
    v = None if r.out_values is None else r.out_values.numpy().view(np.uint32)
    return k, v


def bits(a):
    return a.view(np.uint64 if a.dtype.itemsize == 8 else np.uint32)


def clone(reqs):
    return [Request(r.rid, r.kt, r.keys, r.values, r.arrival) for r in reqs]


def test_served_mix_equals_oracle_and_alone(gpu):
    reqs = make_requests(60, 5, 1 << 10, 1 << 17, rate=50000.0, big=[(1 << 21) + 3, 3 << 19])
    srv = SortServer(budget_bytes=3 << 30, slots=4)
    srv.run(reqs)
    assert srv.coalesced > 0 and srv.groups < len(reqs), "no request was coalesced"
    assert srv.max_inflight > 1, "launch groups never overlapped"
    assert all(r.error is None for r in reqs), "a launch group reported a device-side error"
    alone = serve_serial(clone(reqs))
    for r, a in zip(sorted(reqs, key=lambda x: x.rid), sorted(alone, key=lambda x: x.rid)):
        gk, gv = outputs(r)
        wk, wv = oracle.sort(r.keys, r.values)
        assert np.array_equal(bits(gk), bits(wk)), f"request {r.rid} keys differ from the oracle"
        ak, av = outputs(a)
        assert np.array_equal(bits(gk), bits(ak)), f"request {r.rid} differs alone vs in the mix"
        if r.values is not None:
            assert np.array_equal(gv, wv) and np.array_equal(gv, av)


def test_tight_budget_only_delays(gpu):
    reqs = make_requests(24, 9, 1 << 12, 1 << 18, rate=100000.0)
    srv = SortServer(budget_bytes=48 << 20, slots=3, batch_max=1 << 19)
    srv.run(reqs)
    assert srv.peak_bytes <= 48 << 20
    for r in reqs:
        gk, gv = outputs(r)
        wk, wv = oracle.sort(r.keys, r.values)
        assert np.array_equal(bits(gk), bits(wk))
        if r.values is not None:
            assert np.array_equal(gv, wv)
