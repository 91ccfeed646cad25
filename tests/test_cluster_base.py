"""GPU parity of the cluster base case (runs of 2, 4 or 8 CTA tiles sorted by one
thread-block cluster, Sec. 4.3) through the C ABI, against the CPU oracle.

The cluster base case is an option (mms_options.base_items); the default base
case sorts one CTA tile per run.  Sizes at or below one run leave no merge
round, so the base case's output is
the whole result; larger sizes add ragged last clusters (CTAs with a partial
tile or none) and the merge rounds over the longer runs.  Keys are compared
bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

from test_gpu_parity import assert_bits_equal, kt_of, to_dev, to_host

pytestmark = pytest.mark.gpu


def sort_with(gpu, keys, **kw):
    t = to_dev(keys)
    gpu.sort_keys(t, kt=kt_of(keys.dtype, gpu), **kw)
    return to_host(t, keys.dtype)


def make(kind, n, seed):
    if kind == "uniform":
        return synth.uniform(n, seed, np.uint32)
    if kind == "dups":
        return synth.uniform(n, seed, np.uint32) % np.uint32(7)
    if kind == "f32":
        return synth.normal_f32(n, seed)
    if kind == "sorted":
        return np.arange(n, dtype=np.uint32)
    if kind == "reversed":
        return np.arange(n, dtype=np.uint32)[::-1].copy()
    if kind == "equal":
        return np.full(n, 0xFFFFFFFF, np.uint32)       # equal to the pad key
    raise ValueError(kind)


@pytest.mark.parametrize("n", [8193, 8196, 16384, 20000, 32767, 32768])
@pytest.mark.parametrize("kind", ["uniform", "dups", "f32"])
def test_one_run_is_the_base_case_alone(gpu, n, kind):
    kt = gpu.KEY_F32 if kind == "f32" else gpu.KEY_U32
    assert gpu.base_run_items(kt, n, base_items=32768) == 32768
    assert gpu.plan(kt, n, base_items=32768) == []
    keys = make(kind, n, n % 97)
    assert_bits_equal(sort_with(gpu, keys, base_items=32768), oracle.sort(keys)[0])


@pytest.mark.parametrize("base", [16384, 32768, 65536])
@pytest.mark.parametrize("fanout", [0, 2, 16])
def test_cluster_runs_then_merge_rounds(gpu, base, fanout):
    n = 3 * base + 4097                                # full clusters and a ragged one
    keys = make("uniform", n, base // 1024 + fanout)
    assert gpu.base_run_items(gpu.KEY_U32, n, base_items=base) == base
    assert_bits_equal(sort_with(gpu, keys, fanout=fanout, base_items=base), oracle.sort(keys)[0])


@pytest.mark.parametrize("base", [16384, 65536])
@pytest.mark.parametrize("extra", [1, 8191, 8192 + 5])
def test_ragged_last_cluster(gpu, base, extra):
    n = 2 * base + extra                               # last cluster: one partial CTA, others empty
    keys = make("dups", n, extra)
    assert_bits_equal(sort_with(gpu, keys, base_items=base), oracle.sort(keys)[0])


@pytest.mark.parametrize("kind", ["sorted", "reversed", "equal", "f32"])
def test_structured_inputs(gpu, kind):
    n = 5 * 32768 + 3
    keys = make(kind, n, 5)
    assert_bits_equal(sort_with(gpu, keys, base_items=32768), oracle.sort(keys)[0])


def test_same_result_as_one_cta_runs(gpu):
    """The run length changes the plan, not the result."""
    n = 777_777
    keys = make("uniform", n, 3)
    a = sort_with(gpu, keys, base_items=32768)         # runs of a 4-CTA cluster
    b = sort_with(gpu, keys)                           # runs of one CTA tile (the default)
    assert gpu.plan(gpu.KEY_U32, n, base_items=32768) != gpu.plan(gpu.KEY_U32, n)
    assert_bits_equal(a, b)
    assert_bits_equal(a, oracle.sort(keys)[0])


def test_offset_slice_and_workspace(gpu):
    """Keys at a 4-byte offset from the 16-byte grid, with a caller workspace."""
    import torch
    n = 2 * 32768 + 999
    keys = make("uniform", n, 8)
    t = to_dev(np.concatenate([np.zeros(1, np.uint32), keys]))
    sl = t[1:]
    ws = torch.empty(gpu.workspace_bytes(gpu.KEY_U32, n), dtype=torch.uint8, device="cuda")
    gpu.sort_keys(sl, workspace=ws, kt=gpu.KEY_U32, base_items=32768)
    gpu.workspace_status(ws)
    assert_bits_equal(to_host(sl, np.uint32), oracle.sort(keys)[0])


@pytest.mark.slow
@pytest.mark.parametrize("base", [16384, 32768, 65536])
def test_full_size_permutation_1e8(gpu, base):
    """The bench workload (a uniform permutation of 0..10^8-1) sorted from
    cluster runs must give iota."""
    import torch
    n = 10**8
    t = to_dev(synth.permutation(n, 1))
    gpu.sort_keys(t, kt=gpu.KEY_U32, base_items=base)
    step = 1 << 26
    for a in range(0, n, step):
        b = min(n, a + step)
        want = torch.arange(a, b, dtype=torch.int64, device=t.device)
        assert torch.equal(t[a:b].to(torch.int64) & 0xFFFFFFFF, want)
