"""GPU parity of the paper's merge variants (Sec. 7, future work): the
heap-free partition merge (multiway merging driven by the parallel
partitioning alone; mms_merge_pass_partition, MMS_MERGE_PARTITION) and the
pipelined merge (a producer warp staging the next tile while the merging
warps merge the current one; mms_merge_pass_pipelined, MMS_MERGE_PIPELINED).
Every merge round of either against the CPU oracle, bit for bit, over the
fanouts, key types, input structures and ragged group shapes the CTA-tree
merge is tested on.
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import assert_bits_equal, kt_of, sorted_runs, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["partition", "pipelined"])
def variant(request, gpu):
    return {"partition": gpu.MERGE_PARTITION, "pipelined": gpu.MERGE_PIPELINED}[request.param]


def part_sort(mms, keys, fanout=0, variant=None):
    t = to_dev(keys)
    mms.sort_keys(t, fanout=fanout, kt=kt_of(keys.dtype, mms),
                  merge_variant=mms.MERGE_PARTITION if variant is None else variant)
    return to_host(t, keys.dtype)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("K,runs_mult,mod", [(2, 1, 0), (3, 1, 0), (4, 2, 0), (5, 1, 0), (8, 1, 5),
                                             (8, 3, 0), (16, 1, 0), (16, 1, 2), (32, 1, 0)])
def test_variant_merge_pass_matches_oracle(gpu, variant, dtype, K, runs_mult, mod):
    """One round fed the oracle's pivot table: several tiles per group, a
    short last group and a ragged last tile; `mod` makes heavy duplicates."""
    import torch
    kt = kt_of(dtype, gpu)
    S = gpu.tile_items(kt)
    run_len = S * runs_mult
    n = run_len * (2 * K + 1) + S + 77
    keys = synth.uniform(n, 7 + K, dtype)
    if mod:
        keys = keys % dtype(mod)
    pre = sorted_runs(keys, run_len)
    table = torch.from_numpy(oracle.splitter_table(pre, run_len, K, S)).cuda()
    out = to_dev(np.zeros_like(pre))
    ws = torch.zeros(gpu.workspace_bytes(kt, 16), dtype=torch.uint8, device="cuda")
    gpu.merge_pass(to_dev(pre), out, run_len, K, table, workspace=ws, kt=kt, merge_variant=variant)
    want, _ = oracle.merge_pass(pre, run_len, K)
    assert_bits_equal(to_host(out, dtype), want)
    gpu.workspace_status(ws)


@pytest.mark.parametrize("fanout", [2, 3, 4, 6, 8, 12, 16, 24, 32, 0])
def test_variant_sort_u32_fanouts(gpu, variant, fanout):
    n = 8192 * 70 + 4321
    keys = synth.uniform(n, fanout + 300, np.uint32)
    want, _ = oracle.sort(keys)
    assert_bits_equal(part_sort(gpu, keys, fanout, variant), want)


@pytest.mark.parametrize("kind", ["sorted", "reversed", "equal", "two_values", "sortedness",
                                  "interleaved", "permutation"])
def test_variant_sort_u32_structured(gpu, variant, kind):
    """Presorted and reversed runs (pieces that are whole segments or empty),
    all-ones keys (bit-identical to the networks' pads), two values, and the
    stride-32 interleaving of C3."""
    n = 8192 * 40 + 999
    if kind == "sorted":
        keys = np.arange(n, dtype=np.uint32)
    elif kind == "reversed":
        keys = np.arange(n, dtype=np.uint32)[::-1].copy()
    elif kind == "equal":
        keys = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    elif kind == "two_values":
        keys = (synth.uniform(n, 3, np.uint32) & np.uint32(1)) * np.uint32(0xFFFFFFFF)
    elif kind == "sortedness":
        keys = synth.sortedness(n, 1000, 4)
    elif kind == "interleaved":
        keys = synth.interleaved(n, 8, 32, np.uint32)
    else:
        keys = synth.permutation(n, 9)
    want, _ = oracle.sort(keys)
    for fanout in (4, 16, 0):
        assert_bits_equal(part_sort(gpu, keys, fanout, variant), want)


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 8193, 4096 * 37 + 11])
def test_variant_sort_u64(gpu, variant, n):
    keys = synth.uniform(n, 23, np.uint64)
    keys[1::2] = keys[0::2][: keys[1::2].size]          # every key at least twice
    want, _ = oracle.sort(keys)
    for fanout in (0, 8):
        assert_bits_equal(part_sort(gpu, keys, fanout, variant), want)


def test_variant_sort_f32_specials(gpu, variant):
    """Float keys: the order transform is undone on the root level of the
    warp's tree, including roots that are copies (one side empty)."""
    n = 8192 * 20 + 333
    keys = synth.normal_f32(n, 5)
    keys[::97] = np.float32(-0.0)
    keys[::89] = np.float32(0.0)
    keys[::101] = np.float32(np.inf)
    keys[::103] = np.float32(-np.inf)
    keys[::107] = np.float32(np.nan)
    keys[:: 8192 * 3] = np.float32(1.5)
    want, _ = oracle.sort(keys)
    for fanout in (2, 5, 0):
        assert_bits_equal(part_sort(gpu, keys, fanout, variant), want)
    sortd = np.sort(keys[np.isfinite(keys)])
    assert_bits_equal(part_sort(gpu, sortd, 8, variant), oracle.sort(sortd)[0])


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64, np.float32])
@pytest.mark.parametrize("tiles,tail,fanout", [(3, 7, 8), (5, 100, 4), (9, 0, 8), (17, 1, 16),
                                               (33, 4095, 32), (6, 0, 4)])
def test_variant_groups_with_fewer_runs_than_k(gpu, variant, dtype, tiles, tail, fanout):
    T = gpu.tile_items(gpu.KEY_U64 if dtype == np.uint64 else gpu.KEY_U32)
    n = tiles * T + tail
    if dtype == np.float32:
        keys = synth.normal_f32(n, 17 * tiles + fanout)
    else:
        keys = synth.uniform(n, 19 * tiles + fanout, dtype)
    want, _ = oracle.sort(keys)
    assert_bits_equal(part_sort(gpu, keys, fanout, variant), want)


@pytest.mark.parametrize("kt_name", ["u32", "f32", "u64"])
def test_variant_pairs_stable(gpu, variant, kt_name):
    """Key-value sorts (rounds on 8-byte composites, two passes for 8-byte
    keys): keys and the stable order of the index payload."""
    import torch
    n = 4096 * 50 + 77
    if kt_name == "u32":
        keys = synth.uniform(n, 31, np.uint32) % np.uint32(5000)
    elif kt_name == "f32":
        keys = synth.normal_f32(n, 31)
        keys[::13] = np.float32(-0.0)
    else:
        keys = synth.uniform(n, 31, np.uint64) % np.uint64(1 << 40)
    vals = np.arange(n, dtype=np.uint32)
    kt = kt_of(keys.dtype, gpu)
    tk, tv = to_dev(keys), torch.from_numpy(vals.view(np.int32)).cuda()
    gpu.sort_pairs(tk, tv, kt=kt, merge_variant=variant)
    want_k, want_v = oracle.sort(keys, vals)
    assert_bits_equal(to_host(tk, keys.dtype), want_k)
    assert np.array_equal(to_host(tv, np.uint32), want_v)


def test_variant_same_bits_as_tree(gpu, variant):
    """Both variants on the same inputs give the same bits (several plans)."""
    n = 8192 * 123 + 45
    for seed, fanout in ((1, 0), (2, 7), (3, 32)):
        keys = synth.uniform(n, seed, np.uint32) % np.uint32(100000)
        t1, t2 = to_dev(keys), to_dev(keys)
        gpu.sort_keys(t1, fanout=fanout, kt=gpu.KEY_U32)
        gpu.sort_keys(t2, fanout=fanout, kt=gpu.KEY_U32, merge_variant=variant)
        assert_bits_equal(to_host(t2, np.uint32), to_host(t1, np.uint32))


def test_variant_rejects_other_tile_geometry(gpu, variant):
    t = to_dev(synth.uniform(100000, 1, np.uint32))
    with pytest.raises(gpu.MMSError):
        gpu.sort_keys(t, kt=gpu.KEY_U32, tile_items=4096, merge_variant=variant)
    with pytest.raises(gpu.MMSError):
        gpu.sort_keys(t, kt=gpu.KEY_U32, merge_variant=7)


@pytest.mark.slow
def test_variant_full_size_permutation_1e8_u32(gpu, variant):
    """The bench workload (10^8 u32, uniform permutation of 0..n-1, plan
    16,16,8,8) sorts to iota; checked on the device."""
    import torch
    n = 100_000_000
    g = torch.Generator(device="cuda").manual_seed(1234)
    t = torch.randperm(n, device="cuda", generator=g).to(torch.int32)
    gpu.sort_keys(t, kt=gpu.KEY_U32, merge_variant=variant)
    ok = bool(torch.equal(t, torch.arange(n, device="cuda", dtype=torch.int32)))
    del t
    torch.cuda.empty_cache()
    assert ok
