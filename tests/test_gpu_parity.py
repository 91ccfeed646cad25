"""GPU parity: every hot-path step through the C ABI against the CPU oracle.

Integer and float keys are compared bit for bit (sorting does no arithmetic on
keys, so the tolerance is exactly zero).  Inputs are seeded and synthetic,
shaped like the paper's workloads.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

VIEW = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64, np.dtype(np.float32): np.float32}


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(VIEW[a.dtype])).cuda()


def to_host(t, dtype):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().view(dtype)


def kt_of(dtype, mms):
    return {np.dtype(np.uint32): mms.KEY_U32, np.dtype(np.uint64): mms.KEY_U64,
            np.dtype(np.float32): mms.KEY_F32}[np.dtype(dtype)]


def assert_bits_equal(got, want):
    assert got.shape == want.shape and got.dtype.itemsize == want.dtype.itemsize
    ut = np.uint64 if got.dtype.itemsize == 8 else np.uint32
    gb, wb = got.view(ut), want.view(ut)
    if not np.array_equal(gb, wb):
        bad = np.flatnonzero(gb != wb)
        raise AssertionError(f"{bad.size} mismatches, first at {bad[0]}: got {gb[bad[0]]:#x} want {wb[bad[0]]:#x}")


def gpu_sort(mms, keys, fanout=0):
    t = to_dev(keys)
    mms.sort_keys(t, fanout=fanout, kt=kt_of(keys.dtype, mms))
    return to_host(t, keys.dtype)


# ---- base case (Sec. 4.3) --------------------------------------------------------

@pytest.mark.parametrize("dtype,kind", [(np.uint32, "uniform"), (np.uint64, "uniform"),
                                        (np.uint32, "dups"), (np.float32, "normal_f32")])
def test_tile_sort_matches_oracle(gpu, dtype, kind):
    S = gpu.tile_items(kt_of(dtype, gpu))
    n = 5 * S + 1234
    if kind == "uniform":
        keys = synth.uniform(n, 11, dtype)
    elif kind == "dups":
        keys = synth.uniform(n, 12, dtype) % dtype(7)
    else:
        keys = synth.normal_f32(n, 13)
    t = to_dev(keys)
    out = to_dev(np.zeros_like(keys))
    gpu.tile_sort(t, out, kt=kt_of(dtype, gpu))
    want, _ = oracle.tile_sort(keys, S)
    assert_bits_equal(to_host(out, keys.dtype), want)


def test_tile_sort_in_place_and_tiny(gpu):
    for n in [1, 2, 31, 32, 33, 1023, 1024, 1025, 8191, 8192, 8193]:
        keys = synth.uniform(n, n, np.uint32)
        t = to_dev(keys)
        gpu.tile_sort(t, kt=gpu.KEY_U32)
        want, _ = oracle.tile_sort(keys, 8192)
        assert_bits_equal(to_host(t, np.uint32), want)


def test_f32_total_order_specials(gpu):
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "f32_total_order.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(int(line.split()[0], 16))
    want = np.array(rows, dtype=np.uint32)
    rng = np.random.default_rng(5)
    keys = np.concatenate([rng.permutation(want) for _ in range(700)]).view(np.float32)
    got = gpu_sort(gpu, keys)
    ref, _ = oracle.sort(keys)
    assert_bits_equal(got, ref)
    assert np.array_equal(got.view(np.uint32), np.repeat(want, 700))


# ---- splitter (Sec. 4.1) -----------------------------------------------------------

def sorted_runs(keys, run_len):
    out, _ = oracle.tile_sort(keys, run_len)
    return out


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("K,runs_mult,mod", [(2, 1, 0), (4, 1, 50), (3, 1, 0), (8, 2, 0),
                                             (32, 1, 3), (16, 1, 1)])
def test_splitter_matches_brute_force(gpu, dtype, K, runs_mult, mod):
    kt = kt_of(dtype, gpu)
    S = gpu.tile_items(kt)
    run_len = S * runs_mult
    n = run_len * (2 * K + 1) + 3 * S // 2 + 5         # two full groups and a ragged third
    keys = synth.uniform(n, K * 7 + runs_mult, dtype)
    if mod:
        keys = keys % dtype(mod)
    pre = sorted_runs(keys, run_len)
    table = gpu.splitter(to_dev(pre), run_len, K, kt=kt)
    got = table.cpu().numpy()
    want = oracle.splitter_table(pre, run_len, K, S)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_splitter_adversarial_interleaved(gpu):
    S = 8192
    K = 8
    keys = synth.interleaved(S * K * 3, K, 32, np.uint32)
    pre = sorted_runs(keys, S)
    got = gpu.splitter(to_dev(pre), S, K, kt=gpu.KEY_U32).cpu().numpy()
    assert np.array_equal(got, oracle.splitter_table(pre, S, K, S))


# ---- merge pass (Sec. 4.2), fed the oracle's pivot table ----------------------------

@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("K,runs_mult,mod", [(2, 1, 0), (4, 2, 0), (8, 1, 5), (32, 1, 0), (5, 1, 0)])
def test_merge_pass_matches_oracle(gpu, dtype, K, runs_mult, mod):
    import torch
    kt = kt_of(dtype, gpu)
    S = gpu.tile_items(kt)
    run_len = S * runs_mult
    n = run_len * (2 * K + 1) + S + 77
    keys = synth.uniform(n, 3 + K, dtype)
    if mod:
        keys = keys % dtype(mod)
    pre = sorted_runs(keys, run_len)
    table = torch.from_numpy(oracle.splitter_table(pre, run_len, K, S)).cuda()
    out = to_dev(np.zeros_like(pre))
    ws = torch.zeros(gpu.workspace_bytes(kt, 16), dtype=torch.uint8, device="cuda")
    gpu.merge_pass(to_dev(pre), out, run_len, K, table, workspace=ws, kt=kt)
    want, _ = oracle.merge_pass(pre, run_len, K)
    assert_bits_equal(to_host(out, dtype), want)
    gpu.workspace_status(ws)


# ---- whole sort --------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 3, 100, 8191, 8192, 8193, 3 * 8192 * 5 + 777, 1 << 20])
def test_sort_u32_sizes(gpu, n):
    keys = synth.uniform(n, n + 1, np.uint32)
    want, _ = oracle.sort(keys)
    assert_bits_equal(gpu_sort(gpu, keys), want)


@pytest.mark.parametrize("fanout", [2, 3, 4, 8, 16, 32, 0])
def test_sort_u32_fanouts(gpu, fanout):
    n = 8192 * 70 + 4321
    keys = synth.uniform(n, fanout + 100, np.uint32)
    want, _ = oracle.sort(keys)
    assert_bits_equal(gpu_sort(gpu, keys, fanout), want)


@pytest.mark.parametrize("kind", ["sorted", "reversed", "equal", "two_values", "sortedness",
                                  "interleaved", "permutation"])
def test_sort_u32_structured(gpu, kind):
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
    for fanout in (4, 0):
        assert_bits_equal(gpu_sort(gpu, keys, fanout), want)


@pytest.mark.parametrize("n", [2, 4097, 4096 * 37 + 11])
def test_sort_u64(gpu, n):
    keys = synth.uniform(n, 21, np.uint64)
    keys[1::2] = keys[0::2][: keys[1::2].size]          # every key at least twice
    want, _ = oracle.sort(keys)
    assert_bits_equal(gpu_sort(gpu, keys), want)
    assert_bits_equal(gpu_sort(gpu, keys, 4), want)


def test_sort_u64_high_word(gpu):
    n = 4096 * 9 + 3
    lo = np.uint64(12345)
    keys = (synth.uniform(n, 5, np.uint32).astype(np.uint64) << np.uint64(32)) | lo
    want, _ = oracle.sort(keys)
    assert_bits_equal(gpu_sort(gpu, keys, 2), want)


@pytest.mark.parametrize("n", [5, 8192 * 11 + 5])
def test_sort_f32(gpu, n):
    keys = synth.normal_f32(n, 8)
    want, _ = oracle.sort(keys)
    assert_bits_equal(gpu_sort(gpu, keys), want)
    assert_bits_equal(gpu_sort(gpu, keys, 2), want)


def test_workspace_reuse_and_status(gpu):
    import torch
    n = 8192 * 20 + 17
    ws = torch.empty(gpu.workspace_bytes(gpu.KEY_U32, n), dtype=torch.uint8, device="cuda")
    ws.zero_()
    for seed in range(3):
        keys = synth.uniform(n, seed, np.uint32)
        t = to_dev(keys)
        gpu.sort_keys(t, workspace=ws, kt=gpu.KEY_U32)
        want, _ = oracle.sort(keys)
        assert_bits_equal(to_host(t, np.uint32), want)
    gpu.workspace_status(ws)


def test_workspace_too_small_is_rejected(gpu):
    import torch
    n = 8192 * 4
    ws = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    t = to_dev(synth.uniform(n, 1, np.uint32))
    with pytest.raises(gpu.MMSError):
        gpu.sort_keys(t, workspace=ws, kt=gpu.KEY_U32)


# ---- key-value sort (stable) -------------------------------------------------------

def gpu_sort_pairs(mms, keys, vals, fanout=0, tile=0):
    kt = kt_of(keys.dtype, mms)
    tk, tv = to_dev(keys), to_dev(vals)
    mms.sort_pairs(tk, tv, fanout=fanout, kt=kt, tile_items=tile)
    return to_host(tk, keys.dtype), to_host(tv, np.uint32)


@pytest.mark.parametrize("n", [2, 3, 1000, 4096, 4097, 4096 * 23 + 5, 1 << 20])
def test_pairs_u32_index_payload_stable(gpu, n):
    keys = synth.uniform(n, n, np.uint32) % np.uint32(max(2, n // 7))   # many equal keys
    vals = synth.index_payload(n)
    wk, wv = oracle.sort(keys, vals)
    gk, gv = gpu_sort_pairs(gpu, keys, vals)
    assert_bits_equal(gk, wk)
    assert_bits_equal(gv, wv)


@pytest.mark.parametrize("fanout,tile", [(2, 0), (4, 2048), (8, 4096), (32, 0)])
def test_pairs_u32_random_payload(gpu, fanout, tile):
    n = 4096 * 41 + 333
    keys = synth.uniform(n, 17, np.uint32) % np.uint32(5000)
    vals = synth.uniform(n, 18, np.uint32)
    wk, wv = oracle.sort(keys, vals)
    gk, gv = gpu_sort_pairs(gpu, keys, vals, fanout, tile)
    assert_bits_equal(gk, wk)
    assert_bits_equal(gv, wv)


def test_pairs_f32_specials(gpu):
    n = 4096 * 9 + 71
    keys = synth.normal_f32(n, 19)
    keys[::5] = keys[1::5][: keys[::5].size]              # repeated floats, NaNs and -0.0 included
    vals = synth.index_payload(n)
    wk, wv = oracle.sort(keys, vals)
    gk, gv = gpu_sort_pairs(gpu, keys, vals)
    assert_bits_equal(gk, wk)
    assert_bits_equal(gv, wv)


@pytest.mark.parametrize("n,kind", [(2, "uniform"), (777, "uniform"), (4096 * 31 + 9, "hi_dups"),
                                    (4096 * 31 + 9, "lo_dups"), (1 << 20, "both_dups")])
def test_pairs_u64_two_passes(gpu, n, kind):
    """8-byte keys with values: two stable 4-byte passes (low half, then high
    half); duplicates confined to one half or both exercise the tie rules."""
    keys = synth.uniform(n, 41 + n, np.uint64)
    if kind == "hi_dups":       # high halves from 5 values: ties decided by the low halves
        keys = (keys & np.uint64(0xFFFFFFFF)) | ((keys >> np.uint64(32)) % np.uint64(5) << np.uint64(32))
    elif kind == "lo_dups":     # low halves from 3 values
        keys = (keys & np.uint64(0xFFFFFFFF00000000)) | (keys % np.uint64(3))
    elif kind == "both_dups":   # whole keys repeat: stability decides the values' order
        keys = ((keys % np.uint64(7)) << np.uint64(32)) | (keys % np.uint64(3))
    vals = synth.uniform(n, 42 + n, np.uint32)
    wk, wv = oracle.sort(keys, vals)
    gk, gv = gpu_sort_pairs(gpu, keys, vals)
    assert_bits_equal(gk, wk)
    assert_bits_equal(gv, wv)


@pytest.mark.slow
def test_full_size_pairs_permutation_1e8(gpu):
    """10^8 uint32 keys, permutation of 0..N-1, index payload: keys sort to iota
    and the payload becomes the inverse permutation (closed form)."""
    import torch
    n = 10**8
    keys = synth.permutation(n, 5)
    tk = to_dev(keys)
    tv = torch.arange(n, dtype=torch.int32, device="cuda")
    gpu.sort_pairs(tk, tv, kt=gpu.KEY_U32)
    iota = torch.arange(n, dtype=torch.int64, device="cuda")
    assert torch.equal(tk.to(torch.int64) & 0xFFFFFFFF, iota)
    src = torch.from_numpy(keys.view(np.int32)).cuda().to(torch.int64) & 0xFFFFFFFF
    inv = torch.empty(n, dtype=torch.int64, device="cuda")
    inv[src] = iota
    assert torch.equal(tv.to(torch.int64), inv)


# ---- full-size configurations: closed forms ----------------------------------------

@pytest.mark.slow
def test_full_size_permutation_1e8_u32(gpu):
    """10^8 uint32, fully random permutation of 0..N-1: must sort to iota."""
    import torch
    n = 10**8
    keys = synth.permutation(n, 1)
    t = to_dev(keys)
    gpu.sort_keys(t, kt=gpu.KEY_U32)
    iota = torch.arange(n, dtype=torch.int64, device="cuda")
    assert torch.equal(t.to(torch.int64) & 0xFFFFFFFF, iota)


@pytest.mark.slow
@pytest.mark.parametrize("r", [0, 10**3, 10**5])
def test_full_size_sortedness_1e8_u32(gpu, r):
    import torch
    n = 10**8
    keys = synth.sortedness(n, r, 2)
    t = to_dev(keys)
    gpu.sort_keys(t, kt=gpu.KEY_U32)
    iota = torch.arange(n, dtype=torch.int64, device="cuda")
    assert torch.equal(t.to(torch.int64) & 0xFFFFFFFF, iota)


@pytest.mark.slow
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_full_size_interleaved_2p28(gpu, dtype):
    """2^28 keys in 8 runs interleaved at stride 32: dense unique values -> iota."""
    import torch
    n = 1 << 28
    keys = synth.interleaved(n, 8, 32, dtype)
    t = to_dev(keys)
    gpu.sort_keys(t, kt=kt_of(dtype, gpu))
    iota = torch.arange(n, dtype=torch.int64, device="cuda")
    if np.dtype(dtype) == np.uint64:
        want = (iota << 32) | iota
        assert torch.equal(t, want)
    else:
        assert torch.equal(t.to(torch.int64) & 0xFFFFFFFF, iota)


@pytest.mark.parametrize("dtype,tile", [(np.uint32, 4096), (np.uint64, 2048), (np.float32, 4096)])
@pytest.mark.parametrize("fanout", [0, 2, 5, 8])
def test_sort_other_tile_width(gpu, dtype, tile, fanout):
    n = tile * 37 + 123
    keys = synth.normal_f32(n, 3) if np.dtype(dtype) == np.float32 else synth.uniform(n, 4, dtype) % dtype(1000)
    want, _ = oracle.sort(keys)
    t = to_dev(keys)
    gpu.sort_keys(t, fanout=fanout, kt=kt_of(dtype, gpu), tile_items=tile)
    assert_bits_equal(to_host(t, keys.dtype), want)


def test_bad_tile_width_is_rejected(gpu):
    t = to_dev(synth.uniform(10000, 1, np.uint32))
    with pytest.raises(gpu.MMSError):
        gpu.sort_keys(t, kt=gpu.KEY_U32, tile_items=2048)


@pytest.mark.parametrize("fanout,merge_tile", [(4, 7168), (4, 4096), (8, 5120), (2, 6144), (3, 7168), (4, 8192)])
def test_sort_merge_tile_sizes(gpu, fanout, merge_tile):
    """Merge output tiles smaller than the base-case run (groups then end in a
    short tile): any multiple of 1024 gives the same bits."""
    n = 8192 * 37 + 5000
    keys = synth.uniform(n, fanout * 31 + merge_tile, np.uint32) % np.uint32(50000)
    want, _ = oracle.sort(keys)
    t = to_dev(keys)
    gpu.sort_keys(t, fanout=fanout, kt=gpu.KEY_U32, merge_tile_items=merge_tile)
    assert_bits_equal(to_host(t, np.uint32), want)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64, np.float32])
@pytest.mark.parametrize("tiles,tail,fanout", [(3, 7, 8), (5, 100, 4), (9, 0, 8), (17, 1, 16),
                                               (33, 4095, 32), (6, 0, 4)])
def test_sort_groups_with_fewer_runs_than_k(gpu, dtype, tiles, tail, fanout):
    """Last groups holding fewer runs than K (down to one run, ragged or not):
    the merge tree spans the runs the group holds, with the same bits."""
    T = gpu.tile_items(gpu.KEY_U64 if dtype == np.uint64 else gpu.KEY_U32)
    n = tiles * T + tail
    if dtype == np.float32:
        keys = synth.normal_f32(n, 11 * tiles + fanout)
    else:
        keys = synth.uniform(n, 13 * tiles + fanout, dtype)
    want, _ = oracle.sort(keys)
    assert_bits_equal(gpu_sort(gpu, keys, fanout), want)
