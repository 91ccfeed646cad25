"""Batched (segmented) sorting through the C ABI against the CPU oracle.

Every segment must equal the oracle's stable sort of that segment alone,
bit for bit, whatever the mix of sizes, key types, fanout table or buffer
parity; a CUDA-graph replay must equal a direct call; and a segment sorted
in a batch must equal the same array sorted alone by the whole-array path.
Inputs: seeded synthetic batches whose sizes are log-uniform, like the
batched workload, plus hand-picked edge sizes around the tile size.
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


def bits(a):
    return a.view(np.uint64 if a.dtype.itemsize == 8 else np.uint32)


def kt_of(dtype, mms):
    return {np.dtype(np.uint32): mms.KEY_U32, np.dtype(np.uint64): mms.KEY_U64,
            np.dtype(np.float32): mms.KEY_F32}[np.dtype(dtype)]


def make_keys(n, seed, dtype):
    if np.dtype(dtype) == np.float32:
        return synth.normal_f32(n, seed)
    return synth.uniform(n, seed, dtype)


EDGE = [0, 1, 2, 3, 5, 1023, 1024, 4095, 4096, 4097, 8191, 8192, 8193, 3 * 8192 + 17,
        40 * 8192 + 5, 0, 7]


def batch(seed, dtype, count=60, hi=1 << 18):
    sizes = np.concatenate([synth.segment_sizes(count, 1, hi, seed), np.array(EDGE, dtype=np.int64)])
    np.random.default_rng(seed).shuffle(sizes)
    off = synth.offsets_of(sizes)
    return make_keys(int(off[-1]), seed + 1, dtype), off


def run(gpu, keys, off, values=None, **kw):
    import torch
    k = to_dev(keys)
    v = None if values is None else to_dev(values)
    o = torch.from_numpy(off).cuda()
    kt = kt_of(keys.dtype, gpu)
    ws = torch.zeros(gpu.segmented_workspace_bytes(kt, keys.size, off.size - 1, values is not None,
                                                   kw.get("class_fanout"), kw.get("max_segment_items", 0),
                                                   kw.get("tile_items", 0)), dtype=torch.uint8, device="cuda")
    gpu.segmented_sort(k, o, v, workspace=ws, kt=kt, **kw)
    gpu.workspace_status(ws)
    return to_host(k, keys.dtype), (None if v is None else to_host(v, np.uint32))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64, np.float32])
def test_segmented_keys_match_oracle(gpu, dtype):
    keys, off = batch(11, dtype)
    got, _ = run(gpu, keys, off)
    want, _ = oracle.segmented_sort(keys, off)
    assert np.array_equal(bits(got), bits(want))


@pytest.mark.parametrize("dtype", [np.uint32, np.float32, np.uint64])
def test_segmented_pairs_match_oracle(gpu, dtype):
    keys, off = batch(23, dtype)
    keys[::3] = keys[1::3][: keys[::3].size] if keys.size > 2 else keys[::3]     # many equal keys
    if np.dtype(dtype) == np.uint64:        # and equal high halves with distinct low halves
        keys[1::4] = (keys[1::4] & np.uint64(0xFFFFFFFF)) | np.uint64(0x1234 << 32)
    vals = synth.index_payload(keys.size)
    got_k, got_v = run(gpu, keys, off, vals)
    want_k, want_v = oracle.segmented_sort(keys, off, vals)
    assert np.array_equal(bits(got_k), bits(want_k))
    assert np.array_equal(got_v, want_v)


@pytest.mark.parametrize("table", [{c: 2 for c in range(33)}, {c: 3 for c in range(33)},
                                   {c: (32 if c > 15 else 8) for c in range(33)}])
def test_segmented_fanout_tables(gpu, table):
    keys, off = batch(31, np.uint32, count=30)
    got, _ = run(gpu, keys, off, class_fanout=table)
    want, _ = oracle.segmented_sort(keys, off)
    assert np.array_equal(got, want)


def test_segmented_small_tiles_and_max_hint(gpu):
    keys, off = batch(41, np.uint32, count=40, hi=1 << 16)
    mx = int(np.max(np.diff(off)))
    got, _ = run(gpu, keys, off, tile_items=4096, max_segment_items=mx)
    want, _ = oracle.segmented_sort(keys, off)
    assert np.array_equal(got, want)


def test_segmented_heavy_duplicates_and_sortedness(gpu):
    sizes = np.array([70000, 3, 130000, 8192 * 4, 9000, 1], dtype=np.int64)
    off = synth.offsets_of(sizes)
    parts = [synth.uniform(70000, 1) % np.uint32(3), np.array([5, 5, 1], np.uint32),
             synth.sortedness(130000, 1000, 2), np.arange(8192 * 4, dtype=np.uint32)[::-1].copy(),
             np.full(9000, 0xFFFFFFFF, np.uint32), np.array([0], np.uint32)]
    keys = np.concatenate(parts)
    got, _ = run(gpu, keys, off)
    want, _ = oracle.segmented_sort(keys, off)
    assert np.array_equal(got, want)


def test_segment_alone_equals_segment_in_batch(gpu):
    """Each result is the same sorted alone (whole-array path) and in the mix."""
    keys, off = batch(53, np.uint32, count=20)
    got, _ = run(gpu, keys, off)
    for s in range(off.size - 1):
        a, b = int(off[s]), int(off[s + 1])
        if b - a < 2 or (s % 3):
            continue
        t = to_dev(keys[a:b].copy())
        gpu.sort_keys(t, kt=gpu.KEY_U32)
        assert np.array_equal(to_host(t, np.uint32), got[a:b]), f"segment {s} differs"


def test_segmented_graph_replay_equals_direct(gpu):
    import torch
    keys, off = batch(61, np.uint32, count=40)
    vals = synth.index_payload(keys.size)
    want_k, want_v = oracle.segmented_sort(keys, off, vals)
    k = to_dev(keys)
    v = to_dev(vals)
    o = torch.from_numpy(off).cuda()
    src_k, src_v = k.clone(), v.clone()
    g = gpu.SegmentedGraph(k, o, v, kt=gpu.KEY_U32)
    assert torch.equal(k, src_k)                     # creating the graph queues no work
    for _ in range(2):
        k.copy_(src_k)
        v.copy_(src_v)
        g.launch()
        assert np.array_equal(to_host(k, np.uint32), want_k)
        assert np.array_equal(to_host(v, np.uint32), want_v)
    gpu.workspace_status(g.workspace)
    g.close()


def test_segmented_single_segment_equals_whole_sort(gpu):
    n = 8192 * 50 + 3
    keys = synth.permutation(n, 7)
    got, _ = run(gpu, keys, np.array([0, n], dtype=np.int64))
    assert np.array_equal(got, np.arange(n, dtype=np.uint32))


def test_segmented_bad_offsets_flag_the_status_word(gpu):
    import torch
    keys = synth.uniform(300, 3)
    k = to_dev(keys)
    o = torch.tensor([0, 100, 200], dtype=torch.int64, device="cuda")   # does not end at 300
    ws = torch.zeros(gpu.segmented_workspace_bytes(gpu.KEY_U32, 300, 2), dtype=torch.uint8, device="cuda")
    import ctypes
    L = gpu.load()
    opts = gpu._seg_opts()
    st = L.mms_segmented_sort(gpu.KEY_U32, gpu._ptr(k), None, gpu._ptr(o), 2, 300, gpu._ptr(ws), ws.numel(),
                              gpu._stream_handle(None), ctypes.byref(opts))
    assert st == 0
    with pytest.raises(gpu.MMSError):
        gpu.workspace_status(ws)
