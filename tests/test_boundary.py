"""The C ABI's contract beyond the sorted bits (GPU): arrays aligned only to
their element size, the status word of a caller's workspace cleared by every
call, the status of sorts whose workspace the library allocates, and the
device-side time-out path (a bounded wait that runs out returns
MMS_ERR_TIMEOUT through the status word, with nothing left in flight, and the
next sort on the same workspace is exact again).  Every result is compared bit
for bit with the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

VIEW = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64, np.dtype(np.float32): np.float32}


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(VIEW[a.dtype])).cuda()


def bits(t, dtype):
    import torch
    torch.cuda.synchronize()
    a = t.cpu().numpy().view(dtype)
    return a.view(np.uint64 if a.dtype.itemsize == 8 else np.uint32)


def kt_of(dtype, mms):
    return {np.dtype(np.uint32): mms.KEY_U32, np.dtype(np.uint64): mms.KEY_U64,
            np.dtype(np.float32): mms.KEY_F32}[np.dtype(dtype)]


@pytest.mark.parametrize("dtype,off", [(np.uint32, 1), (np.uint32, 3), (np.float32, 2), (np.uint64, 1)])
@pytest.mark.parametrize("fanout", [0, 3, 8])
def test_sort_keys_on_a_slice_off_the_16_byte_grid(gpu, dtype, off, fanout):
    """A tensor slice at an element offset (4 or 8 bytes off the 16-byte grid)
    sorts to the oracle's result and leaves the items around it untouched."""
    T = gpu.tile_items(kt_of(dtype, gpu))
    n = 9 * T + 777
    keys = synth.normal_f32(n + off + 5, 3) if np.dtype(dtype) == np.float32 else \
        synth.uniform(n + off + 5, 4, dtype) % dtype(100000)
    buf = to_dev(keys)
    view = buf[off:off + n]
    assert view.data_ptr() % 16 != 0
    gpu.sort_keys(view, fanout=fanout, kt=kt_of(dtype, gpu))
    got = bits(buf, dtype)
    want, _ = oracle.sort(keys[off:off + n])
    raw = keys.view(got.dtype)
    assert np.array_equal(got[off:off + n], want.view(got.dtype))
    assert np.array_equal(got[:off], raw[:off]) and np.array_equal(got[off + n:], raw[off + n:])


@pytest.mark.parametrize("dtype", [np.uint32, np.float32, np.uint64])
def test_sort_pairs_on_slices_off_the_16_byte_grid(gpu, dtype):
    n = 4096 * 13 + 91
    keys = synth.normal_f32(n + 8, 9) if np.dtype(dtype) == np.float32 else \
        synth.uniform(n + 8, 10, dtype) % dtype(3000)
    vals = synth.uniform(n + 8, 11, np.uint32)
    kb, vb = to_dev(keys), to_dev(vals)
    kv, vv = kb[1:1 + n], vb[3:3 + n]
    gpu.sort_pairs(kv, vv, kt=kt_of(dtype, gpu))
    wk, wv = oracle.sort(keys[1:1 + n], vals[3:3 + n])
    gk, gv = bits(kb, dtype), bits(vb, np.uint32)
    assert np.array_equal(gk[1:1 + n], wk.view(gk.dtype))
    assert np.array_equal(gv[3:3 + n], wv)


def test_tile_sort_on_slices_off_the_16_byte_grid(gpu):
    import torch
    n = 8192 * 4 + 100
    keys = synth.uniform(n + 4, 12, np.uint32)
    src = to_dev(keys)
    dst = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
    gpu.tile_sort(src[1:1 + n], dst[3:3 + n], kt=gpu.KEY_U32)
    want, _ = oracle.tile_sort(keys[1:1 + n], 8192)
    assert np.array_equal(bits(dst, np.uint32)[3:3 + n], want)


def test_workspace_with_garbage_status_word_sorts_and_reports_ok(gpu):
    """Every call clears its workspace's status word first: a workspace fresh
    from an allocator (here all bits set) neither fails the sort nor reports a
    stale error."""
    import torch
    n = 8192 * 30 + 5
    keys = synth.uniform(n, 21, np.uint32)
    ws = torch.full((gpu.workspace_bytes(gpu.KEY_U32, n),), 0xFF, dtype=torch.uint8, device="cuda")
    t = to_dev(keys)
    gpu.sort_keys(t, workspace=ws, kt=gpu.KEY_U32)
    gpu.workspace_status(ws)
    assert np.array_equal(bits(t, np.uint32), oracle.sort(keys)[0])
    wsp = torch.full((gpu.workspace_bytes(gpu.KEY_U32, n, True),), 0xFF, dtype=torch.uint8, device="cuda")
    t = to_dev(keys)
    v = to_dev(synth.index_payload(n))
    gpu.sort_pairs(t, v, workspace=wsp, kt=gpu.KEY_U32)
    gpu.workspace_status(wsp)
    wk, wv = oracle.sort(keys, synth.index_payload(n))
    assert np.array_equal(bits(t, np.uint32), wk) and np.array_equal(bits(v, np.uint32), wv)


def test_library_allocated_workspace_does_not_wait_and_reports_ok(gpu):
    n = 8192 * 40 + 3
    keys = synth.uniform(n, 22, np.uint32)
    t = to_dev(keys)
    gpu.sort_keys(t, kt=gpu.KEY_U32)           # no workspace: allocated stream-ordered
    gpu.stream_status()
    assert np.array_equal(bits(t, np.uint32), oracle.sort(keys)[0])


def test_device_timeout_is_reported_and_the_workspace_recovers(gpu):
    """The test hook makes every merge CTA's extra bounded wait run out after
    its real copies have landed: the sort returns at once, the status word
    reads MMS_ERR_TIMEOUT, and the next plain sort on the same workspace is
    bit-exact with a clean status."""
    import torch
    n = 8192 * 24 + 999
    keys = synth.uniform(n, 23, np.uint32)
    ws = torch.zeros(gpu.workspace_bytes(gpu.KEY_U32, n), dtype=torch.uint8, device="cuda")
    t = to_dev(keys)
    gpu.sort_keys(t, fanout=4, workspace=ws, kt=gpu.KEY_U32, test_flags=gpu.TEST_STAGING_TIMEOUT)
    with pytest.raises(gpu.MMSError) as e:
        gpu.workspace_status(ws)
    assert e.value.status == 5                 # MMS_ERR_TIMEOUT
    gpu.workspace_status(ws)                   # read and cleared
    t = to_dev(keys)
    gpu.sort_keys(t, fanout=4, workspace=ws, kt=gpu.KEY_U32)
    gpu.workspace_status(ws)
    assert np.array_equal(bits(t, np.uint32), oracle.sort(keys)[0])


def test_device_timeout_without_a_workspace_reaches_stream_status(gpu):
    n = 8192 * 9 + 1
    keys = synth.uniform(n, 24, np.uint32)
    t = to_dev(keys)
    gpu.sort_keys(t, kt=gpu.KEY_U32, test_flags=gpu.TEST_STAGING_TIMEOUT)
    with pytest.raises(gpu.MMSError) as e:
        gpu.stream_status()
    assert e.value.status == 5
    gpu.stream_status()                        # cleared by the read
    t = to_dev(keys)
    gpu.sort_keys(t, kt=gpu.KEY_U32)
    gpu.stream_status()
    assert np.array_equal(bits(t, np.uint32), oracle.sort(keys)[0])
