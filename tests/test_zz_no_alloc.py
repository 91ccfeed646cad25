"""The entry point that allocates nothing (mms_sort_keys_noalloc), for callers
that cannot allocate device memory while they run: called through the C ABI,
its output must equal mms_sort_keys's bit for bit, on two calls in a row (the
fixed scratch keeps the previous call's contents, which must not leak into the
next result).  Collected last so that a failure here stops a run only after
every other test has run; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

VIEW = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64, np.dtype(np.float32): np.float32}


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(VIEW[a.dtype])).cuda()


def _bits(t, dtype):
    import torch
    torch.cuda.synchronize()
    out = t.cpu().numpy().view(dtype)
    return out.view(np.uint64 if out.dtype.itemsize == 8 else np.uint32)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64, np.float32])
def test_noalloc_matches_sort_keys_on_two_calls(gpu, dtype):
    import torch
    L = gpu.load()
    kt = {np.dtype(np.uint32): gpu.KEY_U32, np.dtype(np.uint64): gpu.KEY_U64,
          np.dtype(np.float32): gpu.KEY_F32}[np.dtype(dtype)]
    cap = gpu.NOALLOC_MAX_KEYS[kt]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # first call at the maximum size, second call smaller with other data
    for call, n in enumerate([cap, cap // 3 + 7]):
        if np.dtype(dtype) == np.float32:
            keys = synth.normal_f32(n, 40 + call)
        else:
            keys = synth.uniform(n, 40 + call, dtype) % dtype(1 << 20)
        ref = _dev(keys)
        gpu.sort_keys(ref, kt=kt)                       # the existing entry point
        got = _dev(keys)
        status = L.mms_sort_keys_noalloc(kt, ctypes.c_void_p(got.data_ptr()), n, stream)
        assert status == 0
        assert L.mms_noalloc_status(stream) == 0        # no device-side error recorded
        assert np.array_equal(_bits(got, dtype), _bits(ref, dtype)), f"call {call}: outputs differ"


def test_noalloc_rejects_more_than_its_maximum(gpu):
    L = gpu.load()
    t = _dev(np.zeros(16, dtype=np.uint32))
    too_many = gpu.NOALLOC_MAX_KEYS[gpu.KEY_U32] + 1
    # beyond the maximum: rejected before any work is queued (the buffer is not touched)
    assert L.mms_sort_keys_noalloc(gpu.KEY_U32, ctypes.c_void_p(t.data_ptr()), too_many, None) == 1
    with pytest.raises(ValueError):
        import torch
        gpu.sort_keys_noalloc(torch.empty(too_many, dtype=torch.int32, device="cuda"), kt=gpu.KEY_U32)
