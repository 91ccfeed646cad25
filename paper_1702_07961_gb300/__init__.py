"""GB300-native GPU Multiway Mergesort (Casanova, Iacono, Karsin, Sitchinava,
Weichert, "An Efficient Multiway Mergesort for GPU Architectures").

A thin Python binding over ``libmms.so`` (C ABI in ``include/mms.h``): it only
marshals arguments.  Every step of the sort runs in the library's CUDA kernels;
PyTorch provides device memory and streams.  There is no CPU fallback: when the
library has not been built, :func:`load` raises.

Keys: ``torch.uint32``/``torch.int32`` tensors are sorted as unsigned 32-bit
integers, ``torch.uint64``/``torch.int64`` as unsigned 64-bit integers,
``torch.float32`` by IEEE-754 totalOrder on bit patterns.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = ["load", "KEY_U32", "KEY_U64", "KEY_F32", "key_type_of", "sort_keys", "sort_pairs",
           "workspace_bytes", "tile_items", "base_run_items", "plan", "tile_sort", "splitter_rows", "splitter",
           "merge_pass", "workspace_status", "stream_status", "MMSError", "sort_keys_noalloc",
           "noalloc_status", "NOALLOC_MAX_KEYS", "TEST_STAGING_TIMEOUT",
           "segmented_workspace_bytes", "segmented_rounds", "segmented_sort", "SegmentedGraph"]

KEY_U32, KEY_U64, KEY_F32 = 0, 1, 2
_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libmms.so")

_lock = threading.Lock()
_lib = None


class MMSError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"mms status {status}: {detail}")
        self.status = status
        self.detail = detail


class _Options(ctypes.Structure):
    _fields_ = [("fanout", ctypes.c_int), ("num_events", ctypes.c_int),
                ("events", ctypes.POINTER(ctypes.c_void_p)), ("tile_items", ctypes.c_int),
                ("merge_tile_items", ctypes.c_int), ("test_flags", ctypes.c_int),
                ("merge_variant", ctypes.c_int), ("base_items", ctypes.c_int)]


# mms_options.test_flags: a test hook that makes every merge CTA's extra
# bounded wait run out (MMS_TEST_STAGING_TIMEOUT).
TEST_STAGING_TIMEOUT = 1

# mms_options.merge_variant: the CTA merge tree (default), the heap-free
# partition variant or the pipelined variant (MMS_MERGE_TREE,
# MMS_MERGE_PARTITION, MMS_MERGE_PIPELINED).
MERGE_TREE = 0
MERGE_PARTITION = 1
MERGE_PIPELINED = 2


class _SegOptions(ctypes.Structure):
    _fields_ = [("class_fanout", ctypes.c_int * 33), ("max_segment_items", ctypes.c_size_t),
                ("tile_items", ctypes.c_int), ("num_events", ctypes.c_int),
                ("events", ctypes.POINTER(ctypes.c_void_p)), ("reserved", ctypes.c_int * 4)]


def load() -> ctypes.CDLL:
    """Loads libmms.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(SO_PATH):
            raise FileNotFoundError(
                f"{SO_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(SO_PATH)
        vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        L.mms_sort_workspace_bytes.argtypes = [i32, sz, i32]
        L.mms_sort_workspace_bytes.restype = sz
        L.mms_sort_keys.argtypes = [i32, vp, sz, vp, sz, vp]
        L.mms_sort_keys.restype = i32
        L.mms_sort_keys_ex.argtypes = [i32, vp, sz, vp, sz, vp, ctypes.POINTER(_Options)]
        L.mms_sort_keys_ex.restype = i32
        L.mms_sort_pairs.argtypes = [i32, vp, vp, sz, vp, sz, vp]
        L.mms_sort_pairs.restype = i32
        L.mms_sort_pairs_ex.argtypes = [i32, vp, vp, sz, vp, sz, vp, ctypes.POINTER(_Options)]
        L.mms_sort_pairs_ex.restype = i32
        L.mms_workspace_status.argtypes = [vp, sz, vp]
        L.mms_workspace_status.restype = i32
        L.mms_stream_status.argtypes = [vp]
        L.mms_stream_status.restype = i32
        L.mms_noalloc_status.argtypes = [vp]
        L.mms_noalloc_status.restype = i32
        L.mms_tile_items.argtypes = [i32]
        L.mms_tile_items.restype = sz
        L.mms_base_run_items.argtypes = [i32, sz, ctypes.POINTER(_Options)]
        L.mms_base_run_items.restype = sz
        L.mms_plan.argtypes = [i32, sz, ctypes.POINTER(_Options), ctypes.POINTER(ctypes.c_int), i32]
        L.mms_plan.restype = i32
        L.mms_tile_sort.argtypes = [i32, vp, vp, sz, vp]
        L.mms_tile_sort.restype = i32
        L.mms_splitter_rows.argtypes = [i32, sz, sz, i32]
        L.mms_splitter_rows.restype = sz
        L.mms_splitter.argtypes = [i32, vp, sz, sz, i32, vp, vp]
        L.mms_splitter.restype = i32
        L.mms_merge_pass.argtypes = [i32, vp, vp, sz, sz, i32, vp, vp, sz, vp]
        L.mms_merge_pass.restype = i32
        L.mms_merge_pass_partition.argtypes = [i32, vp, vp, sz, sz, i32, vp, vp, sz, vp]
        L.mms_merge_pass_partition.restype = i32
        L.mms_merge_pass_pipelined.argtypes = [i32, vp, vp, sz, sz, i32, vp, vp, sz, vp]
        L.mms_merge_pass_pipelined.restype = i32
        L.mms_sort_keys_noalloc.argtypes = [i32, vp, sz, vp]
        L.mms_sort_keys_noalloc.restype = i32
        L.mms_segmented_workspace_bytes.argtypes = [i32, sz, sz, i32, ctypes.POINTER(_SegOptions)]
        L.mms_segmented_workspace_bytes.restype = sz
        L.mms_segmented_rounds.argtypes = [i32, sz, i32, ctypes.POINTER(_SegOptions)]
        L.mms_segmented_rounds.restype = i32
        L.mms_segmented_sort.argtypes = [i32, vp, vp, vp, sz, sz, vp, sz, vp, ctypes.POINTER(_SegOptions)]
        L.mms_segmented_sort.restype = i32
        L.mms_segmented_graph_create.argtypes = [i32, vp, vp, vp, sz, sz, vp, sz,
                                                 ctypes.POINTER(_SegOptions), ctypes.POINTER(vp)]
        L.mms_segmented_graph_create.restype = i32
        L.mms_graph_launch.argtypes = [vp, vp]
        L.mms_graph_launch.restype = i32
        L.mms_graph_destroy.argtypes = [vp]
        L.mms_graph_destroy.restype = None
        L.mms_status_string.argtypes = [i32]
        L.mms_status_string.restype = ctypes.c_char_p
        L.mms_last_error_detail.argtypes = [ctypes.c_char_p, sz]
        L.mms_last_error_detail.restype = i32
        _lib = L
        return L


def _check(status: int) -> None:
    if status != 0:
        L = load()
        buf = ctypes.create_string_buffer(256)
        L.mms_last_error_detail(buf, 256)
        raise MMSError(status, f"{L.mms_status_string(status).decode()}: {buf.value.decode()}")


def key_type_of(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return KEY_F32
    if t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32)):
        return KEY_U32
    if t.dtype in (torch.int64, getattr(torch, "uint64", torch.int64)):
        return KEY_U64
    raise TypeError(f"unsupported key dtype {t.dtype}")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _opts(fanout: int, events=None, stream=None, tile_items: int = 0, merge_tile_items: int = 0,
          test_flags: int = 0, merge_variant: int = 0, base_items: int = 0):
    o = _Options()
    o.fanout = int(fanout)
    o.base_items = int(base_items)
    o.tile_items = int(tile_items)
    o.merge_tile_items = int(merge_tile_items)
    o.test_flags = int(test_flags)
    o.merge_variant = int(merge_variant)
    if events:
        for e in events:
            if not e.cuda_event:          # torch creates the CUDA event on first record
                e.record(stream)
        arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
        o.num_events = len(events)
        o.events = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
        o._keep = arr
    return o


def workspace_bytes(kt: int, n: int, with_values: bool = False) -> int:
    return int(load().mms_sort_workspace_bytes(kt, n, int(with_values)))


def tile_items(kt: int) -> int:
    return int(load().mms_tile_items(kt))


def base_run_items(kt: int, n: int, tile_items: int = 0, base_items: int = 0) -> int:
    """Length of the sorted runs the base case of a keys-only sort of n keys produces."""
    o = _opts(0, tile_items=tile_items, base_items=base_items)
    return int(load().mms_base_run_items(kt, n, ctypes.byref(o)))


def plan(kt: int, n: int, fanout: int = 0, tile_items: int = 0, pairs: bool = False,
         base_items: int = 0):
    """Fanout of every merge round of a sort of n keys (of n pairs when `pairs`:
    the rounds of a key-value sort run on 8-byte composites)."""
    if pairs:
        kt = KEY_U64
    buf = (ctypes.c_int * 64)()
    o = _opts(fanout, tile_items=tile_items, base_items=base_items)
    r = load().mms_plan(kt, n, ctypes.byref(o), buf, 64)
    return [buf[i] for i in range(r)]


def sort_keys(keys, fanout: int = 0, workspace=None, stream=None, kt: int | None = None, events=None,
              tile_items: int = 0, merge_tile_items: int = 0, test_flags: int = 0,
              merge_variant: int = MERGE_TREE, base_items: int = 0):
    """Sorts a contiguous CUDA tensor of keys in place; returns it.

    ``events``: optional list of ``torch.cuda.Event(enable_timing=True)``; the
    library records them before the first kernel and after each kernel.
    ``test_flags``: test hooks (``TEST_STAGING_TIMEOUT``), 0 in normal use.
    ``merge_variant``: ``MERGE_TREE``, ``MERGE_PARTITION`` or ``MERGE_PIPELINED``.
    ``base_items``: length of the base case's sorted runs (0: the library's
    default, ``base_run_items``).
    """
    assert keys.is_cuda and keys.is_contiguous()
    kt = key_type_of(keys) if kt is None else kt
    n = keys.numel()
    ws_ptr, ws_len = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    o = _opts(fanout, events, stream, tile_items, merge_tile_items, test_flags, merge_variant,
              base_items)
    _check(load().mms_sort_keys_ex(kt, _ptr(keys), n, ws_ptr, ws_len, _stream_handle(stream), ctypes.byref(o)))
    return keys


def sort_pairs(keys, values, fanout: int = 0, workspace=None, stream=None, kt: int | None = None,
               events=None, tile_items: int = 0, merge_variant: int = MERGE_TREE):
    """Stable sort of (key, 32-bit value) pairs in place (4-byte keys)."""
    assert keys.is_cuda and values.is_cuda and keys.numel() == values.numel()
    assert keys.is_contiguous() and values.is_contiguous() and values.element_size() == 4
    kt = key_type_of(keys) if kt is None else kt
    ws_ptr, ws_len = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    o = _opts(fanout, events, stream, tile_items, merge_variant=merge_variant)
    _check(load().mms_sort_pairs_ex(kt, _ptr(keys), _ptr(values), keys.numel(), ws_ptr, ws_len,
                                    _stream_handle(stream), ctypes.byref(o)))
    return keys, values


def workspace_status(workspace, stream=None) -> None:
    """Raises MMSError if a kernel recorded a device-side error in the workspace."""
    _check(load().mms_workspace_status(_ptr(workspace), workspace.numel() * workspace.element_size(),
                                       _stream_handle(stream)))


def stream_status(stream=None) -> None:
    """Raises MMSError if a sort that ran without a caller workspace on the
    current device recorded a device-side error (waits for ``stream``)."""
    _check(load().mms_stream_status(_stream_handle(stream)))


def tile_sort(inp, out=None, stream=None, kt: int | None = None):
    """Base case: sorts every tile of tile_items(kt) keys of ``inp`` into ``out``."""
    kt = key_type_of(inp) if kt is None else kt
    out = inp if out is None else out
    _check(load().mms_tile_sort(kt, _ptr(inp), _ptr(out), inp.numel(), _stream_handle(stream)))
    return out


def splitter_rows(kt: int, n: int, run_len: int, K: int) -> int:
    return int(load().mms_splitter_rows(kt, n, run_len, K))


def splitter(data, run_len: int, K: int, table=None, stream=None, kt: int | None = None):
    """Pivot table of a merge round (rows x K int64 tensor on the device)."""
    import torch
    kt = key_type_of(data) if kt is None else kt
    rows = splitter_rows(kt, data.numel(), run_len, K)
    if table is None:
        table = torch.empty((rows, K), dtype=torch.int64, device=data.device)
    _check(load().mms_splitter(kt, _ptr(data), data.numel(), run_len, K, _ptr(table), _stream_handle(stream)))
    return table


def merge_pass(inp, out, run_len: int, K: int, table, workspace=None, stream=None, kt: int | None = None,
               merge_variant: int = MERGE_TREE):
    """One K-way merge round of ``inp`` into ``out`` driven by ``table``
    (``mms_merge_pass``; ``mms_merge_pass_partition`` / ``mms_merge_pass_pipelined``
    for MERGE_PARTITION / MERGE_PIPELINED)."""
    kt = key_type_of(inp) if kt is None else kt
    ws_ptr, ws_len = (None, 0) if workspace is None else (_ptr(workspace), workspace.numel() * workspace.element_size())
    L = load()
    fn = {MERGE_PARTITION: L.mms_merge_pass_partition,
          MERGE_PIPELINED: L.mms_merge_pass_pipelined}.get(merge_variant, L.mms_merge_pass)
    _check(fn(kt, _ptr(inp), _ptr(out), inp.numel(), run_len, K, _ptr(table),
              ws_ptr, ws_len, _stream_handle(stream)))
    return out


# Largest n mms_sort_keys_noalloc accepts, by key type (MMS_NOALLOC_MAX_KEYS_*).
NOALLOC_MAX_KEYS = {KEY_U32: 1 << 20, KEY_F32: 1 << 20, KEY_U64: 1 << 19}


def sort_keys_noalloc(keys, stream=None, kt: int | None = None):
    """In-place sort that allocates no device memory (fixed library scratch).

    For callers that cannot allocate device memory while they run.  Sizes up
    to NOALLOC_MAX_KEYS[kt]; calls that overlap on the GPU race, since they
    share one scratch array.
    """
    assert keys.is_cuda and keys.is_contiguous()
    kt = key_type_of(keys) if kt is None else kt
    n = keys.numel()
    if n > NOALLOC_MAX_KEYS[kt]:
        raise ValueError(f"sort_keys_noalloc takes at most {NOALLOC_MAX_KEYS[kt]} keys of this type, got {n}")
    _check(load().mms_sort_keys_noalloc(kt, _ptr(keys), n, _stream_handle(stream)))
    return keys


def noalloc_status(stream=None) -> None:
    """Raises MMSError if the latest sort_keys_noalloc call on the current device
    recorded a device-side error (waits for ``stream``); allocates nothing."""
    _check(load().mms_noalloc_status(_stream_handle(stream)))


# ---- batched (segmented) sorting ------------------------------------------------------

def _seg_opts(class_fanout=None, max_segment_items: int = 0, tile_items: int = 0, events=None,
              stream=None):
    o = _SegOptions()
    if class_fanout:
        items = class_fanout.items() if isinstance(class_fanout, dict) else enumerate(class_fanout)
        for c, k in items:
            o.class_fanout[int(c)] = int(k)
    o.max_segment_items = int(max_segment_items)
    o.tile_items = int(tile_items)
    if events:
        for e in events:
            if not e.cuda_event:
                e.record(stream)
        arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
        o.num_events = len(events)
        o.events = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
        o._keep = arr
    return o


def segmented_workspace_bytes(kt: int, total_n: int, num_segments: int, with_values: bool = False,
                              class_fanout=None, max_segment_items: int = 0, tile_items: int = 0) -> int:
    o = _seg_opts(class_fanout, max_segment_items, tile_items)
    return int(load().mms_segmented_workspace_bytes(kt, total_n, num_segments, int(with_values),
                                                    ctypes.byref(o)))


def segmented_rounds(kt: int, max_segment_items: int, with_values: bool = False, class_fanout=None,
                     tile_items: int = 0) -> int:
    o = _seg_opts(class_fanout, 0, tile_items)
    return int(load().mms_segmented_rounds(kt, max_segment_items, int(with_values), ctypes.byref(o)))


def segmented_sort(keys, offsets, values=None, workspace=None, stream=None, kt: int | None = None,
                   class_fanout=None, max_segment_items: int = 0, tile_items: int = 0, events=None):
    """Sorts every segment keys[offsets[s]:offsets[s+1]] in place (one batched call).

    ``offsets``: int64 CUDA tensor of num_segments + 1 entries from 0 to keys.numel().
    ``values``: optional 32-bit values that move with 4-byte keys.
    ``class_fanout``: fanout K per size class ceil(log2 n) (dict or list), e.g. from
    :mod:`paper_1702_07961_gb300.autotune`.
    """
    import torch
    assert keys.is_cuda and keys.is_contiguous() and offsets.is_cuda and offsets.is_contiguous()
    assert offsets.dtype == torch.int64
    kt = key_type_of(keys) if kt is None else kt
    nseg = offsets.numel() - 1
    total = keys.numel()
    if workspace is None:
        workspace = torch.empty(segmented_workspace_bytes(kt, total, nseg, values is not None, class_fanout,
                                                          max_segment_items, tile_items),
                                dtype=torch.uint8, device=keys.device)
    o = _seg_opts(class_fanout, max_segment_items, tile_items, events, stream)
    _check(load().mms_segmented_sort(kt, _ptr(keys), _ptr(values), _ptr(offsets), nseg, total,
                                     _ptr(workspace), workspace.numel(), _stream_handle(stream),
                                     ctypes.byref(o)))
    return keys, values


class SegmentedGraph:
    """One batched sort captured into a CUDA graph: ``launch()`` replays it on the
    same buffers (whose contents may change between launches) with one graph launch."""

    def __init__(self, keys, offsets, values=None, workspace=None, kt: int | None = None,
                 class_fanout=None, max_segment_items: int = 0, tile_items: int = 0):
        import torch
        kt = key_type_of(keys) if kt is None else kt
        nseg = offsets.numel() - 1
        total = keys.numel()
        if workspace is None:
            workspace = torch.empty(segmented_workspace_bytes(kt, total, nseg, values is not None, class_fanout,
                                                              max_segment_items, tile_items),
                                    dtype=torch.uint8, device=keys.device)
        self._keep = (keys, offsets, values, workspace)
        self.workspace = workspace
        o = _seg_opts(class_fanout, max_segment_items, tile_items)
        h = ctypes.c_void_p()
        _check(load().mms_segmented_graph_create(kt, _ptr(keys), _ptr(values), _ptr(offsets), nseg, total,
                                                 _ptr(workspace), workspace.numel(), ctypes.byref(o),
                                                 ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(load().mms_graph_launch(self._h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None):
            load().mms_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
