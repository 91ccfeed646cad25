"""CPU oracle for the GPU Multiway Mergesort hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_1702_07961_gb300``) never imports, links or runs it,
and this package imports nothing from the product: the two share no code.

Every function below is the plain definition of what one step of the method
computes, written as slowly and as directly as possible:

* :func:`sort` -- the sort itself (Sec. 4 "Multiway Mergesort"): the unique
  stable ascending order, computed by the textbook two-way mergesort in
  ``mms_oracle.c`` (ties taken from the left run).
* :func:`tile_sort` -- the base case (Sec. 4.3 "Internal Memory Sort"):
  every fixed-size tile sorted on its own.
* :func:`corank` / :func:`splitter_table` -- the parallel partitioning
  (Sec. 4.1): for output rank ``k`` of a group of K sorted runs, the number
  of items each run contributes to the ``k`` smallest.  The paper's
  non-overlap condition ("a <= b implies i <= j") cannot hold with repeated
  keys; the reading taken is the strict order (key, run index, position in
  run), which makes the pivot tuple unique.  Brute force: stable-sort the
  concatenated group (concatenation order *is* (run, position) order) and
  count the origin runs of the first ``k`` items.
* :func:`merge_pass` -- one K-way merge round (Sec. 4.2): each group of K
  consecutive sorted runs becomes one sorted run; by the definition it is
  the stable sort of the group's concatenation.

Floats follow IEEE-754 totalOrder on bit patterns (the paper sorts only
integers; this is the reading taken for binary32 keys).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mms_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")

KEY_TYPES = {"u32": 0, "u64": 1, "f32": 2}
DTYPES = {"u32": np.uint32, "u64": np.uint64, "f32": np.float32}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles ``mms_oracle.c`` with the host C compiler (plain C, -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-pthread", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            L.oracle_sort.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
            L.oracle_sort.restype = ctypes.c_int
            L.oracle_sort_threads.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_size_t, ctypes.c_int]
            L.oracle_sort_threads.restype = ctypes.c_int
            L.oracle_argsort.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
            L.oracle_argsort.restype = ctypes.c_int
            L.oracle_less.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t]
            L.oracle_less.restype = ctypes.c_int
            L.oracle_set_mutation.argtypes = [ctypes.c_int]
            L.oracle_set_mutation.restype = None
            L.oracle_get_mutation.argtypes = []
            L.oracle_get_mutation.restype = ctypes.c_int
            _lib = L
    return _lib


def key_type_of(a: np.ndarray) -> str:
    for name, dt in DTYPES.items():
        if a.dtype == dt:
            return name
    raise TypeError(f"unsupported key dtype {a.dtype}")


@contextlib.contextmanager
def mutation(m: int):
    """Plants mistake ``m`` in the oracle for the duration of the block (tests only)."""
    L = lib()
    old = L.oracle_get_mutation()
    L.oracle_set_mutation(int(m))
    try:
        yield
    finally:
        L.oracle_set_mutation(old)


def less(keys: np.ndarray, i: int, j: int) -> bool:
    """keys[i] strictly before keys[j] in the key order."""
    keys = np.ascontiguousarray(keys)
    return bool(lib().oracle_less(KEY_TYPES[key_type_of(keys)], keys.ctypes.data, i, j))


def argsort(keys: np.ndarray) -> np.ndarray:
    """Stable ascending permutation: out[p] = input index landing at position p."""
    keys = np.ascontiguousarray(keys)
    perm = np.empty(keys.shape[0], dtype=np.uint64)
    rc = lib().oracle_argsort(KEY_TYPES[key_type_of(keys)], keys.ctypes.data, keys.shape[0], perm.ctypes.data)
    if rc != 0:
        raise MemoryError(f"oracle_argsort failed ({rc})")
    return perm


def sort(keys: np.ndarray, values: np.ndarray | None = None):
    """Stable ascending sort (Sec. 4); returns sorted copies (keys, values)."""
    k = np.array(keys, copy=True, order="C")
    v = None if values is None else np.array(values, dtype=np.uint32, copy=True, order="C")
    if v is not None and v.shape[0] != k.shape[0]:
        raise ValueError("keys and values differ in length")
    rc = lib().oracle_sort(KEY_TYPES[key_type_of(k)], k.ctypes.data,
                           None if v is None else v.ctypes.data, k.shape[0])
    if rc != 0:
        raise MemoryError(f"oracle_sort failed ({rc})")
    return k, v


def sort_parallel(keys: np.ndarray, values: np.ndarray | None = None, threads: int | None = None):
    """:func:`sort` with the mergesort's top recursion levels split over
    ``threads`` host threads (default: every core this process may use).  The
    same ranges are split and merged the same way, so the result is the
    same; only the CPU baseline's timing uses it."""
    if threads is None:
        threads = host_cores()
    k = np.array(keys, copy=True, order="C")
    v = None if values is None else np.array(values, dtype=np.uint32, copy=True, order="C")
    if v is not None and v.shape[0] != k.shape[0]:
        raise ValueError("keys and values differ in length")
    rc = lib().oracle_sort_threads(KEY_TYPES[key_type_of(k)], k.ctypes.data,
                                   None if v is None else v.ctypes.data, k.shape[0], int(threads))
    if rc != 0:
        raise MemoryError(f"oracle_sort_threads failed ({rc})")
    return k, v


def host_cores() -> int:
    """Cores this process may run on (the affinity mask, else the CPU count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def tile_sort(keys: np.ndarray, tile: int, values: np.ndarray | None = None):
    """Base case (Sec. 4.3): every tile of ``tile`` consecutive keys sorted on its own."""
    k = np.array(keys, copy=True)
    v = None if values is None else np.array(values, dtype=np.uint32, copy=True)
    for s in range(0, k.shape[0], tile):
        ks, vs = sort(k[s:s + tile], None if v is None else v[s:s + tile])
        k[s:s + tile] = ks
        if v is not None:
            v[s:s + tile] = vs
    return k, v


def corank(runs, k: int) -> np.ndarray:
    """Pivot indices for output rank k of sorted ``runs`` (Sec. 4.1), brute force.

    c[r] = number of items of run r among the k smallest items of the group
    under the strict order (key, run index, position in run).
    """
    lens = [len(r) for r in runs]
    if not 0 <= k <= sum(lens):
        raise ValueError("rank out of range")
    cat = np.concatenate([np.asarray(r) for r in runs]) if runs else np.zeros(0, np.uint32)
    perm = argsort(cat)[:k].astype(np.int64)
    starts = np.cumsum([0] + lens)
    origin = np.searchsorted(starts, perm, side="right") - 1
    return np.bincount(origin, minlength=len(runs)).astype(np.int64)[: len(runs)]


def group_bounds(n: int, run_len: int, K: int):
    """(start, stop) of every group of K consecutive runs of length run_len."""
    g = run_len * K
    return [(s, min(s + g, n)) for s in range(0, n, g)]


def splitter_table(data: np.ndarray, run_len: int, K: int, S: int) -> np.ndarray:
    """Co-ranks at every output-tile start j*S of every group, brute force.

    Row t (tiles numbered group by group) holds, for r = 0..K-1, the number of
    items run r of the tile's group contributes to the group's first j*S
    outputs.  Runs past the end of the array are empty.
    """
    rows = []
    for gs, ge in group_bounds(data.shape[0], run_len, K):
        grp = data[gs:ge]
        perm = argsort(grp).astype(np.int64)
        origin = perm // run_len
        onehot_cum = np.zeros((K, grp.shape[0] + 1), dtype=np.int64)
        for r in range(K):
            onehot_cum[r, 1:] = np.cumsum(origin == r)
        for j in range((grp.shape[0] + S - 1) // S):
            rows.append(onehot_cum[:, j * S])
    return np.array(rows, dtype=np.int64).reshape(-1, K)


def merge_pass(data: np.ndarray, run_len: int, K: int, values: np.ndarray | None = None):
    """One K-way merge round (Sec. 4.2): each group of K runs -> one sorted run."""
    k = np.array(data, copy=True)
    v = None if values is None else np.array(values, dtype=np.uint32, copy=True)
    for gs, ge in group_bounds(k.shape[0], run_len, K):
        ks, vs = sort(k[gs:ge], None if v is None else v[gs:ge])
        k[gs:ge] = ks
        if v is not None:
            v[gs:ge] = vs
    return k, v


def segmented_sort(keys: np.ndarray, offsets, values: np.ndarray | None = None):
    """Batched sort: every segment keys[offsets[s]:offsets[s+1]] sorted on its
    own, stably (values move with their keys) -- the definition of sorting many
    independent arrays, applied one array at a time."""
    k = np.array(keys, copy=True)
    v = None if values is None else np.array(values, dtype=np.uint32, copy=True)
    off = np.asarray(offsets, dtype=np.int64)
    for s in range(off.shape[0] - 1):
        a, b = int(off[s]), int(off[s + 1])
        if b - a > 1:
            ks, vs = sort(k[a:b], None if v is None else v[a:b])
            k[a:b] = ks
            if v is not None:
                v[a:b] = vs
    return k, v
