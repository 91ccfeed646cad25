"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data; it holds none of the sorting method's
arithmetic, so both the CUDA path and the CPU oracle may take their inputs
from it.  Every generator is a pure function of its arguments (numpy's
PCG64 generator seeded with ``seed``).

Workload shapes (Sec. 1 and Sec. 6.3):

* ``sortedness``: a sorted list of unique items 0..n-1 followed by ``r``
  swaps of uniformly random index pairs, applied one after another
  (Sec. 1: inputs of varying "sortedness").
* ``permutation``: a uniform random permutation of 0..n-1, the "fully
  random, uniformly distributed input (without repeats)" of Sec. 6.3.
* ``uniform``: i.i.d. uniform keys over the whole key range (repeats allowed).
* ``interleaved``: K sorted runs interleaved in chunks of ``stride`` items,
  stride 32 = the shared-memory bank count; it stands in for the paper's
  hand-made conflict-heavy input (Sec. 6.4), whose seed pattern is not printed.
* ``normal_f32``: N(0,1) binary32 keys with 1% duplicates, 0.1% -0.0 and
  0.01% NaN (a tenth of those negative or payload NaNs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

__all__ = ["uniform", "permutation", "sortedness", "sortedness_cached", "interleaved", "normal_f32",
           "index_payload", "segment_sizes", "offsets_of", "make"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def uniform(n: int, seed: int, dtype=np.uint32) -> np.ndarray:
    """i.i.d. keys uniform over [0, 2^bits)."""
    dt = np.dtype(dtype)
    g = _rng(seed)
    if dt == np.uint32:
        return g.integers(0, 2**32, size=n, dtype=np.uint32)
    if dt == np.uint64:
        return g.integers(0, 2**64 - 1, size=n, dtype=np.uint64, endpoint=True)
    raise TypeError(dt)


def permutation(n: int, seed: int, dtype=np.uint32) -> np.ndarray:
    """Uniform random permutation of 0..n-1 (Sec. 6.3 'fully random')."""
    return _rng(seed).permutation(n).astype(dtype)


_HERE = os.path.dirname(os.path.abspath(__file__))
_SWAPS_SRC = os.path.join(_HERE, "swaps.c")
_SWAPS_SO = os.path.join(_HERE, "_build", "libswaps.so")
_swaps_lock = threading.Lock()
_swaps_lib = None


def build() -> str:
    """Compiles the swap applier (plain C) that large sortedness inputs use."""
    os.makedirs(os.path.dirname(_SWAPS_SO), exist_ok=True)
    if not os.path.exists(_SWAPS_SO) or os.path.getmtime(_SWAPS_SO) < os.path.getmtime(_SWAPS_SRC):
        tmp = _SWAPS_SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SWAPS_SRC])
        os.replace(tmp, _SWAPS_SO)
    return _SWAPS_SO


def _swaps():
    global _swaps_lib
    with _swaps_lock:
        if _swaps_lib is None:
            L = ctypes.CDLL(build())
            for f in (L.synth_apply_swaps_u32, L.synth_apply_swaps_u64):
                f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
                f.restype = None
            _swaps_lib = L
    return _swaps_lib


def _sortedness_batch_size(n: int) -> int:
    return max(1, min(1 << 17, int(np.sqrt(n)) * 4))


def sortedness(n: int, r: int, seed: int, dtype=np.uint32, batch: int | None = None,
               native: bool | None = None) -> np.ndarray:
    """0..n-1 followed by r random pair swaps applied in order (Sec. 1).

    Swaps are drawn in batches (i then j of every batch).  The numpy path
    applies, within a batch, the swaps that touch a position no other swap of
    the batch touches at once (they commute with everything else in the
    batch) and the rest one by one in draw order; the native path (a small C
    loop, used when ``native`` is true or, by default, for r >= 10^6) applies
    every swap in draw order.  Both give exactly the result of the r swaps
    applied sequentially, so they agree bit for bit.
    """
    dt = np.dtype(dtype)
    a = np.arange(n, dtype=dt)
    if n < 2 or r <= 0:
        return a
    g = _rng(seed)
    if batch is None:
        batch = _sortedness_batch_size(n)
    if native is None:
        native = r >= 10**6 and dt in (np.dtype(np.uint32), np.dtype(np.uint64))
    apply = None
    if native:
        L = _swaps()
        apply = L.synth_apply_swaps_u32 if dt == np.dtype(np.uint32) else L.synth_apply_swaps_u64
    left = int(r)
    while left > 0:
        b = min(batch, left)
        i = g.integers(0, n, size=b, dtype=np.int64)
        j = g.integers(0, n, size=b, dtype=np.int64)
        if apply is not None:
            apply(a.ctypes.data, i.ctypes.data, j.ctypes.data, b)
        else:
            pos = np.concatenate([i, j])
            uniq, counts = np.unique(pos, return_counts=True)
            multi = uniq[counts > 1]
            clash = np.isin(i, multi) | np.isin(j, multi)
            gi, gj = i[~clash], j[~clash]
            a[gi], a[gj] = a[gj], a[gi].copy()
            for x, y in zip(i[clash].tolist(), j[clash].tolist()):
                a[x], a[y] = a[y], a[x]
        left -= b
    return a


def sortedness_cached(n: int, r: int, seed: int, dtype=np.uint32) -> np.ndarray:
    """sortedness(), stored once per (n, r, seed, dtype) in the system's
    temporary directory, for the inputs that take a while to draw (r = 10^9 at
    n = 10^8: about half a minute)."""
    dt = np.dtype(dtype)
    path = os.path.join(tempfile.gettempdir(), f"mms_sortedness_{n}_{r}_{seed}_{dt.name}.npy")
    if os.path.exists(path):
        a = np.load(path)
        if a.shape == (n,) and a.dtype == dt:
            return a
    a = sortedness(n, r, seed, dt)
    tmp = path + f".{os.getpid()}.tmp.npy"
    np.save(tmp, a)
    os.replace(tmp, path)
    return a


def interleaved(n: int, K: int, stride: int = 32, dtype=np.uint32) -> np.ndarray:
    """K ascending runs interleaved in chunks of ``stride`` items.

    Position p is in chunk c = p // stride, which belongs to run r = c mod K;
    it is item j = (c // K) * stride + p % stride of that run and holds the
    value j*K + r.  Values are dense and unique when n is a multiple of
    K*stride.  For 64-bit keys both halves carry the value.
    """
    p = np.arange(n, dtype=np.uint64)
    c = p // np.uint64(stride)
    r = c % np.uint64(K)
    j = (c // np.uint64(K)) * np.uint64(stride) + p % np.uint64(stride)
    v = j * np.uint64(K) + r
    dt = np.dtype(dtype)
    if dt == np.uint64:
        return (v << np.uint64(32)) | v
    return v.astype(dt)


def normal_f32(n: int, seed: int) -> np.ndarray:
    """N(0,1) binary32 keys with duplicates, -0.0 and NaNs of both signs."""
    g = _rng(seed)
    x = g.standard_normal(n, dtype=np.float32)
    if n == 0:
        return x
    bits = x.view(np.uint32)
    nd = n // 100
    if nd:
        dst = g.integers(0, n, size=nd)
        src = g.integers(0, n, size=nd)
        bits[dst] = bits[src]
    nz = n // 1000
    if nz:
        bits[g.integers(0, n, size=nz)] = np.uint32(0x80000000)
    nn = max(n // 10000, 1 if n >= 64 else 0)
    if nn:
        where = g.integers(0, n, size=nn)
        bits[where] = np.uint32(0x7FC00000)
        k = max(nn // 10, 1)
        neg, pos_pay, neg_pay = where[:k], where[k:2 * k], where[2 * k:3 * k]
        payload = g.integers(1, 1 << 22, size=k, dtype=np.uint32)
        bits[neg] = np.uint32(0xFFC00000)
        bits[pos_pay] = np.uint32(0x7F800000) | payload[: len(pos_pay)]
        bits[neg_pay] = np.uint32(0xFF800000) | payload[: len(neg_pay)]
    return bits.view(np.float32)


def segment_sizes(num: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Sizes of a batch of independent arrays, log-uniform on [lo, hi] (the
    batched workload: thousands of arrays of uneven size)."""
    g = _rng(seed)
    x = np.exp(g.uniform(np.log(lo), np.log(hi + 1), size=num))
    return np.minimum(np.floor(x).astype(np.int64), hi)


def offsets_of(sizes) -> np.ndarray:
    """Exclusive prefix sums of sizes, with the total appended (int64)."""
    o = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(np.asarray(sizes, dtype=np.int64), out=o[1:])
    return o


def index_payload(n: int) -> np.ndarray:
    """32-bit payload equal to the original index, so stability can be read off."""
    return np.arange(n, dtype=np.uint32)


def make(kind: str, n: int, seed: int = 1, **kw) -> np.ndarray:
    """Dispatch by workload name (used by the tests and the benchmark)."""
    if kind == "uniform":
        return uniform(n, seed, kw.get("dtype", np.uint32))
    if kind == "permutation":
        return permutation(n, seed, kw.get("dtype", np.uint32))
    if kind == "sortedness":
        return sortedness(n, kw["r"], seed, kw.get("dtype", np.uint32))
    if kind == "interleaved":
        return interleaved(n, kw.get("K", 8), kw.get("stride", 32), kw.get("dtype", np.uint32))
    if kind == "normal_f32":
        return normal_f32(n, seed)
    raise ValueError(kind)
