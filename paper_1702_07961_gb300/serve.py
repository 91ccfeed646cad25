"""Serving loop with continuous batching over the library's sorts.

Sort requests (keys from host memory, u32 / u64 / f32, optionally with 32-bit
values) arrive over time.  The loop admits them while device memory and
launch slots are free, and keeps every request's buffers resident in one
device arena allocated once up front.  It coalesces small requests of one
key class into a single batched launch (mms_segmented_sort), and sorts large
ones as whole arrays (mms_sort_keys / mms_sort_pairs).  Each launch group
runs on its own CUDA stream, so groups started at different times overlap
on the device.  A group's inputs are copied in from pinned host memory, and
its results are copied back, on the same stream.  Requests that arrive
while others are in flight join the next group that a freed slot and freed
memory allow.

Nothing here changes the sorting arithmetic: a request's output is the same
bits whether it is sorted alone or in a mix (the parity tests check this).

The paper sorts one array at a time; serving is this package's extension of
its method to a stream of requests.
"""
from __future__ import annotations

import bisect
import time
from dataclasses import dataclass, field

import numpy as np

from . import (KEY_F32, KEY_U32, KEY_U64, _check, _ptr, _seg_opts, _stream_handle, load,
               segmented_workspace_bytes, workspace_bytes)

ALIGN = 256
KEY_BYTES = {KEY_U32: 4, KEY_F32: 4, KEY_U64: 8}
NP_DTYPE = {KEY_U32: np.uint32, KEY_F32: np.float32, KEY_U64: np.uint64}


def _torch_dtype(kt):
    import torch
    return {KEY_U32: torch.int32, KEY_F32: torch.float32, KEY_U64: torch.int64}[kt]


class DeviceArena:
    """First-fit sub-allocator over one fixed byte range (offsets only: the
    caller maps them onto one device allocation).  Blocks are multiples of
    256 bytes; freed blocks merge with free neighbours."""

    def __init__(self, size: int):
        self.size = size // ALIGN * ALIGN
        self.free_list = [(0, self.size)]          # (offset, length), sorted by offset
        self.used = {}                             # offset -> length

    def alloc(self, nbytes: int):
        need = max(ALIGN, (nbytes + ALIGN - 1) // ALIGN * ALIGN)
        for i, (off, ln) in enumerate(self.free_list):
            if ln >= need:
                if ln == need:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + need, ln - need)
                self.used[off] = need
                return off
        return None

    def free(self, off: int) -> None:
        ln = self.used.pop(off)
        i = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(i, (off, ln))
        # merge with the right and left neighbours
        if i + 1 < len(self.free_list) and off + ln == self.free_list[i + 1][0]:
            self.free_list[i] = (off, ln + self.free_list[i + 1][1])
            self.free_list.pop(i + 1)
        if i > 0 and self.free_list[i - 1][0] + self.free_list[i - 1][1] == self.free_list[i][0]:
            self.free_list[i - 1] = (self.free_list[i - 1][0], self.free_list[i - 1][1] + self.free_list[i][1])
            self.free_list.pop(i)

    @property
    def bytes_used(self) -> int:
        return sum(self.used.values())


@dataclass
class Request:
    """One sort job.  `keys` (and `values`) are host arrays; results land in
    `out_keys` / `out_values` (pinned host tensors) when `done` is set."""
    rid: int
    kt: int
    keys: np.ndarray
    values: np.ndarray | None = None
    arrival: float = 0.0                      # seconds after the run starts
    # filled in by the server
    h_keys: object = None
    h_values: object = None
    out_keys: object = None
    out_values: object = None
    start: float | None = None
    finish: float | None = None
    group: int = -1
    error: str | None = None                  # set when the group's sort reported a device error

    @property
    def n(self) -> int:
        return int(self.keys.shape[0])

    @property
    def klass(self):
        return (self.kt, self.values is not None)

    def latency(self) -> float:
        return self.finish - self.arrival


def _round(x: int) -> int:
    return (x + ALIGN - 1) // ALIGN * ALIGN


def group_bytes(reqs) -> int:
    """Device bytes a launch group needs: keys and values back to back, the
    segment offsets, and the sort's workspace."""
    kt, pairs = reqs[0].klass
    total = sum(r.n for r in reqs)
    kb = KEY_BYTES[kt]
    b = _round(total * kb) + (_round(total * 4) if pairs else 0)
    if len(reqs) == 1:
        return b + _round(workspace_bytes(kt, max(total, 2), pairs))
    return b + _round(8 * (len(reqs) + 1)) + _round(segmented_workspace_bytes(
        kt, total, len(reqs), pairs, None, max(r.n for r in reqs)))


def form_group(queue, small_max: int, batch_max: int, max_segments: int):
    """Takes the next launch group off the FIFO queue: the head request, plus,
    when it is small, every later queued small request of the same key class
    while the group stays within batch_max items and max_segments requests."""
    head = queue[0]
    if head.n > small_max:
        return [head]
    group = [head]
    items = head.n
    for r in queue[1:]:
        if len(group) >= max_segments:
            break
        if r.klass == head.klass and r.n <= small_max and items + r.n <= batch_max:
            group.append(r)
            items += r.n
    return group


# Workspace status words the library writes (the first word of a workspace).
_DEVICE_ERRORS = {1: "device-side wait timed out", 2: "device consistency check failed"}


def finish_group(reqs, status_word: int, t: float) -> None:
    """Marks a completed launch group's requests finished at time t; a non-zero
    workspace status word means the sort stopped early on the device, so its
    results are not sorted: every request of the group is marked failed."""
    err = None
    if status_word != 0:
        err = _DEVICE_ERRORS.get(int(status_word), f"device status {int(status_word)}")
    for r in reqs:
        r.finish = t
        r.error = err


@dataclass
class _Launch:
    reqs: list
    offset: int
    stream: object
    event: object
    slot: int
    keep: list = field(default_factory=list)
    status: object = None                     # pinned copy of the workspace status word


class SortServer:
    """Continuous-batching sort server on one GPU.

    budget_bytes: device memory for request buffers and workspaces (one arena).
    slots: launch groups in flight at once (one CUDA stream each).
    small_max: requests up to this many keys are coalesced into batched launches
    of at most batch_max items and max_segments requests.
    """

    def __init__(self, budget_bytes: int = 40 << 30, slots: int = 4, small_max: int = 1 << 20,
                 batch_max: int = 1 << 25, max_segments: int = 4096, device=None):
        import torch
        self.device = torch.device("cuda") if device is None else device
        self.arena = DeviceArena(budget_bytes)
        self.mem = torch.empty(self.arena.size, dtype=torch.uint8, device=self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.small_max, self.batch_max, self.max_segments = small_max, batch_max, max_segments
        self.inflight: list[_Launch] = []
        self.groups = 0
        self.coalesced = 0
        self.peak_bytes = 0
        self.max_inflight = 0

    # -- host buffers ---------------------------------------------------------
    @staticmethod
    def prepare(req: Request) -> None:
        """Pins the request's host data and allocates pinned result buffers."""
        import torch
        td = _torch_dtype(req.kt)
        req.h_keys = torch.from_numpy(np.ascontiguousarray(req.keys).view(
            {KEY_U32: np.int32, KEY_F32: np.float32, KEY_U64: np.int64}[req.kt])).pin_memory()
        req.out_keys = torch.empty(req.n, dtype=td, pin_memory=True)
        if req.values is not None:
            req.h_values = torch.from_numpy(np.ascontiguousarray(req.values).view(np.int32)).pin_memory()
            req.out_values = torch.empty(req.n, dtype=torch.int32, pin_memory=True)

    def _view(self, off: int, nbytes: int, dtype):
        return self.mem[off:off + nbytes].view(dtype)

    # -- one launch group ------------------------------------------------------
    def _launch(self, reqs, now: float) -> bool:
        import torch
        nbytes = group_bytes(reqs)
        off = self.arena.alloc(nbytes)
        if off is None:
            return False
        self.peak_bytes = max(self.peak_bytes, self.arena.bytes_used)
        slot = self.free_slots.pop()
        st = self.streams[slot]
        kt, pairs = reqs[0].klass
        kb = KEY_BYTES[kt]
        total = sum(r.n for r in reqs)
        p = off
        keys = self._view(p, total * kb, _torch_dtype(kt))
        p += _round(total * kb)
        vals = None
        if pairs:
            vals = self._view(p, total * 4, torch.int32)
            p += _round(total * 4)
        L = load()
        keep = []
        with torch.cuda.stream(st):
            pos = 0
            for r in reqs:
                keys[pos:pos + r.n].copy_(r.h_keys, non_blocking=True)
                if pairs:
                    vals[pos:pos + r.n].copy_(r.h_values, non_blocking=True)
                r.start = now
                r.group = self.groups
                pos += r.n
            if len(reqs) == 1:
                ws_len = _round(workspace_bytes(kt, max(total, 2), pairs))
                ws = self._view(p, ws_len, torch.uint8)
                if pairs:
                    _check(L.mms_sort_pairs(kt, _ptr(keys), _ptr(vals), total, _ptr(ws), ws_len,
                                            _stream_handle(st)))
                else:
                    _check(L.mms_sort_keys(kt, _ptr(keys), total, _ptr(ws), ws_len, _stream_handle(st)))
            else:
                offs_h = torch.zeros(len(reqs) + 1, dtype=torch.int64, pin_memory=True)
                offs_h[1:] = torch.tensor(np.cumsum([r.n for r in reqs]), dtype=torch.int64)
                offs = self._view(p, 8 * (len(reqs) + 1), torch.int64)
                offs.copy_(offs_h, non_blocking=True)
                keep.append(offs_h)
                p += _round(8 * (len(reqs) + 1))
                mx = max(r.n for r in reqs)
                ws_len = _round(segmented_workspace_bytes(kt, total, len(reqs), pairs, None, mx))
                ws = self._view(p, ws_len, torch.uint8)
                o = _seg_opts(None, mx)
                import ctypes
                _check(L.mms_segmented_sort(kt, _ptr(keys), _ptr(vals), _ptr(offs), len(reqs), total, _ptr(ws),
                                            ws_len, _stream_handle(st), ctypes.byref(o)))
                self.coalesced += len(reqs)
            pos = 0
            for r in reqs:
                r.out_keys.copy_(keys[pos:pos + r.n], non_blocking=True)
                if pairs:
                    r.out_values.copy_(vals[pos:pos + r.n], non_blocking=True)
                pos += r.n
            # The sort cleared its workspace's status word before running; read
            # it back with the results, so a sort stopped on the device is
            # reported as failed rather than returned as sorted.
            status = torch.empty(1, dtype=torch.int32, pin_memory=True)
            status.copy_(ws[:4].view(torch.int32), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.inflight.append(_Launch(reqs, off, st, ev, slot, keep, status))
        self.max_inflight = max(self.max_inflight, len(self.inflight))
        self.groups += 1
        return True

    def _poll(self, clock) -> int:
        done = 0
        still = []
        for g in self.inflight:
            if g.event.query():
                finish_group(g.reqs, int(g.status[0]) if g.status is not None else 0, clock())
                self.arena.free(g.offset)
                self.free_slots.append(g.slot)
                done += len(g.reqs)
            else:
                still.append(g)
        self.inflight = still
        return done

    # -- the loop ----------------------------------------------------------------
    def run(self, requests, time_scale: float = 1.0):
        """Serves `requests` (with `arrival` times in seconds) in real time.
        Returns the requests with start/finish times filled in."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            if r.h_keys is None:
                self.prepare(r)
        t0 = time.perf_counter()

        def clock():
            return (time.perf_counter() - t0) / time_scale

        nxt = 0
        queue = []
        finished = 0
        while finished < len(reqs):
            now = clock()
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                queue.append(reqs[nxt])
                nxt += 1
            finished += self._poll(clock)
            while queue and self.free_slots:
                group = form_group(queue, self.small_max, self.batch_max, self.max_segments)
                if not self._launch(group, clock()):
                    if self.inflight:
                        break                   # memory full: wait for a group to finish
                    # Nothing in flight, so the arena is empty: fall back to the
                    # head request alone, and refuse one that can never fit.
                    if len(group) > 1 and self._launch(group[:1], clock()):
                        group = group[:1]
                    else:
                        raise MemoryError(f"request {group[0].rid} ({group[0].n} keys) needs "
                                          f"{group_bytes(group[:1])} bytes, more than the "
                                          f"{self.arena.size}-byte budget")
                ids = {id(r) for r in group}
                queue = [r for r in queue if id(r) not in ids]
            if not queue or not self.free_slots:
                time.sleep(2e-5)
        return reqs


def serve_serial(requests, device=None, time_scale: float = 1.0):
    """The plain baseline: requests in arrival order, one at a time, each
    copied in, sorted as a whole array, copied out and waited for."""
    import torch
    dev = torch.device("cuda") if device is None else device
    reqs = sorted(requests, key=lambda r: r.arrival)
    for r in reqs:
        if r.h_keys is None:
            SortServer.prepare(r)
    mx = max(r.n for r in reqs)
    ws = torch.empty(max(workspace_bytes(KEY_U64, max(mx, 2), True), workspace_bytes(KEY_U32, max(mx, 2), True)),
                     dtype=torch.uint8, device=dev)
    kbuf = torch.empty(mx * 8, dtype=torch.uint8, device=dev)
    vbuf = torch.empty(mx, dtype=torch.int32, device=dev)
    st = torch.cuda.Stream(device=dev)
    L = load()
    t0 = time.perf_counter()

    def clock():
        return (time.perf_counter() - t0) / time_scale

    for r in reqs:
        while clock() < r.arrival:
            time.sleep(2e-5)
        r.start = clock()
        keys = kbuf[:r.n * KEY_BYTES[r.kt]].view(_torch_dtype(r.kt))
        with torch.cuda.stream(st):
            keys.copy_(r.h_keys, non_blocking=True)
            if r.values is not None:
                vbuf[:r.n].copy_(r.h_values, non_blocking=True)
                _check(L.mms_sort_pairs(r.kt, _ptr(keys), _ptr(vbuf), r.n, _ptr(ws), ws.numel(), _stream_handle(st)))
                r.out_values.copy_(vbuf[:r.n], non_blocking=True)
            else:
                _check(L.mms_sort_keys(r.kt, _ptr(keys), r.n, _ptr(ws), ws.numel(), _stream_handle(st)))
            r.out_keys.copy_(keys, non_blocking=True)
        st.synchronize()
        r.finish = clock()
    return reqs


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process of `rate` requests per second."""
    g = np.random.default_rng(np.random.PCG64(seed))
    return np.cumsum(g.exponential(1.0 / rate, size=count))


def summarize(reqs) -> dict:
    lat = np.array([r.latency() for r in reqs]) * 1e3
    keys = sum(r.n for r in reqs)
    span = max(r.finish for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "failed": sum(r.error is not None for r in reqs),
            "keys": keys, "seconds": span, "gkeys_per_s": keys / span / 1e9,
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "latency_ms_mean": float(lat.mean())}
