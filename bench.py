#!/usr/bin/env python
"""Benchmark: GPU Multiway Mergesort of 10^8 uint32 keys on one GB300.

One step = one whole sort through the C ABI (base case, then for every merge
round the splitter and the merge pass) of a fresh copy of the workload: a
uniform random permutation of 0..N-1, the paper's "fully random" input
(Sec. 6.3), N = 10^8 4-byte integers.  The input (400 MB) is larger than L2
(129 MB), and a 400 MB device copy restores the unsorted input before every
step, outside the timed events.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
textbook stable mergesort) on a bounded sample of the same workload instead.
Multi-GPU runs are independent replicas (weak scaling): each rank sorts its own
array; value = all ranks' keys / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gkeys/s at 1e8 uint32"
UNIT = "Gkeys/s"
DEFAULT_N = 10**8
KEY_BYTES = 4
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "merge_pass_traffic.json")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="mms", choices=["mms", "reference"])
    p.add_argument("--n", type=int, default=DEFAULT_N)
    p.add_argument("--fanout", type=int, default=0, help="merge fanout K (0 = planner)")
    p.add_argument("--tile", type=int, default=0, help="tile items (0 = library default)")
    p.add_argument("--base-items", type=int, default=0,
                   help="length of the base case's sorted runs (0 = library default, one CTA tile; "
                        "16384 / 32768 / 65536 for 4-byte keys: one cluster of 2 / 4 / 8 CTAs per run)")
    p.add_argument("--pairs", action="store_true", help="key + uint32 index payload (stable key-value sort)")
    p.add_argument("--merge-variant", default="tree", choices=["tree", "partition", "pipelined"],
                   help="merge rounds: the CTA merge tree (default), the heap-free partition variant or "
                        "the pipelined variant")
    p.add_argument("--key", default="u32", choices=["u32", "u64", "f32"],
                   help="sort workload: key type (the headline is u32)")
    p.add_argument("--input", default="permutation", choices=["permutation", "sortedness", "interleaved"],
                   help="sort workload: a uniform permutation (the headline), a sortedness input with "
                        "--swaps pair swaps, or --runs runs interleaved at --stride")
    p.add_argument("--swaps", type=int, default=0)
    p.add_argument("--seed", type=int, default=1,
                   help="seed of the synthetic input (rank r of a replica run uses seed + r)")
    p.add_argument("--runs", type=int, default=8)
    p.add_argument("--stride", type=int, default=32)
    p.add_argument("--min-timed-s", type=float, default=1.0,
                   help="repeat the K-step timed window until the windows span this many seconds")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-slots", type=int, default=3,
                   help="end-to-end pipeline depth: steps in flight, each with its own buffers and stream")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=1 << 26)
    p.add_argument("--workload", default="sort", choices=["sort", "batched", "serve", "configs", "sweep"],
                   help="sort: one 10^8-key array per step; batched: 20000 arrays of "
                        "log-uniform size in [2^8, 2^20] with uint32 payloads per step")
    p.add_argument("--arrays", type=int, default=20000)
    p.add_argument("--retune", action="store_true", help="batched: re-run the autotuner")
    p.add_argument("--tuned-out", default="", help="batched: where --retune writes its table "
                   "(default: the package's tuned table)")
    p.add_argument("--requests", type=int, default=100, help="serve: requests per arrival-rate run")
    p.add_argument("--slots", type=int, default=4, help="serve: launch slots (streams) of the server")
    p.add_argument("--small-max", type=int, default=1 << 20,
                   help="serve: requests of at most this many keys are coalesced (0: no coalescing)")
    p.add_argument("--sweep-sizes", default="",
                   help="sweep: comma-separated sizes (default 2^20, 2^22, 2^24, 2^26, 10^8, 2^28 for u32)")
    p.add_argument("--max-swaps", type=float, default=1e8,
                   help="configs: largest sortedness swap count r (10^9 takes minutes on the host)")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---- clocks sampled during the timed region ---------------------------------------

class ClockSampler:
    FIELDS = ["timestamp", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={','.join(self.FIELDS)}",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        rows = [r for (t, r) in self.rows if t0 - 0.15 <= t <= t1 + 0.15] or [r for (_, r) in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ---- CPU oracle timing --------------------------------------------------------------

def time_oracle(keys_np, sample: int):
    """The oracle on the host: the textbook stable mergesort with its top
    recursion levels on every core (the record reported), and the plain
    single-threaded run beside it."""
    import oracle
    cores = oracle.host_cores()
    s = keys_np[:sample].copy()
    t0 = time.perf_counter()
    oracle.sort_parallel(s, None, cores)
    dt_all = time.perf_counter() - t0
    s1 = keys_np[:sample].copy()
    t0 = time.perf_counter()
    oracle.sort(s1)
    dt_one = time.perf_counter() - t0
    return {"value": s.shape[0] / dt_all / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {s.shape[0]} keys of the workload; textbook stable top-down mergesort, "
                      f"top recursion levels split over {cores} host threads",
            "seconds": round(dt_all, 3),
            "single_core": {"value": s1.shape[0] / dt_one / 1e9, "unit": UNIT, "cores": 1,
                            "seconds": round(dt_one, 3)}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import synth
    import oracle
    cores = oracle.host_cores()
    n_sample = min(args.n, 1 << 23)
    keys = synth.permutation(args.n, 1)[:n_sample].copy()      # first keys of the GPU arm's workload
    for _ in range(args.warmup):
        oracle.sort_parallel(keys, None, cores)
    times = []
    for _ in range(args.steps):
        s = keys.copy()
        t0 = time.perf_counter()
        oracle.sort_parallel(s, None, cores)
        times.append(time.perf_counter() - t0)
    sec = sum(times)
    value = n_sample * args.steps / sec / 1e9
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"uniform random permutation of 0..N-1, N={args.n} uint32 (Sec. 6.3 fully random); "
                               f"reference arm sorts a {n_sample}-key sample per step on the host",
                   "global_batch": n_sample, "seq_len": None, "parallelism": "cpu"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_sample} keys of the workload per step, textbook stable mergesort "
                                   f"with its top recursion levels on {cores} host threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ---- the GPU arm --------------------------------------------------------------------

def aggregate_over_ranks(total_ms: float, keys_per_rank: int, steps: int, world: int, device=None):
    """Replicas: every rank sorts its own array.  Returns (ms per step of the
    slowest rank, Gkeys/s of the whole job = all ranks' keys / that time)."""
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item()) / steps
    return ms, keys_per_rank * world / (ms / 1e3) / 1e9


def hbm_peak() -> float:
    """Measured HBM copy bandwidth of the GB300s (GB/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


KERNEL_SOURCES = {
    "merge_pass_kernel": ["merge_pass.cu", "merge_tile.cuh", "mms_common.cuh", "mms_kernels.cuh"],
    "tile_sort_kernel": ["tile_sort.cu", "tile_sort.cuh", "mms_common.cuh", "mms_kernels.cuh"],
    "tile_sort_cluster_kernel": ["tile_sort_cluster.cu", "tile_sort.cuh", "mms_common.cuh",
                                 "mms_kernels.cuh"],
}


def kernel_source_hash(kernel: str = "merge_pass_kernel") -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1702_07961_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(n: int, kernel: str):
    """DRAM bytes (read + write) of one launch of `kernel` from the committed ncu
    summary, taken at the bench workload's size (scaled if n differs, the
    traffic being proportional to the keys moved); None when absent or taken
    on a different kernel source."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            p = json.load(f).get(kernel)
    except (OSError, ValueError, AttributeError):
        return None
    if not p or p.get("kernel_source_hash") != kernel_source_hash(kernel):
        return None
    return p["dram_bytes_per_launch"] * n / p["n"]


def make_sort_input(args, N: int, rank: int):
    """The sort workload's keys (numpy, host) and a description: a uniform
    permutation of 0..N-1 (Sec. 6.3 'fully random', the headline), a
    sortedness input (Sec. 1), runs interleaved at a stride (the C3 layout),
    or N(0,1) floats with duplicates, -0.0 and NaNs for f32 keys."""
    import numpy as np
    import synth
    if args.key == "f32":
        return (synth.normal_f32(N, args.seed + 2 + rank),
                "N(0,1) float32 with 1% duplicates, 0.1% -0.0, 0.01% NaN")
    if args.input == "sortedness":
        v = synth.sortedness_cached(N, args.swaps, args.seed + 1 + rank) if args.swaps >= 10**6 else \
            synth.sortedness(N, args.swaps, args.seed + 1 + rank)
        desc = f"sortedness: 0..N-1 then {args.swaps} random pair swaps (Sec. 1)"
    elif args.input == "interleaved":
        v = synth.interleaved(N, args.runs, args.stride)
        desc = f"{args.runs} sorted runs interleaved at stride {args.stride} (C3 layout)"
    else:
        v = synth.permutation(N, args.seed + rank)
        desc = "uniform random permutation of 0..N-1 (Sec. 6.3 'fully random')"
    if args.key == "u64":
        w = v.astype(np.uint64)
        return (w << np.uint64(32)) | w, desc + ", as u64 keys (v << 32 | v)"
    return v.astype(np.uint32), desc


def verify_sort(work, src, vals, args, N: int) -> bool:
    """Checks one sort of the workload on the device.  Integer inputs whose
    values are 0..N-1 (permutation, sortedness, interleaved at a multiple of
    runs x stride) must sort to iota (v << 32 | v for u64), with the index
    payload becoming the inverse permutation; otherwise the output must be
    non-decreasing (totalOrder for floats) with an unchanged multiset hash."""
    import torch
    dev = work.device
    dense = args.input != "interleaved" or N % (args.runs * args.stride) == 0
    if args.key != "f32" and dense:
        iota = torch.arange(N, dtype=torch.int64, device=dev)
        if args.key == "u64":
            ok = bool(torch.equal(work, (iota << 32) | iota))
            kv = work & 0xFFFFFFFF
        else:
            ok = bool(torch.equal(work.to(torch.int64) & 0xFFFFFFFF, iota))
            kv = src.to(torch.int64) & 0xFFFFFFFF
        if vals is not None and ok:
            if args.key == "u64":
                kv = src & 0xFFFFFFFF
            inv = torch.empty(N, dtype=torch.int64, device=dev)
            inv[kv] = iota
            ok = bool(torch.equal(vals.to(torch.int64) & 0xFFFFFFFF, inv))
        return ok
    if args.key == "f32":
        b = work.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        sb = src.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        ordv = torch.where(b >= 2**31, 0xFFFFFFFF - b, b + 2**31)     # totalOrder on bit patterns
        ok = bool(torch.all(ordv[1:] >= ordv[:-1]))
    elif args.key == "u64":
        b, sb = work, src
        hi, lo = (work >> 32) & 0xFFFFFFFF, work & 0xFFFFFFFF
        ok = bool(torch.all((hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] >= lo[:-1]))))
    else:
        b, sb = work.to(torch.int64) & 0xFFFFFFFF, src.to(torch.int64) & 0xFFFFFFFF
        ok = bool(torch.all(b[1:] >= b[:-1]))
    mix = lambda x: ((x * 0x9E3779B97F4A7C15) ^ (x >> 7)) & 0xFFFFFFFFFFFF
    return ok and bool(mix(b).sum() == mix(sb).sum())


TUNED = os.path.join(ROOT, "paper_1702_07961_gb300", "tuned", "batched_u32_pairs.json")


def verify_batched(work_k, work_v, src_k, off, sizes, chunk=1 << 27):
    """Checks a batched key-value sort completely, on the device, in chunks:
    within every segment keys are non-decreasing (unsigned), every value lies
    in its own segment, keys[i] == source_keys[values[i]], and equal keys have
    strictly increasing values.  Together these force the exact stable result."""
    import torch
    dev = work_k.device
    n = work_k.numel()
    seg = torch.repeat_interleave(torch.arange(sizes.size, dtype=torch.int32, device=dev),
                                  torch.from_numpy(sizes).to(dev), output_size=n)
    ok = True
    for a in range(0, n, chunk):
        b = min(n, a + chunk + 1)
        k = work_k[a:b].to(torch.int64) & 0xFFFFFFFF
        v = work_v[a:b].to(torch.int64) & 0xFFFFFFFF       # uint32 payloads (> 2^31 in big batches)
        sg = seg[a:b]
        same = sg[1:] == sg[:-1]
        ok &= bool(torch.all(~same | (k[1:] >= k[:-1])))
        ok &= bool(torch.all(~same | (k[1:] != k[:-1]) | (v[1:] > v[:-1])))
        ok &= bool(torch.all(seg[v] == sg))
        ok &= bool(torch.all((src_k[v].to(torch.int64) & 0xFFFFFFFF) == k))
        del k, v, sg, same
    del seg
    return ok


def run_batched(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1702_07961_gb300 as mms
    from paper_1702_07961_gb300 import autotune
    import synth

    dev = torch.device("cuda", local)
    # C4: sizes log-uniform in [2^8, 2^20], rounded down to whole 16-byte
    # vectors so every array also suits the whole-array API (16-byte aligned).
    sizes = synth.segment_sizes(args.arrays, 256, 1 << 20, 7 + rank) // 4 * 4
    off_np = synth.offsets_of(sizes)
    N = int(off_np[-1])
    g = torch.Generator(device=dev).manual_seed(1234 + rank)
    src_k = torch.randint(-2**31, 2**31 - 1, (N,), dtype=torch.int32, device=dev, generator=g)
    src_v = torch.arange(N, dtype=torch.int32, device=dev)
    work_k = torch.empty_like(src_k)
    work_v = torch.empty_like(src_v)
    off = torch.from_numpy(off_np).to(dev)

    if os.path.exists(TUNED) and not args.retune:
        table, tile = autotune.load_table(TUNED)
        tuned_from = "paper_1702_07961_gb300/tuned/batched_u32_pairs.json"
    else:
        res = autotune.tune(mms.KEY_U32, True, classes=range(8, 21), weights=autotune.class_weights(sizes))
        table, tile = {int(c): int(k) for c, k in res["class_fanout"].items()}, int(res["tile_items"])
        tuned_from = "autotuner run in this process"
        if rank == 0:
            dest = args.tuned_out or TUNED
            os.makedirs(os.path.dirname(os.path.abspath(dest)), exist_ok=True)
            autotune.save(res, dest)
    mx = int(sizes.max())
    graph = mms.SegmentedGraph(work_k, off, work_v, kt=mms.KEY_U32, class_fanout=table, tile_items=tile,
                               max_segment_items=mx)
    stream = torch.cuda.current_stream()

    def refill():
        work_k.copy_(src_k)
        work_v.copy_(src_v)

    for _ in range(args.warmup):
        refill()
        graph.launch()
    torch.cuda.synchronize()
    mms.workspace_status(graph.workspace)
    verified = verify_batched(work_k, work_v, src_k, off_np, sizes)
    # and a sample of arrays against the CPU oracle
    rng = np.random.default_rng(3)
    for s in rng.choice(sizes.size, size=min(6, sizes.size), replace=False):
        a, b = int(off_np[s]), int(off_np[s + 1])
        want_k, want_v = oracle.sort(src_k[a:b].cpu().numpy().view(np.uint32),
                                     src_v[a:b].cpu().numpy().view(np.uint32))
        verified &= bool(np.array_equal(work_k[a:b].cpu().numpy().view(np.uint32), want_k))
        verified &= bool(np.array_equal(work_v[a:b].cpu().numpy().view(np.uint32), want_v))
    if not verified:
        raise SystemExit("bench: batched output is wrong")

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    for a, b in evs:
        refill()                      # 20 GB device copy, outside the events
        a.record(stream)
        graph.launch(stream)
        b.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms_per_step, value = aggregate_over_ranks(sum(step_ms), N, args.steps, world, dev)

    # The plain path: one whole-array key-value sort per array, in order, on one
    # stream (every array submitted at once, served one after another).
    ws = torch.empty(mms.workspace_bytes(mms.KEY_U32, mx, True), dtype=torch.uint8, device=dev)
    refill()
    torch.cuda.synchronize()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(sizes.size + 1)]
    marks[0].record(stream)
    for s in range(sizes.size):
        a, b = int(off_np[s]), int(off_np[s + 1])
        mms.sort_pairs(work_k[a:b], work_v[a:b], workspace=ws, kt=mms.KEY_U32)
        marks[s + 1].record(stream)
    torch.cuda.synchronize()
    done = np.array([marks[0].elapsed_time(m) for m in marks[1:]])
    plain_ms = float(done[-1])
    plain_ok = verify_batched(work_k, work_v, src_k, off_np, sizes)
    own = np.diff(np.concatenate([[0.0], done]))

    out = {
        "metric": "batched Gkeys/s (20000 arrays)", "value": value, "unit": "Gkeys/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"{sizes.size} independent arrays, sizes log-uniform in [2^8, 2^20] (multiples of 4), "
                               f"{N} uint32 keys in all (uniform, seeded device generator) with uint32 index "
                               "payloads, one CUDA-graph launch of the batched sort per step",
                   "global_batch": N * world, "seq_len": None, "parallelism": f"replicas{world}",
                   "tile_items": tile, "class_fanout": {str(k): v for k, v in sorted(table.items())},
                   "tuned_from": tuned_from, "l2": "inputs 20 GB > 129 MB L2"},
        "batched": {"ms_per_batch": ms_per_step, "latency_ms_p50": ms_per_step, "latency_ms_p99": ms_per_step,
                    "note": "every array of a batch completes with the batch"},
        "plain": {"ms_total": plain_ms, "gkeys_per_s": N / (plain_ms / 1e3) / 1e9,
                  "latency_ms_p50": float(np.percentile(done, 50)), "latency_ms_p99": float(np.percentile(done, 99)),
                  "per_call_ms_p50": float(np.percentile(own, 50)), "per_call_ms_p99": float(np.percentile(own, 99)),
                  "verified": plain_ok,
                  "note": "one mms_sort_pairs call per array on one stream; latency = completion time "
                          "from submitting all arrays at once"},
        "speedup_vs_plain": plain_ms / ms_per_step,
        # plan, scan, descriptors, base case, (splitter, merge) per round, value gather
        "gpu_launches": args.steps * (5 + 2 * mms.segmented_rounds(mms.KEY_U32, mx, True, table, tile)),
        "verified": verified,
        "clocks": sampler.summary(t0, t1),
    }
    graph.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def run_serve(args):
    """C5: Poisson arrivals of sort requests, sizes log-uniform in [2^10, 2^26],
    key type uniform over {u32, u64, f32}, half with uint32 values, 40 GB budget;
    the continuous-batching server against serial plain sorts at swept rates."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1702_07961_gb300 as mms
    from paper_1702_07961_gb300 import serve
    import synth

    count = args.requests
    sizes = synth.segment_sizes(count, 1 << 10, 1 << 26, 11 + rank)
    rng = np.random.default_rng(12 + rank)
    kts = rng.choice([mms.KEY_U32, mms.KEY_U64, mms.KEY_F32], size=count)
    with_vals = rng.random(count) < 0.5
    reqs = []
    for i in range(count):
        n, kt = int(sizes[i]), int(kts[i])
        seed = 1000 * (rank + 1) + i
        keys = (synth.normal_f32(n, seed) if kt == mms.KEY_F32 else
                synth.uniform(n, seed, np.uint64 if kt == mms.KEY_U64 else np.uint32))
        vals = synth.index_payload(n) if with_vals[i] else None
        reqs.append(serve.Request(i, kt, keys, vals, 0.0))
    for r in reqs:
        serve.SortServer.prepare(r)
    total_keys = int(sizes.sum())

    def reset(arrivals):
        for r, a in zip(reqs, arrivals):
            r.arrival, r.start, r.finish = float(a), None, None

    # Serial capacity: every request waiting at t = 0, served one at a time.
    reset(np.zeros(count))
    serve.serve_serial(reqs)                          # warm-up
    reset(np.zeros(count))
    serve.serve_serial(reqs)
    busy = max(r.finish for r in reqs)
    capacity = count / busy
    def bits(t):                                      # compare bit patterns (NaN keys included)
        a = t.numpy()
        return a.view(np.uint64 if a.dtype.itemsize == 8 else np.uint32)

    alone = [(bits(r.out_keys).copy(), None if r.out_values is None else bits(r.out_values).copy())
             for r in reqs]

    srv = serve.SortServer(budget_bytes=40 << 30, slots=args.slots, small_max=args.small_max)
    reset(np.zeros(count))
    srv.run(reqs)                                     # warm-up of the server's kernels and arena
    torch.cuda.synchronize()
    sweep = []
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    t0 = time.time()
    for f in (0.5, 1.0, 2.0, 4.0):
        rate = f * capacity
        arr = serve.poisson_arrivals(count, rate, 77)
        reset(arr)
        g0, c0 = srv.groups, srv.coalesced
        srv.max_inflight = 0
        srv.run(reqs)
        s_srv = serve.summarize(reqs)
        same = all(np.array_equal(bits(r.out_keys), a[0]) and
                   (a[1] is None or np.array_equal(bits(r.out_values), a[1])) for r, a in zip(reqs, alone))
        reset(arr)
        serve.serve_serial(reqs)
        s_ser = serve.summarize(reqs)
        sweep.append({"rate_per_s": rate, "load_vs_serial_capacity": f, "server": s_srv, "serial": s_ser,
                      "groups": srv.groups - g0, "coalesced_requests": srv.coalesced - c0,
                      "max_groups_in_flight": srv.max_inflight, "same_as_alone": same})
    t1 = time.time()
    sampler.stop()
    ok = all(x["same_as_alone"] for x in sweep)
    # a sample of small requests against the CPU oracle
    for r, a in zip(reqs, alone):
        if r.n <= 1 << 16:
            wk, wv = oracle.sort(r.keys, r.values)
            ok &= bool(np.array_equal(a[0], wk.view(a[0].dtype)))
            if wv is not None:
                ok &= bool(np.array_equal(a[1].view(np.uint32), wv))
    if not ok:
        raise SystemExit("bench: served results differ from the same requests served alone")
    top = sweep[-1]
    out = {
        "metric": "served Gkeys/s and p99 latency (Poisson arrivals)", "value": top["server"]["gkeys_per_s"],
        "unit": "Gkeys/s", "n_gpus": 1, "steps": len(sweep), "warmup": 1,
        "ms_per_step": top["server"]["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed(u32,u64,f32)", "data": "synthetic",
        "config": {"workload": f"{count} requests, sizes log-uniform in [2^10, 2^26] ({total_keys} keys), key type "
                               "uniform over {u32, u64, f32}, half with uint32 values, keys from host memory and "
                               "results back to host; Poisson arrivals at 0.5, 1, 2 and 4 times the serial "
                               f"capacity; 40 GB device budget, {args.slots} launch slots, "
                               + (f"requests <= {args.small_max} keys coalesced" if args.small_max > 0
                                  else "no coalescing"),
                   "slots": args.slots, "small_max": args.small_max,
                   "global_batch": total_keys, "seq_len": None, "parallelism": "single GPU",
                   "serial_capacity_req_per_s": capacity},
        "sweep": sweep,
        "latency_ms_p50": top["server"]["latency_ms_p50"], "latency_ms_p99": top["server"]["latency_ms_p99"],
        "serial_latency_ms_p99": top["serial"]["latency_ms_p99"],
        "verified": ok,
        "clocks": sampler.summary(t0, t1),
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def run_configs(args):
    """The paper-shaped configurations beside the headline one: 2^20 uniform
    keys; 10^8 keys by sortedness r (key-only and with index payloads); 2^28
    interleaved stride-32 runs as u32 and u64; 2^28 N(0,1) floats with
    duplicates, -0.0 and NaNs.  Each is sorted `steps` times through the C ABI
    and checked against a closed form, the oracle, or order+multiset."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_1702_07961_gb300 as mms
    import synth
    dev = torch.device("cuda", 0)
    results = []

    def timed(work, src, ws, kt, vals=None, vsrc=None, steps=args.steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(args.warmup + steps):
            work.copy_(src)
            if vals is not None:
                vals.copy_(vsrc)
            if i >= args.warmup:
                evs[i - args.warmup][0].record()
            if vals is None:
                mms.sort_keys(work, workspace=ws, kt=kt)
            else:
                mms.sort_pairs(work, vals, workspace=ws, kt=kt)
            if i >= args.warmup:
                evs[i - args.warmup][1].record()
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    def add(name, n, ms, ok, kt, pairs=False, note=""):
        plan = mms.plan(kt, n, pairs=pairs)
        passes = 1 + len(plan)
        kb = 8 if (pairs or kt == mms.KEY_U64) else 4
        results.append({"config": name, "n": n, "ms": ms, "gkeys_per_s": n / ms / 1e6, "verified": bool(ok),
                        "fanouts": plan, "passes": passes,
                        "hbm_frac_whole_sort": passes * 2 * n * kb / (ms / 1e3) / 1e9 / hbm_peak(), "note": note})

    # C1: 2^20 uniform u32, bit-exact against the oracle
    n = 1 << 20
    keys = synth.uniform(n, 1)
    src = torch.from_numpy(keys.view(np.int32)).to(dev)
    work = torch.empty_like(src)
    ws = torch.zeros(mms.workspace_bytes(mms.KEY_U32, n), dtype=torch.uint8, device=dev)
    ms = timed(work, src, ws, mms.KEY_U32)
    ok = np.array_equal(work.cpu().numpy().view(np.uint32), oracle.sort(keys)[0])
    add("C1 2^20 uniform u32", n, ms, ok, mms.KEY_U32, note="fits in L2")

    # C2: 10^8 by sortedness, key-only and with the index payload (closed forms)
    n = 10**8
    iota = torch.arange(n, dtype=torch.int64, device=dev)
    ws = torch.zeros(mms.workspace_bytes(mms.KEY_U32, n, True), dtype=torch.uint8, device=dev)
    vsrc = torch.arange(n, dtype=torch.int32, device=dev)
    vals = torch.empty_like(vsrc)
    swaps = [0, 10**3, 10**5, 10**7, 10**8, 10**9]
    for r in [x for x in swaps if x <= args.max_swaps] + ["permutation"]:
        keys = synth.permutation(n, 1) if r == "permutation" else synth.sortedness(n, int(r), 2)
        src = torch.from_numpy(keys.view(np.int32)).to(dev)
        work = torch.empty_like(src)
        for pairs in (False, True):
            ms = timed(work, src, ws, mms.KEY_U32, vals if pairs else None, vsrc)
            ok = bool(torch.equal(work.to(torch.int64) & 0xFFFFFFFF, iota))
            if pairs:
                inv = torch.empty(n, dtype=torch.int64, device=dev)
                inv[src.to(torch.int64) & 0xFFFFFFFF] = iota
                ok &= bool(torch.equal(vals.to(torch.int64), inv))
                del inv
            label = "fully random permutation" if r == "permutation" else f"sortedness r={int(r):.0e}"
            add(f"C2 10^8 u32 {label}" + (" + index payload" if pairs else ""), n, ms, ok, mms.KEY_U32, pairs)
        del src, work
    del ws, vals, vsrc, iota
    torch.cuda.empty_cache()

    # C3: 2^28 interleaved stride-32 runs (u32, u64): sorted result is iota
    n = 1 << 28
    for dt, kt in ((np.uint32, mms.KEY_U32), (np.uint64, mms.KEY_U64)):
        keys = synth.interleaved(n, 8, 32, dt)
        src = torch.from_numpy(keys.view(np.int32 if dt == np.uint32 else np.int64)).to(dev)
        work = torch.empty_like(src)
        ws = torch.zeros(mms.workspace_bytes(kt, n), dtype=torch.uint8, device=dev)
        ms = timed(work, src, ws, kt, steps=max(3, args.steps // 3))
        want = torch.arange(n, dtype=torch.int64, device=dev)
        if dt == np.uint64:
            want = (want << 32) | want
            ok = bool(torch.equal(work, want))
        else:
            ok = bool(torch.equal(work.to(torch.int64) & 0xFFFFFFFF, want))
        add(f"C3 2^28 {np.dtype(dt).name} interleaved K=8 stride 32", n, ms, ok, kt)
        del src, work, ws, want
        torch.cuda.empty_cache()
    # C3: 2^28 float32 N(0,1) with 1% duplicates, 0.1% -0.0, 0.01% NaN: totalOrder order + multiset
    keys = synth.normal_f32(n, 3)
    src = torch.from_numpy(keys).to(dev)
    work = torch.empty_like(src)
    ws = torch.zeros(mms.workspace_bytes(mms.KEY_F32, n), dtype=torch.uint8, device=dev)
    ms = timed(work, src, ws, mms.KEY_F32, steps=max(3, args.steps // 3))
    b = work.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    ordv = torch.where(b >= 2**31, b ^ 0xFFFFFFFF, b | 2**31)        # totalOrder on bit patterns
    ok = bool(torch.all(ordv[1:] >= ordv[:-1]))
    sb = src.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    mix = lambda x: ((x * 0x9E3779B97F4A7C15) ^ (x >> 7)) & 0xFFFFFFFFFFFF
    ok &= bool(mix(b).sum() == mix(sb).sum()) and bool((b * b).sum() == (sb * sb).sum())
    add("C3 2^28 f32 N(0,1) + dups, -0.0, NaN", n, ms, ok, mms.KEY_F32,
        note="verified by totalOrder non-decreasing + multiset hash")
    out = {"metric": "Gkeys/s per configuration", "unit": "Gkeys/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "dtype": "u32/u64/f32", "data": "synthetic", "results": results,
           "all_verified": all(r["verified"] for r in results)}
    print(json.dumps(out), flush=True)
    return 0 if out["all_verified"] else 1


def run_sweep(args):
    """Fanout K x size N sweep (the paper's Sec. 6.2 tuning and Sec. 6.3 size
    experiments, on GB300): uniform random u32 and u64 keys from a seeded
    device generator, every K in {2, 4, 8, 16, 32}, sizes 2^20 .. 2^28.  Each
    result is checked for non-decreasing order and an unchanged key sum."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1702_07961_gb300 as mms
    dev = torch.device("cuda", 0)
    rows = []
    for kt, name in ((mms.KEY_U32, "u32"), (mms.KEY_U64, "u64")):
        sizes = [1 << 20, 1 << 22, 1 << 24, 1 << 26, 10**8] + ([1 << 28] if kt == mms.KEY_U32 else [])
        if args.sweep_sizes:
            sizes = [int(float(x)) for x in args.sweep_sizes.split(",")]
        for n in sizes:
            g = torch.Generator(device=dev).manual_seed(n + kt)
            if kt == mms.KEY_U32:
                src = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device=dev, generator=g)
            else:
                src = torch.randint(-2**63, 2**63 - 1, (n,), dtype=torch.int64, device=dev, generator=g)
            work = torch.empty_like(src)
            ws = torch.zeros(mms.workspace_bytes(kt, n), dtype=torch.uint8, device=dev)
            ref_sum = int(src.to(torch.int64).sum().item()) if kt == mms.KEY_U32 else None
            for K in (2, 4, 8, 16, 32):
                plan = mms.plan(kt, n, K)
                n_ev = 2 + 2 * len(plan)
                steps = max(3, min(args.steps, 10))
                evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(steps)]
                for i in range(args.warmup + steps):
                    work.copy_(src)
                    mms.sort_keys(work, fanout=K, workspace=ws, kt=kt,
                                  events=evs[i - args.warmup] if i >= args.warmup else None)
                torch.cuda.synchronize()
                if kt == mms.KEY_U32:
                    w = work.to(torch.int64) & 0xFFFFFFFF
                    ok = bool(torch.all(w[1:] >= w[:-1])) and int(work.to(torch.int64).sum().item()) == ref_sum
                else:
                    hi = (work >> 32) & 0xFFFFFFFF
                    lo = work & 0xFFFFFFFF
                    ok = bool(torch.all((hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] >= lo[:-1]))))
                    ok &= bool(torch.equal(torch.sort(work).values, torch.sort(src).values))
                st = [[e[k].elapsed_time(e[k + 1]) for k in range(n_ev - 1)] for e in evs]
                tot = statistics.median(e[0].elapsed_time(e[-1]) for e in evs)
                merge = [statistics.mean(x[2 + 2 * r] for x in st) for r in range(len(plan))]
                split_r = [statistics.mean(x[1 + 2 * r] for x in st) for r in range(len(plan))]
                split = sum(split_r)
                # runs merged per group in each round: K, except in a last round with fewer runs left
                runs = -(-n // mms.base_run_items(kt, n))
                merged = []
                for k in plan:
                    merged.append(min(k, runs))
                    runs = -(-runs // k)
                kb = 8 if kt == mms.KEY_U64 else 4
                rows.append({"key": name, "n": n, "K": K, "rounds": len(plan), "ms": tot,
                             "gkeys_per_s": n / tot / 1e6, "tile_sort_ms": statistics.mean(x[0] for x in st),
                             "merge_pass_ms_avg": statistics.mean(merge) if merge else None,
                             "merge_pass_hbm_frac": (2 * n * kb / (statistics.mean(merge) / 1e3) / 1e9 / hbm_peak())
                             if merge else None,
                             "splitters_ms": split, "merge_pass_ms": merge, "splitter_ms": split_r,
                             "runs_merged": merged, "verified": ok})
            del src, work, ws
            torch.cuda.empty_cache()
    print(json.dumps({"metric": "Gkeys/s by fanout and size", "unit": "Gkeys/s", "n_gpus": 1,
                      "data": "synthetic", "rows": rows, "all_verified": all(r["verified"] for r in rows)}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "configs":
        return run_configs(args)
    if args.workload == "sweep":
        return run_sweep(args)
    import numpy as np
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1702_07961_gb300 as mms
    import synth

    dev = torch.device("cuda", local)
    N = args.n
    kt = {"u32": mms.KEY_U32, "u64": mms.KEY_U64, "f32": mms.KEY_F32}[args.key]
    kb = 8 if args.key == "u64" else 4
    keys_np, input_desc = make_sort_input(args, N, rank)
    host_view = keys_np.view(np.int64 if kb == 8 else (np.float32 if args.key == "f32" else np.int32))
    src = torch.from_numpy(host_view).to(dev)
    work = torch.empty_like(src)
    vals = torch.empty(N, dtype=torch.int32, device=dev)
    iota32 = torch.arange(N, dtype=torch.int32, device=dev)
    ws = torch.zeros(mms.workspace_bytes(kt, N, args.pairs), dtype=torch.uint8, device=dev)
    base_items = 0 if args.pairs else args.base_items
    plan = mms.plan(kt, N, args.fanout, args.tile, pairs=args.pairs, base_items=base_items)
    base_run = (mms.base_run_items(mms.KEY_U64, N, args.tile) if args.pairs
                else mms.base_run_items(kt, N, args.tile, base_items))
    base_kernel = "tile_sort_kernel" if base_run == (args.tile or mms.tile_items(kt)) else "tile_sort_cluster_kernel"
    n_ev = 2 + 2 * len(plan) + (1 if args.pairs else 0)
    stream = torch.cuda.current_stream()
    mv = {"partition": mms.MERGE_PARTITION, "pipelined": mms.MERGE_PIPELINED}.get(args.merge_variant,
                                                                                  mms.MERGE_TREE)

    def step(events=None, bounds=None):
        work.copy_(src)
        if args.pairs:
            vals.copy_(iota32)
        if bounds:
            bounds[0].record(stream)
        if args.pairs:
            mms.sort_pairs(work, vals, fanout=args.fanout, workspace=ws, kt=kt, events=events,
                           tile_items=args.tile, merge_variant=mv)
        else:
            mms.sort_keys(work, fanout=args.fanout, workspace=ws, kt=kt, events=events,
                          tile_items=args.tile, merge_variant=mv, base_items=base_items)
        if bounds:
            bounds[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    verified = verify_sort(work, src, vals if args.pairs else None, args, N)
    mms.workspace_status(ws)
    if not verified:
        raise SystemExit("bench: sorted output is wrong")

    # Timed windows of exactly K steps each (barrier + synchronize on both
    # sides, max over ranks), repeated until they span --min-timed-s seconds so
    # that the clock record and the median rest on more than a few ms.
    # Each step's events bracket the sort call only (the input restore is
    # outside them); no event sits between the sort's own kernels, so each
    # splitter and merge pass can launch programmatically behind the kernel
    # before it.  Per-kernel times come from separate steps (below).
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    time.sleep(0.5)
    windows = []
    t0 = time.time()
    while True:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for s_ in range(args.steps):
            step(bounds=evs[s_])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        windows.append(aggregate_over_ranks(sum(step_ms), N, args.steps, world, dev))
        spent = sum(w[0] for w in windows) * args.steps / 1e3
        # every rank takes the same decision: the window times are max-reduced
        if spent >= args.min_timed_s or len(windows) >= 200:
            break
    t1 = time.time()
    sampler.stop()
    mms.workspace_status(ws)
    if not verify_sort(work, src, vals if args.pairs else None, args, N):
        raise SystemExit("bench: sorted output is wrong after the timed windows")
    order = sorted(range(len(windows)), key=lambda i: windows[i][0])
    ms_per_step, value = windows[order[len(order) // 2]]          # the median window

    # Per-kernel times: steps with an event after every kernel (which keeps
    # each kernel from launching before the previous one has finished).
    prof = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(20)]
    for e in prof:
        step(events=e)
    torch.cuda.synchronize()
    stage = [[e[i].elapsed_time(e[i + 1]) for i in range(n_ev - 1)] for e in prof]
    staged_ms = statistics.median(e[0].elapsed_time(e[-1]) for e in prof)

    # per-kernel averages over every timed step: [tile_sort, (splitter, merge) per round,
    # (value gather for pairs)]
    avg = [statistics.mean(s_[i] for s_ in stage) for i in range(n_ev - 1)]
    tile_ms = avg[0]
    split_ms = [avg[1 + 2 * r] for r in range(len(plan))]
    merge_ms = [avg[2 + 2 * r] for r in range(len(plan))]
    gather_ms = avg[-1] if args.pairs else None
    # algorithmic bytes of one pass: every key (8-byte composite for pairs) read and written once
    item_bytes = 8 if args.pairs else kb
    bytes_pass = 2 * N * item_bytes
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    merge_avg = statistics.mean(merge_ms) if merge_ms else None
    totals = {"tile_sort": tile_ms, "splitter": sum(split_ms), "merge_pass": sum(merge_ms)}
    if gather_ms is not None:
        totals["pairs_finalize"] = gather_ms
    dominant = max(totals, key=totals.get)
    if merge_avg:
        achieved = bytes_pass / (merge_avg / 1e3) / 1e9
    else:
        achieved = bytes_pass / (tile_ms / 1e3) / 1e9
    headline = (args.key == "u32" and not args.pairs and args.input == "permutation"
                and args.merge_variant == "tree")
    partition_run = args.merge_variant != "tree" and args.key == "u32" and not args.pairs
    traffic = load_traffic(N, "merge_pass_kernel") if headline and merge_avg else None
    roofline = {"bound": "hbm", "kernel": "merge_pass" if merge_avg else "tile_sort",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_src, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one merge_pass_kernel "
                                  "launch at this workload (profiles/merge_pass_traffic.json)" if traffic else None,
                "algorithmic_bytes_per_launch": bytes_pass,
                "per_pass_frac": [bytes_pass / (m / 1e3) / 1e9 / peak for m in merge_ms],
                "tile_sort_frac": bytes_pass / (tile_ms / 1e3) / 1e9 / peak}
    if headline:
        roofline["tile_sort_traffic"] = load_traffic(N, base_kernel)

    out = {
        "metric": METRIC if headline else (f"Gkeys/s at {N} {args.key}" + (" pairs" if args.pairs else "")
                                           + (f" ({args.merge_variant} merge)" if args.merge_variant != "tree" else "")),
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.key, "data": "synthetic",
        "config": {"workload": f"{input_desc}, N={N} {args.key} keys, "
                               + ("key + uint32 index payload (stable)" if args.pairs else "key-only")
                               + ", one sort per step",
                   "global_batch": N * world, "seq_len": None, "parallelism": f"replicas{world}",
                   "plan_fanouts": plan, "tile": args.tile or mms.tile_items(kt),
                   "base_run": base_run, "base_kernel": base_kernel,
                   "merge_variant": args.merge_variant, "seed": args.seed + rank,
                   "l2": f"input {N * kb / 1e6:.0f} MB > 129 MB L2; a device copy restores the input "
                         "before every step, outside the timed events" if N * kb > 129e6 else
                         "input fits in L2"},
        "timed_windows": {"count": len(windows), "steps_each": args.steps,
                          "gkeys_per_s": [w[1] for w in windows],
                          "mean": statistics.mean(w[1] for w in windows),
                          "min": min(w[1] for w in windows), "max": max(w[1] for w in windows),
                          "note": "value and ms_per_step are the median window's"},
        "stages_ms": {"tile_sort": tile_ms, "splitter": split_ms, "merge_pass": merge_ms,
                      "pairs_finalize": gather_ms, "dominant": dominant,
                      "sort_ms_with_an_event_after_every_kernel": staged_ms,
                      "note": "per-kernel means over 20 further steps that record an event after every "
                              "kernel; the timed steps record events only around the sort call"},
        "roofline": roofline,
        "gpu_launches": len(windows) * args.steps * (1 + 2 * len(plan) + (1 if args.pairs else 0)),
        "gpu_launches_note": "kernels of the timed windows: base case, splitter and merge pass per round"
                             + (", value gather" if args.pairs else ""),
        "verified_vs_closed_form": verified,
        "clocks": sampler.summary(t0, t1),
    }

    # The per-pass roofline depends on the fanout: a pass of fanout K runs
    # ceil(log2 K) on-chip tree levels per HBM read and write.  Measure the
    # merge pass alone at K = 2 and K = 4 too (same workload, same timing).
    by_k = {}
    if headline or partition_run:
        for kf in ((2, 4) if headline else (2, 4, 8, 16)):
            planf = mms.plan(kt, N, kf, args.tile, base_items=base_items)
            nf = 2 + 2 * len(planf)
            evf = [[torch.cuda.Event(enable_timing=True) for _ in range(nf)] for _ in range(10)]
            for i in range(13):
                work.copy_(src)
                mms.sort_keys(work, fanout=kf, workspace=ws, kt=kt, tile_items=args.tile, base_items=base_items,
                              events=evf[i - 3] if i >= 3 else None, merge_variant=mv)
            torch.cuda.synchronize()
            # merge pass of round r: from event 2 + 2r (after its splitter) to 3 + 2r
            mf = statistics.mean(statistics.mean(e[2 + 2 * r].elapsed_time(e[3 + 2 * r])
                                                 for r in range(len(planf)))
                                 for e in evf)
            okf = verify_sort(work, src, None, args, N)
            by_k[str(kf)] = {"merge_pass_ms": mf, "frac": bytes_pass / (mf / 1e3) / 1e9 / peak,
                             "sort_ms": statistics.mean(e[0].elapsed_time(e[-1]) for e in evf), "verified": okf}
        roofline["per_pass_frac_by_fanout"] = by_k

    if not args.no_e2e and headline:
        # End to end through the public API, as a three-stage pipeline: every
        # step uploads its input from pinned host memory (upload stream), sorts
        # it with mms_sort_keys (compute stream, one sort after another), and
        # downloads the result to pinned host memory (download stream).  Events
        # order each step's three stages, and a buffer slot is reused only after
        # its previous download has finished, so uploads and downloads of other
        # steps overlap the sorts.  --e2e-slots device buffers are in flight.
        # The one-at-a-time figure (upload, sort, download, wait) is reported
        # beside.
        h_in = torch.from_numpy(keys_np.view(np.int32)).pin_memory()
        iota_np = np.arange(N, dtype=np.uint32)
        ns = max(2, args.e2e_slots)
        up, comp, down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        bufs = [work] + [torch.empty_like(work) for _ in range(ns - 1)]
        outs = [torch.empty_like(h_in).pin_memory() for _ in range(ns)]
        freed = [None] * ns                                  # download of the slot's last step done
        last = [None] * ns

        def e2e_step(i):
            j = i % ns
            loaded, sorted_ = torch.cuda.Event(), torch.cuda.Event()
            done = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(up):
                if freed[j] is not None:
                    up.wait_event(freed[j])
                bufs[j].copy_(h_in, non_blocking=True)
                loaded.record(up)
            with torch.cuda.stream(comp):
                comp.wait_event(loaded)
                mms.sort_keys(bufs[j], fanout=args.fanout, workspace=ws, kt=mms.KEY_U32,
                              tile_items=args.tile, stream=comp, base_items=args.base_items)
                sorted_.record(comp)
            with torch.cuda.stream(down):
                down.wait_event(sorted_)
                outs[j].copy_(bufs[j], non_blocking=True)
                done.record(down)
            freed[j] = done
            last[j] = i

        torch.cuda.synchronize()
        for i in range(2 * ns):                             # warm-up of every slot
            e2e_step(i)
        torch.cuda.synchronize()
        n_e2e = max(12, args.steps // 2)
        e2e_windows = []
        ok = True
        for w in range(7):
            start = torch.cuda.Event(enable_timing=True)
            start.record(up)
            comp.wait_event(start)
            down.wait_event(start)
            for i in range(n_e2e):
                e2e_step(i)
            end = torch.cuda.Event(enable_timing=True)
            end.record(down)                                # the last step's download is the last work
            torch.cuda.synchronize()
            e2e_windows.append(start.elapsed_time(end) / n_e2e)
            ok = ok and all(bool(np.array_equal(o.numpy().view(np.uint32), iota_np)) for o in outs)
            if w >= 2 and sum(e2e_windows) * n_e2e / 1e3 >= args.min_timed_s:
                break
        pipe_ms = statistics.median(e2e_windows)
        # one at a time: upload, sort, download, then the next step
        ser = []
        for i in range(max(3, args.steps // 10)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(comp)
            with torch.cuda.stream(comp):
                bufs[0].copy_(h_in, non_blocking=True)
                mms.sort_keys(bufs[0], fanout=args.fanout, workspace=ws, kt=mms.KEY_U32,
                              tile_items=args.tile, stream=comp, base_items=args.base_items)
                outs[0].copy_(bufs[0], non_blocking=True)
            b.record(comp)
            torch.cuda.synchronize()
            ser.append(a.elapsed_time(b))
        ser_ms = statistics.mean(ser)
        ok = ok and bool(np.array_equal(outs[0].numpy().view(np.uint32), iota_np))
        # The copies alone, for the record of which stage bounds the pipeline:
        # host copy bandwidth on this machine varies between and within runs.
        def copy_ms(fn):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ts = []
            for _ in range(3):
                a.record(comp)
                with torch.cuda.stream(comp):
                    fn()
                b.record(comp)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.median(ts)
        h2d_ms = copy_ms(lambda: bufs[0].copy_(h_in, non_blocking=True))
        d2h_ms = copy_ms(lambda: outs[0].copy_(bufs[0], non_blocking=True))
        out["e2e"] = {"value": N / (pipe_ms / 1e3) / 1e9 * world, "unit": UNIT,
                      "h2d_bytes_per_step": N * KEY_BYTES, "d2h_bytes_per_step": N * KEY_BYTES,
                      "ms_per_step": pipe_ms, "steps": n_e2e,
                      "windows_gkeys_per_s": [N / (m / 1e3) / 1e9 * world for m in e2e_windows],
                      "verified_last_output_of_every_slot": ok,
                      "mode": f"pipeline: upload, sort and download streams, {ns} device buffers in flight; "
                              "sorts back to back, copies overlapping them",
                      "one_at_a_time": {"value": N / (ser_ms / 1e3) / 1e9 * world, "ms_per_step": ser_ms},
                      "copies_alone": {"h2d_ms": h2d_ms, "d2h_ms": d2h_ms,
                                       "h2d_gbs": N * KEY_BYTES / (h2d_ms / 1e3) / 1e9,
                                       "d2h_gbs": N * KEY_BYTES / (d2h_ms / 1e3) / 1e9,
                                       "note": "the pipeline is bound by max(sort, upload, download) per step"}}
        del bufs, outs

    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = time_oracle(keys_np, min(args.cpu_sample, N))
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
