"""Autotuner of the batched sort: picks the merge fanout K for every size
class (ceil(log2 n) of a segment's length) and the tile width, by measuring.

The paper tunes its parameters per platform by measurement (Sec. 6.2: the
fanout K and the base-case size are chosen from timed runs at a fixed input
size).  Here the same idea is applied per size class of a batch: for each
class c whose segments need merge rounds, a synthetic batch of segments with
lengths log-uniform in (2^(c-1), 2^c] is sorted with every candidate K for
that class, and the fastest K is kept.  Each tile width supported for the key
type is tuned this way, and the width whose classes sum to the least time
(weighted by the share of keys a workload puts in each class) wins.

The result is a plain dict usable as ``class_fanout``/``tile_items`` of
:func:`paper_1702_07961_gb300.segmented_sort`, and can be written to JSON.
"""
from __future__ import annotations

import json
import math
import statistics

import numpy as np

import synth

from . import KEY_F32, KEY_U32, KEY_U64, SegmentedGraph, segmented_rounds

CANDIDATE_K = (2, 4, 8, 16, 32)


def tile_options(kt: int, pairs: bool):
    return (2048, 4096) if (pairs or kt == KEY_U64) else (4096, 8192)


def class_batch(c: int, total: int, seed: int):
    """Sizes log-uniform in (2^(c-1), 2^c], about `total` items in all."""
    lo, hi = (1 << (c - 1)) + 1, 1 << c
    mean = (hi - lo) / max(math.log(hi / lo), 1e-9) if hi > lo else hi
    count = max(8, int(total / mean))
    return synth.segment_sizes(count, lo, hi, seed)


def _time_batch(keys, offsets, values, kt, table, tile, reps, warmup):
    import torch
    g = SegmentedGraph(keys, offsets, values, kt=kt, class_fanout=table, tile_items=tile,
                       max_segment_items=int((offsets[1:] - offsets[:-1]).max().item()))
    src_k = keys.clone()
    src_v = None if values is None else values.clone()
    ts = []
    for i in range(warmup + reps):
        keys.copy_(src_k)
        if values is not None:
            values.copy_(src_v)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.launch()
        b.record()
        torch.cuda.synchronize()
        if i >= warmup:
            ts.append(a.elapsed_time(b))
    g.close()
    return statistics.median(ts)


def tune(kt: int = KEY_U32, pairs: bool = False, classes=range(8, 21), weights=None,
         items_per_class: int = 1 << 24, reps: int = 3, warmup: int = 1, seed: int = 1,
         candidates=CANDIDATE_K, tiles=None, device="cuda"):
    """Measures and returns {"tile_items": T, "class_fanout": {c: K}, "ms": {...}}.

    ``weights``: share of a workload's keys in each class (default: equal).
    """
    import torch
    tiles = tiles or tile_options(kt, pairs)
    best = None
    report = {}
    for tile in tiles:
        table = {}
        total_ms = 0.0
        per = {}
        for c in classes:
            # A class whose segments fit one tile runs no merge round: its K does
            # not matter, but its time still counts towards the tile width's total.
            cands = candidates if segmented_rounds(kt, 1 << c, pairs, None, tile) > 0 else (0,)
            sizes = class_batch(c, items_per_class, seed + c)
            off = torch.from_numpy(synth.offsets_of(sizes)).to(device)
            n = int(off[-1].item())
            g = torch.Generator(device=device).manual_seed(seed * 1000 + c)
            if kt == KEY_U64:
                keys = torch.randint(-2**63, 2**63 - 1, (n,), dtype=torch.int64, device=device, generator=g)
            elif kt == KEY_F32:
                keys = torch.randn((n,), dtype=torch.float32, device=device, generator=g)
            else:
                keys = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device=device, generator=g)
            values = torch.arange(n, dtype=torch.int32, device=device) if pairs else None
            times = {}
            for K in cands:
                times[K] = _time_batch(keys, off, values, kt, {c: K} if K else None, tile, reps, warmup)
            k_best = min(times, key=times.get)
            if k_best:
                table[c] = k_best
            w = 1.0 if weights is None else float(weights.get(c, 0.0))
            # time per item of the class, weighted by the workload's share of items
            total_ms += w * times[k_best] / n
            per[c] = {"K": k_best, "ms": times, "items": n}
            del keys, values, off
        report[tile] = {"class_fanout": table, "weighted_ms_per_item": total_ms, "classes": per}
        if best is None or total_ms < report[best]["weighted_ms_per_item"]:
            best = tile
    return {"tile_items": best, "class_fanout": report[best]["class_fanout"] if best else {},
            "key_type": kt, "pairs": bool(pairs), "measured": {str(t): r for t, r in report.items()}}


def class_weights(sizes) -> dict:
    """Share of a workload's items in each size class."""
    sizes = np.asarray(sizes, dtype=np.int64)
    cls = np.ceil(np.log2(np.maximum(sizes, 1))).astype(int)
    tot = float(sizes.sum())
    return {int(c): float(sizes[cls == c].sum()) / tot for c in np.unique(cls)}


def save(result: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(result, f, indent=1, sort_keys=True)


def load_table(path: str):
    with open(path) as f:
        r = json.load(f)
    return {int(c): int(k) for c, k in r["class_fanout"].items()}, int(r["tile_items"])


def fit_plan_costs(rows, n: int = 10**8) -> dict:
    """Per-round costs of the whole-array planner, from `bench.py --workload
    sweep` rows: for each key width and K in CANDIDATE_K, the mean time of a
    round (splitter + merge pass) over the rounds that merged K runs per group,
    in ms per 10^8 items.  A plan's last round often merges fewer runs than its
    K (fewer tree levels, so cheaper) and is left out, so that the cost of a
    full round is not underestimated.  Returns {"u32": [...], "u64": [...]}
    in the order of CANDIDATE_K (the planner's kCost4 / kCost8)."""
    out = {}
    for key in ("u32", "u64"):
        costs = []
        for K in CANDIDATE_K:
            vals = []
            for r in rows:
                if r["key"] != key or r["n"] != n or r["K"] != K:
                    continue
                for m, s, runs in zip(r["merge_pass_ms"], r["splitter_ms"], r["runs_merged"]):
                    if runs == K:
                        vals.append((m + s) * 1e8 / n)
            costs.append(statistics.mean(vals) if vals else None)
        out[key] = costs
    return out
