"""Autotuner for the tensor-core tiling of a plan.

The paper tuned its kernel's two compile-time parameters (accumulators per
thread, threads per block) by timing a grid of combinations on the target GPU
(Section 2.2, Fig. 1).  The tensor-core kernel here has three runtime tiling
parameters, set through ``bf_plan_set_tiles``:

  tile_t       samples per tile (the MMA N dimension), a multiple of
               lcm(16, T_int) up to 256;
  group_tiles  128-row weight tiles (64 beams each) kept resident in shared
               memory while a CTA walks along time; fewer groups per channel
               means fewer re-reads of each voltage tile;
  x_stages     voltage tiles in flight (TMA prefetch depth).

``tune`` times every feasible combination on the caller's input with CUDA
events on the plan's stream, applies the fastest and records it in a JSON
cache keyed by the problem shape, so later plans of the same shape start from
the tuned choice (``apply_cached``).
"""
from __future__ import annotations

import json
import math
import os

from . import (BF_C32, BFError, bf_execute, bf_plan_query_tiles, bf_plan_set_tiles)

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1412_4907_gb300", "tiles.json")


def shape_key(plan, n_samp: int) -> str:
    return f"N{plan.N}_B{plan.B}_C{plan.C}_T{n_samp}_Ti{plan.t_int}_d{plan.dtype}"


def candidates(plan, max_tiles: int = 16):
    """Feasible (tile_t, group_tiles, x_stages) triples, largest tiles first."""
    unit = 16 * plan.t_int // math.gcd(16, plan.t_int)
    tiles = [t for t in range(256, unit - 1, -16) if t % unit == 0 and t // plan.t_int <= 16][:3]
    m_tiles = (plan.B + 63) // 64
    groups = sorted({g for g in (m_tiles, 16, 12, 8, 6, 5, 4, 3, 2, 1) if 1 <= g <= min(m_tiles, max_tiles)},
                    reverse=True)
    out = []
    for t in tiles:
        for xs in (2, 3, 4):
            for g in groups:
                try:
                    bf_plan_set_tiles(plan.handle, t, g, xs)
                except BFError:
                    continue
                q = bf_plan_query_tiles(plan.handle)
                key = (q["tile_t"], q["group_tiles"], q["x_stages"])
                if key not in out:
                    out.append(key)
    bf_plan_set_tiles(plan.handle, 0, 0, 0)
    return out


def time_config(plan, x, n_samp: int, out, reps: int = 5) -> float:
    """Mean milliseconds of one bf_execute with the plan's current tiling."""
    import torch
    s = plan.stream
    for _ in range(2):
        bf_execute(plan.handle, x.data_ptr(), n_samp, out.data_ptr(), s.cuda_stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        bf_execute(plan.handle, x.data_ptr(), n_samp, out.data_ptr(), s.cuda_stream)
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune(plan, x, n_samp: int, out=None, reps: int = 5, cache: str | None = DEFAULT_CACHE,
         verbose: bool = False) -> dict:
    """Time every candidate tiling on input ``x`` (device tensor in the plan's
    layout), apply the fastest, and return {"config": ..., "ms": ..., "table": [...]}."""
    import torch
    if plan.dtype == BF_C32:
        return {"config": None, "ms": None, "table": []}
    if out is None:
        out = torch.empty((plan.B, plan.C, n_samp // plan.t_int), dtype=torch.float32, device=x.device)
    table = []
    for t, g, xs in candidates(plan):
        bf_plan_set_tiles(plan.handle, t, g, xs)
        ms = time_config(plan, x, n_samp, out, reps)
        table.append({"tile_t": t, "group_tiles": g, "x_stages": xs, "ms": ms})
        if verbose:
            print(f"tile_t={t:3d} group_tiles={g:2d} x_stages={xs}: {ms:.3f} ms", flush=True)
    best = min(table, key=lambda r: r["ms"])
    bf_plan_set_tiles(plan.handle, best["tile_t"], best["group_tiles"], best["x_stages"])
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = json.load(open(cache)) if os.path.exists(cache) else {}
        data[shape_key(plan, n_samp)] = {k: best[k] for k in ("tile_t", "group_tiles", "x_stages")}
        tmp = cache + f".tmp{os.getpid()}"
        json.dump(data, open(tmp, "w"), indent=1)
        os.replace(tmp, cache)
    return {"config": {k: best[k] for k in ("tile_t", "group_tiles", "x_stages")}, "ms": best["ms"],
            "table": table}


def apply_cached(plan, n_samp: int, cache: str | None = DEFAULT_CACHE) -> bool:
    """Apply a cached tiling for this shape if one exists."""
    if not cache or not os.path.exists(cache):
        return False
    cfg = json.load(open(cache)).get(shape_key(plan, n_samp))
    if not cfg:
        return False
    bf_plan_set_tiles(plan.handle, cfg["tile_t"], cfg["group_tiles"], cfg["x_stages"])
    return True


# ------------------------------------------------------------ batched launch
def batch_key(plans, n_samps) -> str:
    """Cache key of a batch: T_int, operand dtype and the sorted job shapes."""
    shapes = sorted((p.N, p.B, p.C, int(t)) for p, t in zip(plans, n_samps))
    h = hash(tuple(shapes)) & 0xFFFFFFFF
    return f"batch_Ti{plans[0].t_int}_d{plans[0].dtype}_n{len(plans)}_{h:08x}"


def batch_candidates(t_int: int):
    unit = 16 * t_int // math.gcd(16, t_int)
    return [t for t in range(256, unit - 1, -16) if t % unit == 0 and t // t_int <= 16]


def time_batch(batch, reps: int = 5) -> float:
    """Mean milliseconds of one graph replay of a bound, captured batch."""
    import torch
    s = batch.stream
    for _ in range(2):
        batch.replay()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        batch.replay()
    b.record(s)
    b.synchronize()
    batch.sync()
    return a.elapsed_time(b) / reps


def tune_batch(plans, xs, outs, n_samps=None, stream=None, reps: int = 5, cache: str | None = DEFAULT_CACHE,
               verbose: bool = False) -> dict:
    """Time the batched launch of ``plans`` on inputs ``xs`` (outputs ``outs``)
    for every feasible tile width, and return {"tile_t", "ms", "table"}; the
    choice is cached under the batch's shape key."""
    from . import Batch
    if n_samps is None:
        n_samps = [p.n_samp(x) for p, x in zip(plans, xs)]
    table = []
    for t in batch_candidates(plans[0].t_int):
        try:
            batch = Batch(plans, tile_t=t, stream=stream)
        except BFError:
            continue
        for j, (x, o, T) in enumerate(zip(xs, outs, n_samps)):
            batch.set(j, x, o, n_samp=T)
        batch.capture()
        ms = time_batch(batch, reps)
        batch.close()
        table.append({"tile_t": t, "ms": ms})
        if verbose:
            print(f"batch tile_t={t:3d}: {ms:.3f} ms", flush=True)
    best = min(table, key=lambda r: r["ms"])
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = json.load(open(cache)) if os.path.exists(cache) else {}
        data[batch_key(plans, n_samps)] = {"tile_t": best["tile_t"]}
        tmp = cache + f".tmp{os.getpid()}"
        json.dump(data, open(tmp, "w"), indent=1)
        os.replace(tmp, cache)
    return {"tile_t": best["tile_t"], "ms": best["ms"], "table": table}
