"""Autotuner for the pair-area launch parameters.

Picks, by timing on the resident sets and candidate pairs it is given, the sampling-box threshold T
(Sec. 3.4: where subdivision stops and a box is pixelized), the work-item size of the persistent
form (split_pixels: how many warps a large pair is spread over) and the warps per CTA (how many
pairs or items share an SM slot). Every candidate runs the real kernels through the library (CUDA
events on the launching stream, median of a few launches after warm-up); results are identical for
every setting, so the tuner only compares times. The search first tries a short list of (item size,
T) pairs, the two parameters that together decide which kernel runs (one-leaf items stream their
edges; larger ones are subdivided), then a coordinate descent: T over a log grid, split_pixels,
warps per CTA and, where the items are leaves of at most 64 x 64 pixels, the threads per pair
(one warp per item, or one lane per small pair), each with the others fixed at their best so far.

`tune(ctx, A, B, pa, pb)` returns the best parameters and the timing table; `load`/`save` keep
results in a JSON file keyed by a workload signature, so that a serving process or a benchmark can
reuse them.
"""
from __future__ import annotations

import json
import math
import os
import statistics

from . import MODE_PERSISTENT, MODE_PLAIN

T_GRID = (2048, 4096, 8192, 16384, 65536)
SPLIT_GRID = (1024, 2048, 4096, 16384)
WPC_GRID = (2, 4, 8)
LANES_GRID = (32, 1)       # threads per pair in the leaf path: one warp per item, or one lane per small pair
# threads per pair with rasters: pairs of more (row, 32-pixel word) units than this get a CTA (-1: none)
HEAVY_GRID = (-1, 256, 1024, 4096, 16384)
CTAS_GRID = (0, 4, 8)      # resident CTAs per SM (0: occupancy maximum)
RASTER_LANES_GRID = (1, 8, 16, 32)   # threads per light pair with rasters
# Work-item forms of the persistent queue, (split_pixels, T): items of split_pixels pixels are one
# leaf each when split_pixels < T (streamed: windows up to 64 x 64 through the leaf kernel, larger
# ones through the streamed kernel), otherwise they are subdivided into sampling boxes (staged
# kernels). The item size and T decide together which kernel runs, so they are searched as pairs.
FORM_GRID = ((1024, 8192), (2048, 8192), (4096, 8192), (4096, 16384), (16384, 65536), (65536, 262144),
             (4096, 2048), (16384, 8192))


def _time(ctx, fn, reps: int, warm: int) -> float:
    import torch
    ts = []
    for r in range(warm + reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        if r >= warm:
            ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune(ctx, A, B, pa, pb, mode: int = MODE_PERSISTENT, reps: int = 3, warm: int = 1,
         t_grid=T_GRID, split_grid=SPLIT_GRID, wpc_grid=WPC_GRID, form_grid=FORM_GRID,
         lanes_grid=LANES_GRID, heavy_grid=HEAVY_GRID) -> dict:
    """For the persistent form, the best (split_pixels, T) pair of form_grid first; then coordinate
    descent over T, split_pixels (persistent form only) and warps_per_cta for the pair areas of
    (pa, pb). When both sets keep pixel rasters (and the context uses them), the persistent form's
    pair areas AND rasters instead, and the search is over the threads per pair (raster_lanes, and
    raster_heavy: which pairs get a whole CTA) and resident CTAs per SM. Leaves ctx set to the best parameters. Returns
    {"params": {...}, "ms": best, "table": [(params, ms), ...]}."""
    import torch
    n = pa.numel()
    inter = torch.empty(max(n, 1), dtype=torch.int64, device=pa.device)
    uni = torch.empty_like(inter)
    best = dict(ctx.params())
    table = []

    def run(params):
        for k, v in params.items():
            ctx.set_param(k, v)
        ms = _time(ctx, lambda: ctx.pair_areas(A, B, pa, pb, mode=mode, out=(inter, uni)), reps, warm)
        table.append((dict(params), round(ms, 4)))
        return ms

    if best.get("rasters") and A.raster is not None and B.raster is not None and mode == MODE_PERSISTENT:
        # pair areas from rasters: the choices are how many threads a pair gets (8, 16 or 32 lanes, or
        # a whole CTA for pairs of more than raster_heavy (row, word) units), and resident CTAs per SM
        keys = ("raster_lanes", "raster_heavy", "ctas_per_sm")
        best_ms = run({k: best[k] for k in keys})
        tried = {tuple(best[k] for k in keys)}
        for name, grid in (("raster_lanes", RASTER_LANES_GRID), ("raster_heavy", heavy_grid), ("ctas_per_sm", CTAS_GRID)):
            for v in grid:
                trial = {k: best[k] for k in keys} | {name: v}
                if tuple(trial[k] for k in keys) in tried:
                    continue
                tried.add(tuple(trial[k] for k in keys))
                ms = run(trial)
                if ms < best_ms:
                    best_ms, best = ms, dict(best, **trial)
        for k in keys:
            ctx.set_param(k, best[k])
        return {"params": {k: best[k] for k in keys}, "ms": round(best_ms, 4), "mode": "persistent (rasters)",
                "table": table}
    keys = ("T", "split_pixels", "warps_per_cta", "pair_lanes")
    best_ms = run({k: best[k] for k in keys})
    if mode == MODE_PERSISTENT:
        for split, T in form_grid:
            if (split, T) == (best["split_pixels"], best["T"]):
                continue
            trial = {k: best[k] for k in keys} | {"T": T, "split_pixels": split}
            ms = run(trial)
            if ms < best_ms:
                best_ms, best = ms, dict(best, **trial)
    axes = [("T", t_grid)]
    if mode == MODE_PERSISTENT:
        axes.append(("split_pixels", split_grid))
    axes.append(("warps_per_cta", wpc_grid))
    side = math.isqrt(max(best["split_pixels"], 1))
    if mode == MODE_PERSISTENT and side <= 64 and side * side < best["T"]:
        axes.append(("pair_lanes", lanes_grid))        # only the leaf path has the choice
    for name, grid in axes:
        for v in grid:
            if v == best[name]:
                continue
            trial = {k: best[k] for k in keys}
            trial[name] = v
            ms = run(trial)
            if ms < best_ms:
                best_ms, best = ms, dict(best, **trial)
    for k in keys:
        ctx.set_param(k, best[k])
    return {"params": {k: best[k] for k in keys}, "ms": round(best_ms, 4),
            "mode": "persistent" if mode == MODE_PERSISTENT else ("plain" if mode == MODE_PLAIN else str(mode)),
            "table": table}


AREA_T_GRID = (8192, 65536, 262144)


def tune_prepare(ctx, specs, reps: int = 3, warm: int = 1, grid=AREA_T_GRID, raster: bool = False) -> dict:
    """area_T for sccg_prepare on the sets in specs ([(off, xy, tile, (mbr, area)), ...]): the box
    size under which a polygon is one streamed leaf rather than counted by rows (sets prepared
    without rasters; with rasters area_T does not apply). Leaves ctx at the best; returns
    {"area_T": best, "ms": best_ms, "table": [(area_T, ms), ...]}."""
    table = []
    for v in grid:
        ctx.set_param("area_T", v)
        table.append((v, round(_time(ctx, lambda: ctx.prepare_sets(specs, raster=raster), reps, warm), 4)))
    best = min(table, key=lambda t: t[1])
    ctx.set_param("area_T", best[0])
    return {"area_T": best[0], "ms": best[1], "table": table}


def signature(A, B, n_pairs: int) -> str:
    """A workload key: set sizes, vertex counts, largest polygon and extent, pair count."""
    return (f"nA={A.c.n},nB={B.c.n},vA={A.xy.numel() // 2},vB={B.xy.numel() // 2},"
            f"maxnv={max(A.c.max_nv, B.c.max_nv)},maxext={max(A.c.max_extent, B.c.max_extent)},np={n_pairs}")


def load(path: str, key: str) -> dict | None:
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def save(path: str, key: str, result: dict) -> None:
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    data[key] = {"params": result["params"], "ms": result["ms"], "mode": result["mode"]}
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
