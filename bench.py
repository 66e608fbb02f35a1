#!/usr/bin/env python3
"""Throughput of the exact cross-comparison path on GB300: polygon pairs/s with bit-exact int64
intersection/union pixel areas.

One step = the whole path over one synthetic workload resident in HBM:
  a1+a2  prepare both result sets (MBRs, validation, ||p|| per polygon)
  a3     candidate pairs (same tile, overlapping MBRs)
  a4+a5  pair areas ||p n q|| and ||p u q||: by default the persistent form (device work queue of
         64 x 64 sub-window items) replayed with the Jaccard as one CUDA graph (--form graph); also
         one kernel launch per tile as in the per-tile form of Sec. 4.1 (--form tiles), or the
         persistent form launched directly (--form persistent)
  a6     Jaccard J and J' (Sec. 2.1)

Default workload: a 100,000 x 100,000 px slide cut into 4096^2 tiles, ~1M nucleus polygons per set
(synthetic, seeded; stands in for the paper's pathology datasets, Sec. 5.1).

Prints ONE JSON line (rank 0). Launch N>1 with torch.distributed.run: each rank processes its own
slide (seed 1 + rank), no collective on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import contextlib
import gc
import math
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "polygon pairs/s (bit-exact inter/union areas) on 1 GB300; % ALU peak; p99 job ms"
UNIT = "pairs/s"

# Algorithmic int32/fp32 ALU operations per unit of work, counted from the exact tests as the
# kernels formulate them: one 32-pixel row strip against one edge (straddle test, crossing count,
# prefix-mask update), one sampling box against one edge (bounding-box and separating-axis tests,
# reference-centre crossing), one listed straddling edge, and one (edge, row) list entry.
OPS_PER_STRIP_EDGE = 17
OPS_PER_BOX_EDGE = 33
OPS_PER_ROW_WORD = 10      # one (row, 32-pixel word) of a leaf window: parity of both polygons, combine, count
OPS_PER_ROW_ENTRY = 16     # one (edge, row) crossing of a leaf window: exact crossing count, two XOR flips
OPS_PER_SCAN_ENTRY = 14    # one (edge, row) crossing value of the by-rows area: count, N, ceil-divide, store
OPS_PER_SCAN_PAIR = 4      # one comparison while ranking a row's crossing values


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--form", choices=["tiles", "persistent", "graph"], default=None,
                   help="a4 form timed as the headline (default: tiles for config 1, graph for 2-5)")
    p.add_argument("--config", type=int, default=3,
                   help="1 single tile, 2 whole slide, 3 batched uneven tiles (default: the largest single-GPU "
                   "workload), 4 heavy tail, 5 serving over 3")
    p.add_argument("--other-configs", type=str, default="auto",
                   help="comma-separated configs measured after the headline one in the same run and reported under "
                   "other_configs ('auto': 2,4 after config 3 or 5; 'none')")
    p.add_argument("--serve-jobs", type=int, default=0, help="jobs per offered load (default 20000 for configs "
                   "3 and 5, 2000 otherwise)")
    p.add_argument("--serve-loads", type=str, default="", help="comma-separated offered loads (fractions of the "
                   "measured peak); default 0.5,0.8,0.95 for configs 3 and 5 and 0.8 otherwise; 'none' to skip")
    p.add_argument("--tiles", type=int, default=0, help="restrict to the first N tiles (profiling runs)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-chunks", type=int, default=8, help="tile chunks of the end-to-end pipeline (8 equal "
                   "ones: 33.0 ms per step on the uneven tiles, against 38.1 with 3 growing by 1.5)")
    p.add_argument("--e2e-growth", type=float, default=1.0, help="size ratio of consecutive pipeline chunks")
    p.add_argument("--params", type=str, default="", help="JSON tunables for the context")
    p.add_argument("--autotune", choices=["auto", "on", "off"], default="auto",
                   help="time T / split_pixels / warps_per_cta on the workload before the run (untimed); "
                   "auto = on for configs 3-5")
    p.add_argument("--ablation", action="store_true",
                   help="Fig. 8 of the paper: PixelOnly / PixelBox-NoSep / PixelBox pair-area times on the "
                   "first 9 whole-slide tiles with coordinates scaled x1..x5 (prints one JSON line)")
    p.add_argument("--no-rasters", action="store_true",
                   help="prepare the sets without pixel rasters (pair areas pixelize every pair window)")
    p.add_argument("--profile-once", action="store_true",
                   help="run a single step of --form and exit (for ncu captures; prints no bench line)")
    p.add_argument("--traffic-csv", type=str, default="",
                   help="ncu --csv log of dram__bytes_read.sum/dram__bytes_write.sum of a --profile-once run on the "
                        "first --tiles tiles: write the per-step DRAM traffic of the whole workload to "
                        "profiles/traffic.json (scaled by vertices or pairs) and exit")
    return p.parse_args()


# ------------------------------------------------------------------------------------------------
# workload
# ------------------------------------------------------------------------------------------------

def make_workload(config: int, seed: int, tiles: int):
    from paper_1208_0277_gb300 import workload as W
    if config == 1:
        w = W.single_tile(seed=seed)
        desc = {"workload": "single 2048x2048 tile, 1,000 star polygons per set (8-64 vertices, MBR 10-40 px)"}
    elif config == 2:
        w = W.whole_slide(seed=seed)
        desc = {"workload": "whole slide 100,000x100,000 px, 4096x4096 tiles (625), ~1M star nuclei per set "
                            "(8-64 vertices, MBR 10-40 px, 100 per 10^6 px^2); B = A jittered +-3, shifted +-5, "
                            "10% dropped, 10% new"}
    elif config == 4:
        w = W.heavy_tail(seed=seed)
        desc = {"workload": "heavy tail: 200 tiles of 4096^2 px, 20,000 star nuclei per tile (8-64 vertices, MBR "
                            "10-40 px) + 5-20 concave tissue regions per tile (2,000-20,000 vertices, MBR "
                            "log-uniform 500-4,000 px); B = A jittered/shifted, nuclei 10% dropped, 10% new"}
    elif config in (3, 5):
        w = W.batched_uneven(seed=seed)
        desc = {"workload": "2,000 tiles of 4096^2 px, polygons per tile log-uniform 50-20,000 (~6.4M per set), "
                            "MBR lognormal(ln 20, 0.75) clipped to 8-400 px, 4-512 vertices; B = A jittered/"
                            "shifted, 10% dropped, 10% new"}
    else:
        raise SystemExit(f"--config {config} is not a bench workload here")
    if config == 5:
        desc["workload"] = ("serving: jobs of one tile each, a contiguous slice of log-uniform 100-50,000 candidate "
                            "pairs, Poisson arrivals, over resident sets of " + desc["workload"])
    if tiles:
        w = W.subset_tiles(w, range(min(tiles, w.n_tiles)))
        desc["workload"] += f" (first {tiles} tiles)"
    return w, desc


def kernel_source_hash() -> str:
    """Hash of the device code (the kernels whose DRAM traffic profiles/traffic.json records)."""
    h = hashlib.sha256()
    for f in ("leaf64.cuh", "pixelbox.cuh", "scanline.cuh", "kernels.cuh", "raster.cuh"):
        with open(os.path.join(ROOT, "paper_1208_0277_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


@contextlib.contextmanager
def quiet_collector():
    """No garbage-collector pass inside a timed region: the objects alive before it are collected
    once and frozen (the interpreter's import-time objects alone make a full pass take a large
    fraction of a step), and collection stays off until the region ends."""
    gc.collect()
    gc.freeze()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()
        gc.unfreeze()


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def wait_ready(self, timeout_s: float = 10.0):
        """Block until the first sample has arrived (NVML initialised outside the timed region)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout_s:
            time.sleep(0.05)

    def mark(self, which: str):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t_start", 0.0), getattr(self, "t_end", float("inf"))
        inside = [ln for t, ln in self.lines if t0 <= t <= t1 + 0.25]
        if not inside and self.lines:
            # timed region shorter than the sampling period: take the sample nearest to it
            inside = [min(self.lines, key=lambda x: abs(x[0] - t0))[1]]
        for ln in inside:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ------------------------------------------------------------------------------------------------

def whole_job(ms: float, pairs: int, dist, device):
    """Whole-job figures of a timed region under weak scaling (every rank compares its own slide):
    the slowest rank's duration and the pairs of all ranks. dist = torch.distributed or None."""
    if not dist:
        return ms, pairs
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([pairs], dtype=torch.int64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), int(p.item())


def oracle_sample(w, target_s: float):
    """Run the CPU oracle (brute force, all host cores) on the first tiles of the workload, growing
    the sample geometrically until one run costs at least target_s / 2 (or the whole workload is
    covered). Returns (result dict, tiles, seconds of the last run)."""
    import oracle as O
    from paper_1208_0277_gb300 import workload as W
    tiles = 1
    while True:
        sub = W.subset_tiles(w, range(tiles)) if tiles < w.n_tiles else w
        t0 = time.perf_counter()
        res = O.cross_compare(sub.A, sub.B)
        elapsed = time.perf_counter() - t0
        if elapsed >= target_s / 2 or tiles >= w.n_tiles:
            return res, tiles, elapsed
        grow = max(2.0, min(8.0, target_s / max(elapsed, 1e-3)))
        tiles = min(w.n_tiles, int(tiles * grow) + 1)


def oracle_sample_pairs(w, target_s: float, seed: int = 7):
    """For workloads whose single tile is already beyond a bounded oracle run (config 4: tissue
    windows up to 4000^2 px against 20,000-edge rings): the oracle's candidate pairs of tile 0, then
    its exact pair areas (row-interval method) on a seeded uniform sample of them, grown until one
    run costs at least target_s / 2. Returns (tile-0 pairs (pa, pb), sample indices, (inter, uni),
    seconds)."""
    import numpy as np
    import oracle as O
    from paper_1208_0277_gb300 import workload as W
    sub = W.subset_tiles(w, range(1))
    _, mbr_a = O.polygon_areas(sub.A.off, sub.A.xy, method="rle")
    _, mbr_b = O.polygon_areas(sub.B.off, sub.B.xy, method="rle")
    pa, pb = O.candidate_pairs(mbr_a, sub.A.tile, mbr_b, sub.B.tile)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(pa))
    m = 64
    while True:
        idx = np.sort(order[:m])
        t0 = time.perf_counter()
        res = O.pair_areas(sub.A, sub.B, pa[idx], pb[idx], method="rle")
        el = time.perf_counter() - t0
        if el >= target_s / 2 or m >= len(pa):
            return (pa, pb), idx, res, el
        m = min(len(pa), int(m * max(2.0, min(8.0, target_s / max(el, 1e-3)))) + 1)


def ablation(args):
    """PixelOnly (pixelize every window: T above any window), PixelBox-NoSep (union counted directly
    by subdivision) and PixelBox (union from the areas) on the same candidate pairs, coordinates
    scaled x1..x5 (Sec. 5.2, Fig. 8); T tuned per variant and scale over a sweep (Fig. 10), as the
    paper tunes it. Pair-area phase only, one launch, CUDA events; every result checked against the
    oracle's row-interval method."""
    import numpy as np
    import torch
    import oracle as O
    import paper_1208_0277_gb300 as P
    from paper_1208_0277_gb300 import workload as W
    P.build()
    O.build()
    base = W.subset_tiles(W.whole_slide(seed=1), range(9))
    ctx = P.Context(0)
    dev = torch.device("cuda", 0)
    ev = lambda: torch.cuda.Event(enable_timing=True)      # noqa: E731
    t_sweep = [256, 1024, 4096, 16384, 65536]

    def timed(fn, reps=7, warm=2):
        ts = []
        for r in range(warm + reps):
            a, b = ev(), ev()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if r >= warm:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    rows = []
    n_ref = None
    for s in range(1, 6):
        w = W.scaled(base, s)
        A, B = ctx.upload(w.A, raster=False), ctx.upload(w.B, raster=False)
        pa, pb = ctx.candidate_pairs(A, B)
        n = pa.numel()
        n_ref = n_ref or n
        _, ma = O.polygon_areas(w.A.off, w.A.xy, method="rle")
        _, mb = O.polygon_areas(w.B.off, w.B.xy, method="rle")
        opa, opb = O.candidate_pairs(ma, w.A.tile, mb, w.B.tile)
        ri, ru = O.pair_areas(w.A, w.B, opa, opb, method="rle")
        inter = torch.empty(n, dtype=torch.int64, device=dev)
        uni = torch.empty_like(inter)
        row = {"scale": s, "pairs": n, "mean_window_px": None,
               "parity": bool(np.array_equal(pa.cpu().numpy(), opa) and np.array_equal(pb.cpu().numpy(), opb))}
        mbr_a, mbr_b = A.mbr[pa.long()].cpu().numpy(), B.mbr[pb.long()].cpu().numpy()
        ww = np.maximum(0, np.minimum(mbr_a[:, 2], mbr_b[:, 2]) - np.maximum(mbr_a[:, 0], mbr_b[:, 0]))
        wh = np.maximum(0, np.minimum(mbr_a[:, 3], mbr_b[:, 3]) - np.maximum(mbr_a[:, 1], mbr_b[:, 1]))
        row["mean_window_px"] = float((ww * wh).mean())
        for name, mode, words, ts in (("PixelOnly", P.MODE_PLAIN, 0, [1 << 28]),
                                      ("PixelBox-NoSep", P.MODE_NOSEP, 0, t_sweep),
                                      ("PixelBox", P.MODE_PLAIN, 0, t_sweep),
                                      ("PixelOnly+words", P.MODE_PLAIN, 1, [1 << 28]),
                                      ("PixelBox+words", P.MODE_PLAIN, 1, t_sweep)):
            ctx.set_param("leaf_words", words)
            best = None
            for T in ts:
                ctx.set_param("T", T)
                inter.fill_(-7)
                ms = timed(lambda: ctx.pair_areas(A, B, pa, pb, mode=mode, out=(inter, uni)))
                ok = bool(np.array_equal(inter.cpu().numpy(), ri) and np.array_equal(uni.cpu().numpy(), ru))
                row["parity"] = row["parity"] and ok
                row.setdefault("T_sweep_ms", {}).setdefault(name, {})[str(T)] = round(ms, 4)
                if best is None or ms < best[0]:
                    best = (ms, T)
            row[name] = {"ms": round(best[0], 4), "T": best[1]}
        # each polygon pixelized once into a raster kept with the set; pairs AND two rasters
        Ar, Br = ctx.upload(w.A), ctx.upload(w.B)
        for name, mode in (("Rasters", P.MODE_PLAIN), ("Rasters persistent", P.MODE_PERSISTENT)):
            inter.fill_(-7)
            ms = timed(lambda: ctx.pair_areas(Ar, Br, pa, pb, mode=mode, out=(inter, uni)))
            ok = bool(np.array_equal(inter.cpu().numpy(), ri) and np.array_equal(uni.cpu().numpy(), ru))
            row["parity"] = row["parity"] and ok
            row[name] = {"ms": round(ms, 4)}
        specs = [(Ar.off, Ar.xy, Ar.tile, (Ar.mbr, Ar.area, Ar.raster)),
                 (Br.off, Br.xy, Br.tile, (Br.mbr, Br.area, Br.raster))]
        plain = [(Ar.off, Ar.xy, Ar.tile, (A.mbr, A.area)), (Br.off, Br.xy, Br.tile, (B.mbr, B.area))]
        row["prepare_ms"] = {"with_rasters": round(timed(lambda: ctx.prepare_sets(specs, bands=False)), 4),
                             "without": round(timed(lambda: ctx.prepare_sets(plain, bands=False, raster=False)), 4)}
        del Ar, Br
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    # Sec. 3.2's closed form for rectilinear sets (area_method SHOELACE) against the pixel count
    # (ROWS) in sccg_prepare, on 200,000 seeded staircases (the paper's raster-boundary shape)
    rng = np.random.Generator(np.random.PCG64(3))
    rings, heights = W.staircase_rings(rng, 2000, max_cols=30, max_h=25, origin_span=100_000)
    rings = rings * 100
    stairs = W.from_rings(rings)
    d_off = torch.from_numpy(stairs.off).to(dev)
    d_xy = torch.from_numpy(stairs.xy).to(dev)
    ref_area = np.array([int(h.sum()) for h in heights] * 100)
    shoe = {"polygons": stairs.n, "vertices": stairs.n_vertices}
    for name, method in (("rows", P.AREA_ROWS), ("shoelace", P.AREA_SHOELACE)):
        ctx.set_param("area_method", method)
        d = ctx.prepare(d_off, d_xy, raster=False)
        ms = timed(lambda: ctx.prepare(d_off, d_xy, out=(d.mbr, d.area), raster=False))
        shoe[name] = {"ms": round(ms, 4), "exact": bool(np.array_equal(d.area.cpu().numpy()[: stairs.n], ref_area))}
    ctx.set_param("area_method", P.AREA_ROWS)
    print(json.dumps({"shoelace_prepare": shoe}), file=sys.stderr, flush=True)
    line = {"ablation": "Sec. 5.2 Fig. 8: PixelOnly vs PixelBox-NoSep vs PixelBox, coordinates scaled x1..x5; "
                        "leaves as 32-pixel strips tested against every edge (the paper's per-pixel test), "
                        "'+words': leaves from per-row parity words, and 'Rasters': every polygon pixelized once "
                        "when its set is prepared (this build's default), pairs ANDing two rasters "
                        "(prepare_ms: both sets, with and without the rasters)",
            "workload": "first 9 tiles of the whole slide (seed 1), same candidate pairs at every scale",
            "pairs": n_ref, "unit": "ms per pair-area launch (median of 7, CUDA events)", "rows": rows,
            "shoelace_prepare": dict(shoe, note="sccg_prepare of 200,000 staircases (100 copies of 2,000 seeded "
                                                "ones): pixel count by rows against the shoelace closed form "
                                                "for sets flagged rectilinear and simple (Sec. 3.2); exact = "
                                                "areas equal the column sums")}
    print(json.dumps(line), flush=True)


def reference_arm(args):
    """The CPU oracle as the reference arm: each step is a bounded sample of the same workload."""
    import oracle as O
    from paper_1208_0277_gb300 import workload as W
    w, desc = make_workload(args.config, 1, args.tiles)
    O.build()
    # size one step so that warm-up plus timed steps take about two minutes
    target = max(1.0, 120.0 / (args.steps + args.warmup))
    if args.config == 4:
        (o_pa, o_pb), idx, _, _ = oracle_sample_pairs(w, target_s=target)
        sub = W.subset_tiles(w, range(1))
        step = lambda: O.pair_areas(sub.A, sub.B, o_pa[idx], o_pb[idx], method="rle")  # noqa: E731
        pairs_of = lambda r: len(idx)                                                   # noqa: E731
        sample = (f"uniform sample of {len(idx)} of the {len(o_pa)} candidate pairs of tile 0 per step: the "
                  "oracle's exact row-interval pair areas; extrapolated per pair")
    else:
        res, tiles, el = oracle_sample(w, target_s=target)
        sub = W.subset_tiles(w, range(tiles)) if tiles < w.n_tiles else w
        step = lambda: O.cross_compare(sub.A, sub.B)                                    # noqa: E731
        pairs_of = lambda r: len(r["pa"])                                               # noqa: E731
        sample = None
    for _ in range(args.warmup):
        step()
    times, pairs = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = step()
        times.append(time.perf_counter() - t0)
        pairs = pairs_of(r)
    tot = sum(times)
    value = pairs * args.steps / tot
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": desc,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample or (f"first {tiles} of {w.n_tiles} tiles per step ({pairs} candidate "
                                              "pairs; brute-force pixel areas, candidate pairs and Jaccard)")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# serving (continuous batching): peak, then Poisson loads at fractions of it
# ------------------------------------------------------------------------------------------------

def serving_results(A, B, pa, pb, tpo, loads, n_jobs, device, seed=5):
    """Peak (every job submitted at once) and Poisson loads at fractions of it, each replayed from an
    arrival trace; latency from each job's scheduled arrival to its result in host memory."""
    import numpy as np
    from paper_1208_0277_gb300 import serve
    rng = np.random.default_rng(seed)
    srv = serve.Server(A, B, pa, pb, device=device, slots=3, max_batch_pairs=1 << 20, max_batch_jobs=1024)
    import gc
    switch = sys.getswitchinterval()
    sys.setswitchinterval(0.0005)        # the client, batcher and completer threads share the interpreter
    gc.disable()                         # no collector pauses inside the replayed traces
    try:
        warm = serve.draw_jobs(rng, tpo, 64)
        [f.result() for f in srv.submit_many(warm)]
        peak = None
        for _ in range(2):               # the better of two bursts
            burst = serve.draw_jobs(rng, tpo, n_jobs)
            t0 = time.perf_counter()
            futs = srv.submit_many(burst)
            srv.drain()
            res = [f.result() for f in futs]
            p_ = serve.latency_summary(res, max(r.t_done for r in res) - t0)
            if peak is None or p_["pairs_per_s"] > peak["pairs_per_s"]:
                peak = p_
            del res, futs
            gc.collect()
        mean_pairs = peak["pairs"] / peak["jobs"]
        out = {"peak": dict(peak, note="all jobs submitted at once (the better of two bursts)"), "loads": [],
               "server": {"slots": len(srv.slots), "max_batch_pairs": srv.cap_pairs, "arena_pairs": srv.arena_pairs,
                          "device_bytes": srv.device_bytes(), "mem_budget_bytes": srv.mem_budget_bytes},
               "latency": "scheduled arrival (Poisson trace) -> areas and Jaccard of the job in host memory"}
        for load in loads:
            jobs = serve.draw_jobs(rng, tpo, n_jobs)
            rate = load * peak["pairs_per_s"] / mean_pairs
            res, wall = serve.run_load(srv, jobs, rate, rng)
            out["loads"].append(dict(serve.latency_summary(res, wall, rate), offered_load=load,
                                     offered_jobs_per_s=rate))
            del res
            gc.collect()
        out["waited_for_memory"] = srv.waited_for_memory
        out["python_gc"] = "disabled while each trace runs (collected between traces)"
        return out
    finally:
        gc.enable()
        sys.setswitchinterval(switch)
        srv.close()


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------

FORM_NAMES = {"tiles": "one kernel launch per tile",
              "persistent": "persistent single launch, device work queue",
              "graph": "persistent launch + Jaccard replayed as one CUDA graph"}


_ALU = {}
RASTER_BYTES_PER_PAIR = 88    # pa, pb; two MBRs; two raster offsets; two areas; inter and uni written
RASTER_BYTES_PER_WORD = 8     # one 32-bit word of each raster per (row, word) of a pair window


def hbm_peak() -> dict:
    """The measured HBM copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json, written by the
    measurement of the machine), else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return {"gbs": float(m["hbm_gbs"]), "note": f"measured: {m.get('how', 'copy bandwidth')}"}
    except (OSError, ValueError, KeyError):
        return {"gbs": 6800.0, "note": "fallback: 6.8 TB/s, one earlier copy measurement on a GB300"}


def alu_peak(device: int) -> dict:
    """The integer ALU issue rate measured on this GPU (sccg_alu_probe: independent int32 multiply-add,
    three-input XOR and three-input add chains, 64 warps per SM), best of three runs of about 100 ms,
    with the SM clock sampled while they run. Measured once per process."""
    if device in _ALU:
        return _ALU[device]
    import torch
    import paper_1208_0277_gb300 as P
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    ms, _ = P.alu_probe(device, 2048)
    iters = max(64, int(2048 * 100.0 / max(ms, 1e-3)))
    sampler = ClockSampler(device)
    sampler.start()
    sampler.wait_ready()
    sampler.mark("t_start")
    best = 0.0
    for _ in range(3):
        ms, ops = P.alu_probe(device, iters)
        best = max(best, ops / (ms / 1e3))
    sampler.mark("t_end")
    clocks = sampler.stop()
    time.sleep(1.0)
    mhz = clocks["sm_mhz"] if clocks else None
    per_clk = best / (sms * mhz * 1e6) if mhz else None
    _ALU[device] = {"lane_ops_per_s": best, "sm_mhz": mhz, "lane_ops_per_sm_clock": per_clk,
                    "note": (f"measured: sccg_alu_probe (int32 multiply-add / three-input XOR / three-input add "
                             f"chains, {sms} SMs x 64 warps), best of 3 runs of about 100 ms"
                             + (f"; {per_clk:.1f} lane-ops per SM per clock at the sampled {mhz:.0f} MHz"
                                if per_clk else ""))}
    return _ALU[device]


def oracle_dense_tiles(w, pa, pb, tpo, inter, uni, A, B, n_extra: int = 3, seed: int = 7):
    """Parity at full density: the tile with the most polygons and n_extra seeded other tiles, each
    compared element by element with the oracle (its O(n m) candidate pairs and its exact
    row-interval areas of every polygon and every pair of the tile). Returns (summary, seconds)."""
    import numpy as np
    import oracle as O
    from paper_1208_0277_gb300 import workload as W
    O.build()
    counts = np.bincount(w.A.tile, minlength=w.n_tiles)
    dense = int(np.argmax(counts))
    rng = np.random.default_rng(seed)
    rest = np.delete(np.arange(w.n_tiles), dense)
    tiles = sorted([dense] + [int(t) for t in rng.choice(rest, min(n_extra, len(rest)), replace=False)])
    a_start = np.searchsorted(w.A.tile, np.arange(w.n_tiles + 1))
    b_start = np.searchsorted(w.B.tile, np.arange(w.n_tiles + 1))
    ok, pairs, polys = True, 0, 0
    t0 = time.perf_counter()
    for t in tiles:
        sub = W.subset_tiles(w, [t])
        ref = O.cross_compare(sub.A, sub.B, method="rle")
        k0, k1 = int(tpo[t]), int(tpo[t + 1])
        a0, a1, b0, b1 = int(a_start[t]), int(a_start[t + 1]), int(b_start[t]), int(b_start[t + 1])
        g = dict(pa=pa[k0:k1].cpu().numpy().astype(np.int64) - a0, pb=pb[k0:k1].cpu().numpy().astype(np.int64) - b0,
                 inter=inter[k0:k1].cpu().numpy(), uni=uni[k0:k1].cpu().numpy(),
                 area_a=A.area[a0:a1].cpu().numpy(), area_b=B.area[b0:b1].cpu().numpy(),
                 mbr_a=A.mbr[a0:a1].cpu().numpy(), mbr_b=B.mbr[b0:b1].cpu().numpy())
        ok = ok and all(np.array_equal(g[k], ref[k]) for k in g)
        pairs += k1 - k0
        polys += (a1 - a0) + (b1 - b0)
    el = time.perf_counter() - t0
    return {"tiles": tiles, "densest_tile": dense, "densest_tile_polygons": int(counts[dense]),
            "pairs": pairs, "polygons": polys, "bit_exact": bool(ok),
            "how": "oracle O(n m) candidate pairs and exact row-interval areas of every polygon and every pair of "
                   "the densest tile and of seeded other tiles, compared element by element (MBRs, ||p||, pairs, "
                   "inter, union)"}, el


def measure(args, config: int, rank: int, world: int, local_rank: int, dist, full: bool) -> dict:
    """Time one workload: W warm-up and K timed steps of each form (the headline form first, with the
    clock sampled), one counting step for the roofline, and the oracle parity sample. full: also the
    end-to-end pipeline from host memory, the CPU baseline and the serving loads."""
    import numpy as np
    import torch

    import paper_1208_0277_gb300 as P

    form_main = args.form or ("graph" if config in (2, 3, 4, 5) else "tiles")
    params = json.loads(args.params) if args.params else None
    ctx = P.Context(local_rank, params)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    w, desc = make_workload(config, 1 + rank, args.tiles)
    gen_s = time.perf_counter() - t0

    # inputs resident in HBM (also kept in pinned host memory for the end-to-end measurement)
    host, devb = {}, {}
    for name, ps in (("A", w.A), ("B", w.B)):
        for f in ("off", "xy", "tile"):
            a = torch.from_numpy(getattr(ps, f))
            if full:
                a = a.pin_memory()
                host[name + f] = a
            devb[name + f] = a.to(dev)
    nA, nB = w.A.n, w.B.n
    outs = {
        "Ambr": torch.empty((nA, 4), dtype=torch.int32, device=dev), "Aarea": torch.empty(nA, dtype=torch.int64, device=dev),
        "Bmbr": torch.empty((nB, 4), dtype=torch.int32, device=dev), "Barea": torch.empty(nB, dtype=torch.int64, device=dev),
    }
    rasters = not args.no_rasters
    A = ctx.prepare(devb["Aoff"], devb["Axy"], devb["Atile"], out=(outs["Ambr"], outs["Aarea"]), raster=rasters)
    B = ctx.prepare(devb["Boff"], devb["Bxy"], devb["Btile"], out=(outs["Bmbr"], outs["Barea"]), raster=rasters)
    # the sets' pixel rasters stay in device memory, their buffers reused by every later prepare
    outs["Araster"], outs["Braster"] = A.raster, B.raster

    def spec(name):
        return (devb[name + "off"], devb[name + "xy"], devb[name + "tile"],
                (outs[name + "mbr"], outs[name + "area"], outs[name + "raster"]))

    pa0, pb0, tpo0 = ctx.candidate_pairs(A, B, with_tile_offsets=True)
    n_pairs = int(pa0.numel())
    tuned = None
    if args.autotune == "on" or (args.autotune == "auto" and config in (3, 4, 5)):
        from paper_1208_0277_gb300 import tune
        tuned = tune.tune(ctx, A, B, pa0, pb0, mode=P.MODE_PLAIN if form_main == "tiles" else P.MODE_PERSISTENT)
        if rasters:
            tuned_prep = {"area_T": None, "ms": None, "table": [], "note": "sets with rasters: area_T does not apply"}
        else:
            tuned_prep = tune.tune_prepare(ctx, [spec("A"), spec("B")], raster=False)
            tuned["params"]["area_T"] = tuned_prep["area_T"]
        tuned["prepare"] = tuned_prep
        print(f"config {config} autotune: {tuned['params']} ({len(tuned['table'])} trials, {tuned['ms']} ms; "
              f"prepare {tuned_prep['table']})", file=sys.stderr)
    cap = n_pairs
    pa = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    pb = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    inter = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    uni = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    del pa0, pb0
    jres = torch.zeros(48, dtype=torch.uint8, device=dev)    # device Jaccard result of the graph form

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    tpo_box = [tpo0]

    def step(form: str, phases=None):
        e = [ev() for _ in range(5)] if phases is not None else None
        if e: e[0].record(stream)
        a, b = ctx.prepare_sets([spec("A"), spec("B")], raster=rasters)
        if e: e[1].record(stream)
        p_a, p_b, tpo = ctx.candidate_pairs(a, b, capacity=cap, with_tile_offsets=True, out=(pa, pb))
        tpo_box[0] = tpo
        if e: e[2].record(stream)
        if form == "tiles":
            i, u = ctx.pair_areas_tiles(a, b, p_a, p_b, tpo, out=(inter, uni))
        elif form == "persistent":
            i, u = ctx.pair_areas(a, b, p_a, p_b, mode=P.MODE_PERSISTENT, out=(inter, uni))
        else:
            i, u = ctx.batch_run(a, b, p_a, p_b, (inter, uni), jres)
        if e: e[3].record(stream)
        J = ctx.jaccard(i, u) if form != "graph" else ctx.read_jaccard(jres)
        if e:
            e[4].record(stream)
            phases.append(e)
        return J

    if args.profile_once:
        J = step(form_main)
        torch.cuda.synchronize()
        print(json.dumps({"profile_once": form_main, "config": config, "pairs": n_pairs, "J": J["J"]}), flush=True)
        ctx.close()
        return {}

    # one counting step (untimed): algorithmic work per phase for the roofline
    ctx.set_param("count_work", 1)
    ctx.work_counters(reset=True)
    a_, b_ = ctx.prepare_sets([spec("A"), spec("B")], raster=rasters)
    work_prep = ctx.work_counters(reset=True)
    p_a, p_b, tpo = ctx.candidate_pairs(a_, b_, capacity=cap, with_tile_offsets=True, out=(pa, pb))
    if form_main == "tiles":
        ctx.pair_areas_tiles(a_, b_, p_a, p_b, tpo, out=(inter, uni))
    else:
        ctx.pair_areas(a_, b_, p_a, p_b, mode=P.MODE_PERSISTENT, out=(inter, uni))
    torch.cuda.synchronize()
    work_areas = ctx.work_counters(reset=True)
    ctx.set_param("count_work", 0)

    def ops(wc):
        return (wc["strip_edges"] * OPS_PER_STRIP_EDGE + wc["box_edges"] * OPS_PER_BOX_EDGE +
                wc["row_edges"] * OPS_PER_ROW_WORD + wc["row_entries"] * OPS_PER_ROW_ENTRY +
                wc["scan_entries"] * OPS_PER_SCAN_ENTRY + wc["scan_pairs"] * OPS_PER_SCAN_PAIR)

    results = {}
    # the per-tile form gives each pair's whole window to one warp; the heavy tail's tissue windows
    # (up to 4000^2 px against thousands of edges) are what the persistent forms' items are for
    skipped = {"tiles": "not timed on the heavy tail: one warp per whole tissue window (about 12 s per "
                        "step); the persistent forms cut those windows into 64 x 64 items"} \
        if config == 4 and form_main != "tiles" else {}
    for form in [form_main] + [f for f in ("tiles", "persistent", "graph") if f != form_main and f not in skipped]:
        sampler = ClockSampler(local_rank) if form == form_main else None
        if sampler:
            sampler.start()
            sampler.wait_ready()
        for _ in range(max(args.warmup, 3)):
            step(form)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        phases = []
        launches0 = ctx.launch_count()
        torch.cuda.synchronize()
        if sampler:
            sampler.mark("t_start")
        start, end = ev(), ev()
        with quiet_collector():
            start.record(stream)
            J = None
            for _ in range(args.steps):
                J = step(form, phases)
            end.record(stream)
            torch.cuda.synchronize()
        if sampler:
            sampler.mark("t_end")
        clocks = sampler.stop() if sampler else None
        if sampler:
            # nvidia-smi's exit (NVML teardown) can hold up the next form's driver calls: let it settle
            time.sleep(1.0)
        launches = ctx.launch_count() - launches0
        ms, _ = whole_job(start.elapsed_time(end), n_pairs, dist, dev)
        ph = np.array([[p[k].elapsed_time(p[k + 1]) for k in range(4)] for p in phases])
        results[form] = dict(ms=ms, J=J, launches=launches, clocks=clocks,
                             phases_ms=dict(zip(["prepare", "candidate_pairs", "pair_areas", "jaccard"],
                                                ph.mean(axis=0).round(4).tolist())))

    main_r = results[form_main]
    _, total_pairs = whole_job(0.0, n_pairs, dist, dev)       # every rank compares its own slide
    value = total_pairs * args.steps / (main_r["ms"] / 1e3)

    # roofline of both hot kernels (average over the timed steps, CUDA events on their stream)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu = alu_peak(local_rank)
    peak_tops = alu["lane_ops_per_s"] / 1e12
    ph = main_r["phases_ms"]
    prm = ctx.params()
    side = math.isqrt(max(prm["split_pixels"], 1))
    streamed = prm["leaf_words"] and side * side < prm["T"]      # every item one leaf: streamed kernel
    use_rasters = bool(rasters and prm["rasters"] and A.raster is not None and B.raster is not None)
    k_areas = ("k_pair_raster" if use_rasters else
               "k_pair_areas_plain" if form_main == "tiles" else
               ("k_pair_areas_leaf" if side <= 64 else "k_pair_areas_stream") if streamed else
               "k_pair_areas_persistent")
    traffic_tab = {}
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            traffic_tab = json.load(open(prof))
        except (ValueError, OSError):
            traffic_tab = {}

    def roof(kernel, phase_ms, wc):
        achieved = ops(wc) / (phase_ms / 1e3) / 1e12
        ent = traffic_tab.get(kernel, {})
        traffic = (ent.get("bytes_per_step") if ent.get("source_hash") == kernel_source_hash() and
                   ent.get("workload") == desc["workload"] else None)
        return {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s (int32/fp32 ALU lane-ops)",
                "frac": achieved / peak_tops, "traffic": traffic, "kernel": kernel, "phase_ms": phase_ms,
                "peak_note": alu["note"],
                "achieved_note": "algorithmic ops (strip-edge x 17 + box-edge x 33 + leaf (edge, row) crossing x "
                                 "16 + leaf (row, word) x 10 + area crossing value x 14 + area comparison x 4, "
                                 "counted on device) per step / phase time (CUDA events)",
                "work": wc}

    def roof_mem(kernel, phase_ms, wc):
        # pair areas from rasters: bytes the method must move per pair (pair indices, two MBRs, two raster
        # offsets, two areas, the two results) and per (row, word) unit (one word of each raster)
        algo = RASTER_BYTES_PER_PAIR * n_pairs + RASTER_BYTES_PER_WORD * wc["raster_and"]
        achieved = algo / (phase_ms / 1e3) / 1e9
        peak = hbm_peak()
        ent = traffic_tab.get(kernel, {})
        traffic = (ent.get("bytes_per_step") if ent.get("source_hash") == kernel_source_hash() and
                   ent.get("workload") == desc["workload"] else None)
        return {"bound": "hbm", "achieved": achieved, "peak": peak["gbs"], "unit": "GB/s", "frac": achieved / peak["gbs"],
                "traffic": traffic, "kernel": kernel, "phase_ms": phase_ms, "peak_note": peak["note"],
                "achieved_note": f"algorithmic bytes ({RASTER_BYTES_PER_PAIR} per pair + {RASTER_BYTES_PER_WORD} per "
                                 "(row, 32-pixel word) of the pair windows, counted on device) per step / phase "
                                 "time (CUDA events)",
                "algorithmic_bytes": algo, "work": wc}

    r_areas = roof_mem(k_areas, ph["pair_areas"], work_areas) if use_rasters else \
        roof(k_areas, ph["pair_areas"], work_areas)
    r_prep = roof("k_prepare", ph["prepare"], work_prep)
    roofline, roofline_other = (r_areas, r_prep) if ph["pair_areas"] >= ph["prepare"] else (r_prep, r_areas)

    out = {
        "config_id": config, "value": value, "ms_per_step": main_r["ms"] / args.steps,
        "form": FORM_NAMES[form_main], "desc": desc, "pairs_per_step": n_pairs, "polygons": [nA, nB],
        "tiles": w.n_tiles, "input_bytes": sum(devb[k].numel() * devb[k].element_size() for k in devb),
        "generation_s": round(gen_s, 1), "params": prm,
        "autotune": ({"params": tuned["params"], "trials": len(tuned["table"]), "mode": tuned["mode"],
                      "best_ms": tuned["ms"], "prepare_ms_by_area_T": tuned["prepare"]["table"]} if tuned else None),
        "roofline": roofline, "roofline_other": roofline_other,
        # the pair path alone (a3-a6: sets prepared once and resident)
        "a3_a6": {"value": total_pairs * args.steps / ((main_r["ms"] - args.steps * ph["prepare"]) / 1e3),
                  "ms_per_step": main_r["ms"] / args.steps - ph["prepare"],
                  "note": "whole step minus the prepare phase (CUDA events): candidate pairs, pair areas and "
                          "unions, Jaccard on resident prepared sets"},
        "rates": ({"pixel_tests_per_s": work_prep["window_pixels"] / (ph["prepare"] / 1e3),
                   "window_pixels_per_s": work_areas["window_pixels"] / (ph["pair_areas"] / 1e3),
                   "note": "with rasters every (pixel, polygon) membership is decided once, in the prepare phase: "
                           "pixel tests = pixels of the polygons' windows pixelized there, per second of that "
                           "phase; window pixels = pixels of the pair windows resolved by ANDing rasters, per "
                           "second of the pair-area phase"} if use_rasters else
                  {"pixel_tests_per_s": work_areas["leaf_pixels"] / (ph["pair_areas"] / 1e3),
                   "window_pixels_per_s": work_areas["window_pixels"] / (ph["pair_areas"] / 1e3),
                   "note": "pixel tests = (pixel, polygon) memberships decided one pixel at a time in leaves; "
                           "window pixels = pixels of the pair windows (or work items) resolved"}),
        "clocks": main_r["clocks"], "gpu_launches": main_r["launches"], "phases_ms": ph,
        "jaccard": {"J": main_r["J"]["J"], "Jprime": main_r["J"]["Jprime"], "n_nonzero": main_r["J"]["n_nonzero"]},
        "other_forms": {f: {"form": FORM_NAMES[f], "value": total_pairs * args.steps / (o["ms"] / 1e3),
                            "ms_per_step": o["ms"] / args.steps, "phases_ms": o["phases_ms"],
                            "gpu_launches": o["launches"]}
                        for f, o in results.items() if f != form_main} |
                       {f: {"form": FORM_NAMES[f], "skipped": why} for f, why in skipped.items()},
    }

    # end-to-end through the public API with host buffers: the copy-overlapped pipeline over pinned
    # host sets (H2D of every input byte and D2H of every pair's indices and areas plus J each step)
    if full and not args.no_e2e:
        from paper_1208_0277_gb300.pipeline import HostSet, Pipeline
        hA = HostSet(host["Aoff"], host["Axy"], host["Atile"])
        hB = HostSet(host["Boff"], host["Bxy"], host["Btile"])
        n_e2e = max(3, args.steps // 4)

        def e2e_runs(copy):
            pipe = Pipeline(ctx, hA, hB, w.n_tiles, chunks=args.e2e_chunks, initial_pairs=n_pairs + 1024,
                            growth=args.e2e_growth, copy=copy)
            e_pa, _, e_inter, _, e_J = pipe.run()           # warm-up, and the same results as the device run
            same = bool(len(e_pa) == n_pairs and e_J["J"] == main_r["J"]["J"] and
                        e_J["Jprime"] == main_r["J"]["Jprime"])
            pipe.run()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            run_ms = []
            with quiet_collector():
                t0 = time.perf_counter()
                for _ in range(n_e2e):
                    t1 = time.perf_counter()
                    pipe.run()                   # returns after its results are in host memory
                    run_ms.append(round(1e3 * (time.perf_counter() - t1), 2))
                torch.cuda.synchronize()
                t_e2e = time.perf_counter() - t0
            return pipe, same, run_ms, t_e2e

        # the copy engines' form first (for comparison), then the SM copies the number is quoted on
        pipe, same_engine, run_ms_engine, t_engine = e2e_runs("engine")
        del pipe
        pipe, e2e_same, run_ms, t_e2e = e2e_runs("sm")
        e_ms, _ = whole_job(1e3 * t_e2e, n_pairs, dist, dev)
        e_ms_engine, _ = whole_job(1e3 * t_engine, n_pairs, dist, dev)
        # the host link's own rate on this machine, for reading the end-to-end number (a 1 GiB pinned copy)
        xh = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
        xd = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
        xd.copy_(xh, non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            xd.copy_(xh, non_blocking=True)
        torch.cuda.synchronize()
        h2d_gbs = 3 * (1 << 30) / (time.perf_counter() - t0) / 1e9
        del xh, xd
        out["e2e"] = {"value": total_pairs * n_e2e / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": pipe.h2d_bytes,
                      "h2d_gbs_pinned_copy": round(h2d_gbs, 1), "run_ms": run_ms,
                      "median_run_ms": statistics.median(run_ms),
                      "d2h_bytes_per_step": pipe.d2h_bytes, "ms_per_step": e_ms / n_e2e,
                      "chunks": len(pipe.chunks), "chunk_growth": args.e2e_growth,
                      "same_results_as_device_run": e2e_same and same_engine,
                      "copies": "by the SMs (sccg_copy, 16 CTAs on high-priority streams)",
                      "copy_engines": {"value": total_pairs * n_e2e / (e_ms_engine / 1e3),
                                       "ms_per_step": e_ms_engine / n_e2e, "run_ms": run_ms_engine,
                                       "median_run_ms": statistics.median(run_ms_engine)},
                      "how": "paper_1208_0277_gb300.pipeline: tiles in chunks, H2D of chunk k+1 overlapped with chunk "
                             "k (prepare, candidate pairs, persistent pair areas), results D2H as they finish, one "
                             "Jaccard; host wall clock"}
        del pipe

    # oracle parity on the device results of the last timed step (rank 0, N = 1), and the CPU baseline
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        torch.cuda.synchronize()
        if config == 4:
            (o_pa, o_pb), idx, (o_i, o_u), el = oracle_sample_pairs(w, target_s=15.0)
            k0 = len(o_pa)
            cpu = {"value": len(idx) / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"uniform sample of {len(idx)} of the {k0} candidate pairs of tile 0 ({el:.1f} s): the "
                             "oracle's exact row-interval pair areas (its brute force would take hours on the "
                             "4000^2-px tissue windows); extrapolated per pair"}
            parity = {"sample_pairs": int(len(idx)), "tile0_pairs": k0,
                      "bit_exact": bool(np.array_equal(pa[:k0].cpu().numpy(), o_pa) and
                                        np.array_equal(pb[:k0].cpu().numpy(), o_pb) and
                                        np.array_equal(inter[:k0].cpu().numpy()[idx], o_i) and
                                        np.array_equal(uni[:k0].cpu().numpy()[idx], o_u))}
        else:
            res, tiles, el = oracle_sample(w, target_s=15.0)
            k = len(res["pa"])
            cpu = {"value": k / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"first {tiles} of {w.n_tiles} tiles ({k} candidate pairs, {el:.1f} s): brute-force "
                             "pixel areas of both sets, candidate pairs, pair areas, Jaccard"}
            parity = {"sample_pairs": k, "sample_tiles": tiles,
                      "bit_exact": bool(np.array_equal(pa[:k].cpu().numpy(), res["pa"]) and
                                        np.array_equal(pb[:k].cpu().numpy(), res["pb"]) and
                                        np.array_equal(inter[:k].cpu().numpy(), res["inter"]) and
                                        np.array_equal(uni[:k].cpu().numpy(), res["uni"]))}
            if config in (3, 5):
                dense, dense_s = oracle_dense_tiles(w, pa, pb, tpo_box[0], inter, uni, A, B)
                parity["dense_tiles"] = dict(dense, seconds=round(dense_s, 1))
                parity["bit_exact"] = parity["bit_exact"] and dense["bit_exact"]
        out["parity_vs_oracle"] = parity
        if full:
            out["cpu_baseline"] = cpu
        else:
            out["oracle_pairs_per_s"] = cpu["value"]

    # stream admission of tile tasks (Sec. 4.2's buffer triggers, GPU streams only): static round robin
    # against admission by buffer state with the smallest tasks moved to idle streams
    if full and config in (3, 5) and rank == 0:
        from paper_1208_0277_gb300 import schedule
        tasks = schedule.tile_tasks(tpo_box[0])
        sched = {"tasks": len(tasks), "streams": 4, "depth": 4, "window": 2,
                 "task": "one tile's pair areas, one kernel launch (one warp per pair)",
                 "how": "host wall clock from the first admission to the last completion, median of 3 after 1 "
                        "warm-up; results checked against the resident run"}
        for policy in ("static", "dynamic"):
            ts, mig, waits, same = [], 0, 0, True
            for rep in range(4):
                i2 = torch.full_like(inter, -7)
                u2 = torch.full_like(uni, -7)
                ex = schedule.GpuExecutor(ctx, A, B, pa[:n_pairs], pb[:n_pairs], i2, u2, n_streams=4,
                                          device=local_rank)
                sch = schedule.Scheduler(ex, n_streams=4, depth=4, window=2, policy=policy)
                torch.cuda.synchronize()
                el, _ = sch.run(tasks)
                torch.cuda.synchronize()
                if rep:
                    ts.append(el)
                    mig, waits = sch.migrations, sch.producer_waits
                same = same and bool(torch.equal(i2[:n_pairs], inter[:n_pairs]) and
                                     torch.equal(u2[:n_pairs], uni[:n_pairs]))
            el = statistics.median(ts)
            sched[policy] = {"ms": 1e3 * el, "pairs_per_s": n_pairs / el, "migrations": mig,
                             "producer_waits": waits, "same_results": same}
        out["stream_admission"] = sched

    if full:
        loads_arg = args.serve_loads or ("0.5,0.8,0.95" if config in (3, 5) else "0.8")
        if loads_arg != "none":
            loads = [float(x) for x in loads_arg.split(",") if x]
            # long enough traces that the last job's latency is a small part of the measured span
            n_jobs = args.serve_jobs or (20000 if config in (3, 5) else 2000)
            serving = serving_results(A, B, pa[:n_pairs], pb[:n_pairs], tpo0, loads, n_jobs, local_rank)
            serving["jobs_per_load"] = n_jobs
            serving["job_pairs"] = "log-uniform 100-50,000, clipped to the tile's candidate pairs"
            if config in (3, 5):
                serving["workload"] = ("serving (the config-5 workload): jobs of one tile each over the resident sets "
                                       "above, Poisson arrivals at fractions of the measured peak")
            out["serving"] = serving
    ctx.close()
    del A, B, devb, host, outs, pa, pb, inter, uni
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


TRAFFIC_KERNELS = {   # kernel -> what its traffic grows with (per step: both sets' prepare, one pair pass)
    "k_prepare": "vertices", "k_raster_big": "vertices", "k_pair_raster": "pairs",
}


def traffic_table(args):
    """Per-step DRAM traffic of the dominant kernels on the whole workload, from one ncu capture of a
    --profile-once step on its first --tiles tiles: each kernel's dram__bytes_read.sum +
    dram__bytes_write.sum summed over the step's launches, scaled to the whole workload by the vertices
    of both sets (the prepare kernels) or by the candidate pairs (the pair kernel)."""
    import csv

    import torch

    import paper_1208_0277_gb300 as P

    if not args.tiles:
        raise SystemExit("--traffic-csv needs the --tiles of the captured run")
    rows = list(csv.reader(open(args.traffic_csv)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    ki, mi, vi = (rows[hi].index(k) for k in ("Kernel Name", "Metric Name", "Metric Value"))
    sub_bytes = {}
    for r in rows[hi + 1:]:
        if len(r) <= vi or not r[mi].startswith("dram__bytes_"):
            continue
        name = r[ki].split("(")[0].replace("void ", "").split("<")[0].replace("sccg::", "").strip()
        if name in TRAFFIC_KERNELS:
            sub_bytes[name] = sub_bytes.get(name, 0) + int(float(r[vi].replace(",", "")))

    torch.cuda.set_device(0)
    P.build()
    ctx = P.Context(0, json.loads(args.params) if args.params else None)
    dev = torch.device("cuda", 0)

    def units(tiles):
        w, desc = make_workload(args.config, 1, tiles)
        sets = []
        for ps in (w.A, w.B):
            sets.append(ctx.prepare(*(torch.from_numpy(getattr(ps, f)).to(dev) for f in ("off", "xy", "tile")),
                                    raster=False))
        pa, _ = ctx.candidate_pairs(sets[0], sets[1])
        n = {"vertices": int(w.A.off[-1] + w.B.off[-1]), "pairs": int(pa.numel())}
        del sets, pa
        torch.cuda.empty_cache()
        return n, desc

    sub, _ = units(args.tiles)
    whole, desc = units(0)
    cmd = (f"python bench.py --config {args.config} --tiles {args.tiles} --autotune off --params '{args.params}' "
           "--traffic-csv traffic.csv")
    out = {}
    for k, b in sorted(sub_bytes.items()):
        by = TRAFFIC_KERNELS[k]
        scale = whole[by] / sub[by]
        out[k] = {"source_hash": kernel_source_hash(), "workload": desc["workload"],
                  "bytes_per_step": int(b * scale),
                  "note": f"dram__bytes_read.sum + dram__bytes_write.sum of the step's {k} launches on the first "
                          f"{args.tiles} tiles ({b} bytes, {sub[by]} {by}), scaled by the {by} of the whole "
                          f"workload ({whole[by]}: x{scale:.4f})"}
    out["command"] = (f"python bench.py --config {args.config} --tiles {args.tiles} --profile-once --form graph "
                      f"--autotune off --params '{args.params}'; ncu --metrics dram__bytes_read.sum,"
                      "dram__bytes_write.sum,gpu__time_duration.sum --clock-control none -k regex:'k_prepare|"
                      "k_raster_big|k_pair_raster' -s 4 -c 5 --csv --log-file traffic.csv (the same command); "
                      + cmd + " (writes this file)")
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out), flush=True)
    ctx.close()


def other_configs_of(args) -> list:
    if args.other_configs == "auto":
        return [2, 4] if args.config in (3, 5) and not args.tiles else []
    if args.other_configs in ("", "none"):
        return []
    return [int(x) for x in args.other_configs.split(",") if x]


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.ablation:
        ablation(args)
        return
    if args.traffic_csv:
        traffic_table(args)
        return
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return

    import torch

    import paper_1208_0277_gb300 as P

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    P.build()

    head = measure(args, args.config, rank, world, local_rank, dist, full=True)
    if args.profile_once:
        return
    others = {}
    for c in other_configs_of(args):
        sub = measure(args, c, rank, world, local_rank, dist, full=False)
        others[str(c)] = {k: sub[k] for k in ("desc", "value", "ms_per_step", "form", "pairs_per_step", "polygons",
                                              "tiles", "phases_ms", "other_forms", "roofline", "roofline_other",
                                              "a3_a6", "autotune", "params", "clocks", "generation_s",
                                              "parity_vs_oracle", "oracle_pairs_per_s", "gpu_launches")
                          if k in sub}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": head["desc"],
        "run": {k: head[k] for k in ("form", "pairs_per_step", "polygons", "tiles", "input_bytes", "generation_s",
                                     "params", "autotune")} |
               {"config_id": args.config, "seed": 1 + rank, "l2": "inputs larger than L2 (no flush needed)"},
        "roofline": head["roofline"],
        "roofline_other": head["roofline_other"],
        "a3_a6": head["a3_a6"],
        "rates": head["rates"],
        "cpu_baseline": head.get("cpu_baseline"),
        "e2e": head.get("e2e"),
        "clocks": head["clocks"],
        "gpu_launches": head["gpu_launches"],
        "phases_ms": head["phases_ms"],
        "jaccard": head["jaccard"],
        "parity_vs_oracle": head.get("parity_vs_oracle"),
        "serving": head.get("serving"),
        "p99_job_ms": (head["serving"]["loads"][-1]["p99_ms"] if head.get("serving") and head["serving"]["loads"]
                       else None),
        "other_forms": head["other_forms"],
        "stream_admission": head.get("stream_admission"),
        "other_configs": others,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
