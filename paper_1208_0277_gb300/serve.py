"""Continuous-batching server for cross-comparison jobs over resident polygon sets.

A job asks for the exact intersection/union areas of a contiguous slice of the candidate pairs of
one tile, plus the Jaccard similarities over that slice (Sec. 4.1: the work unit is an image tile;
the aggregator groups tasks into GPU batches). The two polygon sets and their candidate pairs stay
resident in device memory; jobs only name pair ranges.

Execution: ``slots`` batch slots, each with its own library context (scratch), CUDA stream and
preallocated device and pinned-host buffers sized by ``max_batch_pairs`` / ``max_batch_jobs``. A
batcher thread forms a batch whenever a slot is free: it admits pending jobs in arrival order while
they fit the slot, so jobs that arrive while other batches run on the GPU join the next batch, and
batches on different slots overlap on the device. Per batch, on the slot's stream:
  1. copy the jobs' (source offset, destination offset) pairs host -> device,
  2. gather the jobs' pair slices into the slot's pair buffer (``sccg_gather_pairs``),
  3. exact pair areas, persistent form (``sccg_pair_areas``),
  4. per-job Jaccard (``sccg_jaccard_segments``),
  5. copy areas and Jaccard structs device -> pinned host, record an event.
A completer thread waits for each batch's event in order and resolves the jobs' futures.

Admission: memory is bounded by construction (``slots`` x the slot buffers, checked against
``mem_budget_bytes`` when the server is built); a job larger than a slot is refused with
``ValueError`` at submit time; otherwise jobs wait in the queue until a slot frees up. A job whose
future the client cancels before it is admitted to a batch is dropped.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time

import numpy as np

from . import Context, MODE_PERSISTENT


@dataclasses.dataclass
class Job:
    p0: int                 # first candidate-pair index (into the resident pair list)
    p1: int                 # one past the last
    tile: int = -1
    t_submit: float = 0.0


@dataclasses.dataclass
class JobResult:
    inter: np.ndarray       # int64 [p1 - p0]
    uni: np.ndarray         # int64 [p1 - p0]
    jaccard: dict
    t_submit: float
    t_done: float
    batch_jobs: int

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.t_submit)


class _Slot:
    def __init__(self, device, params, cap_pairs, cap_jobs):
        import torch
        self.ctx = Context(device, params)
        dev = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=dev)
        self.pa = torch.empty(cap_pairs, dtype=torch.int32, device=dev)
        self.pb = torch.empty(cap_pairs, dtype=torch.int32, device=dev)
        self.inter = torch.empty(cap_pairs, dtype=torch.int64, device=dev)
        self.uni = torch.empty(cap_pairs, dtype=torch.int64, device=dev)
        self.seg_src = torch.empty(cap_jobs, dtype=torch.int64, device=dev)
        self.seg_dst = torch.empty(cap_jobs + 1, dtype=torch.int64, device=dev)
        self.jres = torch.empty(48 * cap_jobs, dtype=torch.uint8, device=dev)
        self.h_src = torch.empty(cap_jobs, dtype=torch.int64).pin_memory()
        self.h_dst = torch.empty(cap_jobs + 1, dtype=torch.int64).pin_memory()
        self.h_inter = torch.empty(cap_pairs, dtype=torch.int64).pin_memory()
        self.h_uni = torch.empty(cap_pairs, dtype=torch.int64).pin_memory()
        self.h_jres = torch.empty(48 * cap_jobs, dtype=torch.uint8).pin_memory()
        self.event = torch.cuda.Event()

    def device_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.pa, self.pb, self.inter, self.uni, self.seg_src,
                                                          self.seg_dst, self.jres))


class Server:
    def __init__(self, A, B, pa, pb, device: int = 0, slots: int = 3, max_batch_pairs: int = 1 << 19,
                 max_batch_jobs: int = 1024, mem_budget_bytes: int = 8 << 30, params: dict | None = None):
        """A, B: prepared DevicePolySets; pa, pb: resident candidate pairs (int32 device tensors)."""
        self.A, self.B, self.pa, self.pb = A, B, pa, pb
        self.cap_pairs, self.cap_jobs = int(max_batch_pairs), int(max_batch_jobs)
        self.slots = [_Slot(device, params, self.cap_pairs, self.cap_jobs) for _ in range(slots)]
        # per-slot context scratch of the persistent form (two item queues, overflow list) is ~48 bytes
        # per pair
        need = sum(s.device_bytes() + 48 * self.cap_pairs for s in self.slots)
        if need > mem_budget_bytes:
            raise ValueError(f"{slots} slots of {max_batch_pairs} pairs need {need} bytes > budget {mem_budget_bytes}")
        self.free = collections.deque(range(slots))
        self.pending = collections.deque()
        self.inflight = collections.deque()
        self.cv = threading.Condition()
        self.done_cv = threading.Condition()
        self.stop = False
        self.batches = 0
        self.batched_jobs = 0
        self.batcher = threading.Thread(target=self._batch_loop, daemon=True)
        self.completer = threading.Thread(target=self._complete_loop, daemon=True)
        self.batcher.start()
        self.completer.start()

    # ------------------------------------------------------------------ client side
    def submit(self, job: Job) -> cf.Future:
        n = job.p1 - job.p0
        if n <= 0 or n > self.cap_pairs or job.p0 < 0 or job.p1 > self.pa.numel():
            raise ValueError(f"job of {n} pairs at [{job.p0}, {job.p1}) does not fit a batch slot")
        fut = cf.Future()
        job.t_submit = time.perf_counter()
        with self.cv:
            self.pending.append((job, fut))
            self.cv.notify()
        return fut

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        with self.done_cv:
            self.done_cv.notify_all()
        self.batcher.join(timeout=10)
        self.completer.join(timeout=10)

    # ------------------------------------------------------------------ server side
    def _batch_loop(self):
        import torch
        while True:
            with self.cv:
                while not self.stop and (not self.pending or not self.free):
                    self.cv.wait(timeout=0.01)
                if self.stop:
                    return
                jobs, npairs = [], 0
                while self.pending and len(jobs) < self.cap_jobs:
                    job, fut = self.pending[0]
                    n = job.p1 - job.p0
                    if npairs + n > self.cap_pairs:
                        break
                    self.pending.popleft()
                    if not fut.set_running_or_notify_cancel():
                        continue                     # cancelled by the client before admission
                    jobs.append((job, fut))
                    npairs += n
                if not jobs:
                    continue
                slot_id = self.free.popleft()
            slot = self.slots[slot_id]
            k = len(jobs)
            src = np.array([j.p0 for j, _ in jobs], dtype=np.int64)
            dst = np.zeros(k + 1, dtype=np.int64)
            np.cumsum([j.p1 - j.p0 for j, _ in jobs], out=dst[1:])
            slot.h_src[:k].copy_(torch.from_numpy(src))
            slot.h_dst[:k + 1].copy_(torch.from_numpy(dst))
            with torch.cuda.stream(slot.stream):
                slot.seg_src[:k].copy_(slot.h_src[:k], non_blocking=True)
                slot.seg_dst[:k + 1].copy_(slot.h_dst[:k + 1], non_blocking=True)
                c = slot.ctx
                c.gather_pairs(self.pa, self.pb, slot.seg_src[:k], slot.seg_dst[:k + 1], slot.pa, slot.pb,
                               stream=slot.stream)
                c.pair_areas(self.A, self.B, slot.pa[:npairs], slot.pb[:npairs], mode=MODE_PERSISTENT,
                             out=(slot.inter, slot.uni), stream=slot.stream)
                c.jaccard_segments(slot.inter, slot.uni, slot.seg_dst[:k + 1], slot.jres, stream=slot.stream)
                slot.h_inter[:npairs].copy_(slot.inter[:npairs], non_blocking=True)
                slot.h_uni[:npairs].copy_(slot.uni[:npairs], non_blocking=True)
                slot.h_jres[:48 * k].copy_(slot.jres[:48 * k], non_blocking=True)
                slot.event.record(slot.stream)
            with self.done_cv:
                self.inflight.append((slot_id, jobs, dst))
                self.batches += 1
                self.batched_jobs += k
                self.done_cv.notify()

    def _complete_loop(self):
        while True:
            with self.done_cv:
                while not self.inflight and not self.stop:
                    self.done_cv.wait(timeout=0.01)
                if not self.inflight and self.stop:
                    return
                slot_id, jobs, dst = self.inflight.popleft()
            slot = self.slots[slot_id]
            slot.event.synchronize()
            k = len(jobs)
            inter = slot.h_inter[:dst[-1]].numpy().copy()
            uni = slot.h_uni[:dst[-1]].numpy().copy()
            jac = Context.decode_jaccard_array(slot.h_jres[:48 * k].numpy())
            with self.cv:
                self.free.append(slot_id)
                self.cv.notify()
            now = time.perf_counter()
            for j, (job, fut) in enumerate(jobs):
                fut.set_result(JobResult(inter[dst[j]:dst[j + 1]], uni[dst[j]:dst[j + 1]], jac[j], job.t_submit,
                                         now, k))


def draw_jobs(rng, tile_pair_off, n_jobs: int, lo: int = 100, hi: int = 50_000):
    """Jobs of one tile each: a contiguous slice of log-uniform [lo, hi] candidate pairs (clipped to
    the tile's pair count), placed uniformly inside the tile's pair range."""
    tpo = np.asarray(tile_pair_off, dtype=np.int64)
    sizes = np.diff(tpo)
    tiles = np.nonzero(sizes >= lo)[0]
    t = rng.choice(tiles, n_jobs)
    want = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), n_jobs))).astype(np.int64)
    n = np.minimum(want, sizes[t])
    start = tpo[t] + (rng.random(n_jobs) * (sizes[t] - n + 1)).astype(np.int64)
    return [Job(int(s), int(s + m), int(tt)) for s, m, tt in zip(start, n, t)]


def run_load(server: Server, jobs, rate_jobs_s: float, rng):
    """Submit `jobs` with Poisson arrivals at rate_jobs_s; return (results, wall seconds)."""
    gaps = rng.exponential(1.0 / rate_jobs_s, len(jobs))
    t0 = time.perf_counter()
    futs = []
    t_next = t0
    for job, g in zip(jobs, gaps):
        t_next += g
        d = t_next - time.perf_counter()
        if d > 0:
            time.sleep(d)
        futs.append(server.submit(job))
    res = [f.result() for f in futs]
    return res, time.perf_counter() - t0


def latency_summary(results, wall_s: float) -> dict:
    lat = np.array([r.latency_ms for r in results])
    pairs = sum(len(r.inter) for r in results)
    return {"jobs": len(results), "pairs": int(pairs), "pairs_per_s": pairs / wall_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch_jobs": float(np.mean([r.batch_jobs for r in results]))}
