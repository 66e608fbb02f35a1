"""Continuous-batching server for cross-comparison jobs over resident polygon sets.

A job asks for the exact intersection/union areas of a contiguous slice of the candidate pairs of
one tile, plus the Jaccard similarities over that slice (Sec. 4.1: the work unit is an image tile;
the aggregator groups tasks into GPU batches). The two polygon sets and their candidate pairs stay
resident in device memory; jobs only name pair ranges.

Device memory and admission. The server is given a device-memory budget. Its fixed part is paid at
construction: per batch slot a library context whose scratch is reserved for the largest batch
(``Context.reserve``: no allocation, hence no device synchronisation, while serving), a CUDA stream
and per-job arrays. The rest of the budget is a pair arena: every batch in flight holds one
contiguous range of it for its pairs' indices and areas (24 bytes per pair). A job is admitted
(in arrival order) only when a slot is free and the arena has room for its pairs next to the other
jobs of the forming batch; otherwise it waits until a batch completes and frees its range. A job
that could never fit (more pairs than a slot or the arena holds) is refused at submit time.

Execution. A batcher thread forms a batch whenever a slot is free and jobs are pending, so jobs that
arrive while other batches run on the GPU join the next batch, and batches on different slots
overlap on the device. Per batch, on the slot's stream:
  1. copy the jobs' (source offset, destination offset) pairs host -> device,
  2. gather the jobs' pair slices into the batch's arena range (``sccg_gather_pairs``),
  3. exact pair areas, persistent form (``sccg_pair_areas``),
  4. per-job Jaccard (``sccg_jaccard_segments``),
  5. copy areas and Jaccard structs device -> pinned host, record an event.
Each slot has its own completer thread that waits for its batch's event, so batches are resolved in
the order they finish, not the order they were formed.

Latency. A job carries its scheduled arrival time (``t_arrival``, set by the client that replays an
arrival trace; the submit time otherwise); a result's latency runs from that arrival to the moment
its areas and Jaccard are in host memory, so a client or batcher that falls behind shows up in the
latency rather than hiding it. A job whose future the client cancels before it is admitted to a
batch is dropped. Each job's handle is a Ticket (result with an optional timeout, cancel): one
condition per server is notified per completed batch, which keeps the host cost per job small at
tens of thousands of jobs per second.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time

import numpy as np

from . import Context, MODE_PERSISTENT

ARENA_BYTES_PER_PAIR = 4 + 4 + 8 + 8     # pair indices and the two areas of one pair in a batch
SCRATCH_BYTES_PER_PAIR = 48              # the persistent form's per-pair queue scratch (context)


@dataclasses.dataclass
class Job:
    p0: int                 # first candidate-pair index (into the resident pair list)
    p1: int                 # one past the last
    tile: int = -1
    t_arrival: float = 0.0  # scheduled arrival (perf_counter clock); 0: the submit time


@dataclasses.dataclass
class JobResult:
    inter: np.ndarray       # int64 [p1 - p0]
    uni: np.ndarray         # int64 [p1 - p0]
    jaccard: dict
    t_arrival: float
    t_done: float
    batch_jobs: int

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.t_arrival)


class _BatchOut:
    """The results of one batch, shared by its jobs' tickets: completing a batch is one write
    (ready), whatever its number of jobs; each ticket cuts its own result out when asked."""
    __slots__ = ("inter", "uni", "jac", "dst", "t_done", "k", "ready")

    def __init__(self):
        self.ready = False


class Ticket:
    """The handle of a submitted job (a light future: one shared condition per server rather than a
    lock per job). result(timeout) blocks until the job's batch has completed; cancel() withdraws a
    job that has not been admitted to a batch yet."""
    # state: 0 queued, 1 admitted (to batch _bo as its job _j), 2 done, 3 cancelled
    __slots__ = ("job", "_srv", "_res", "_state", "_bo", "_j")

    def __init__(self, job, srv):
        self.job, self._srv, self._res, self._state, self._bo, self._j = job, srv, None, 0, None, 0

    def _finished(self) -> bool:
        if self._state == 1 and self._bo is not None and self._bo.ready:
            bo, j = self._bo, self._j
            self._res = JobResult(bo.inter[bo.dst[j]:bo.dst[j + 1]], bo.uni[bo.dst[j]:bo.dst[j + 1]], bo.jac[j],
                                  self.job.t_arrival, bo.t_done, bo.k)
            self._state = 2
        return self._state >= 2

    def cancel(self) -> bool:
        with self._srv.cv:
            if self._state == 0:
                self._state = 3
            return self._state == 3

    def cancelled(self) -> bool:
        return self._state == 3

    def done(self) -> bool:
        return self._finished()

    def result(self, timeout: float | None = None):
        if not self._finished():
            with self._srv.done_cv:
                ok = self._srv.done_cv.wait_for(self._finished, timeout)
            if not ok:
                raise TimeoutError("job not completed in time")
        if self._state == 3:
            raise cf.CancelledError()
        return self._res


class Arena:
    """First-fit allocator of contiguous pair ranges [0, capacity) (host bookkeeping only)."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free = [(0, self.capacity)]          # sorted, disjoint (start, length)

    def largest(self) -> int:
        return max((n for _, n in self.free), default=0)

    def take(self, n: int) -> int:
        for k, (s, m) in enumerate(self.free):
            if m >= n:
                if m == n:
                    del self.free[k]
                else:
                    self.free[k] = (s + n, m - n)
                return s
        raise MemoryError(n)

    def give(self, s: int, n: int):
        self.free.append((s, n))
        self.free.sort()
        merged = []
        for a, m in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + m)
            else:
                merged.append((a, m))
        self.free = merged


class _Slot:
    def __init__(self, device, params, cap_pairs, cap_jobs):
        import torch
        self.ctx = Context(device, params)
        self.ctx.reserve(cap_pairs)
        dev = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=dev)
        self.seg_src = torch.empty(cap_jobs, dtype=torch.int64, device=dev)
        self.seg_dst = torch.empty(cap_jobs + 1, dtype=torch.int64, device=dev)
        self.jres = torch.empty(48 * cap_jobs, dtype=torch.uint8, device=dev)
        self.h_src = torch.empty(cap_jobs, dtype=torch.int64).pin_memory()
        self.h_dst = torch.empty(cap_jobs + 1, dtype=torch.int64).pin_memory()
        self.h_inter = torch.empty(cap_pairs, dtype=torch.int64).pin_memory()
        self.h_uni = torch.empty(cap_pairs, dtype=torch.int64).pin_memory()
        self.h_jres = torch.empty(48 * cap_jobs, dtype=torch.uint8).pin_memory()
        self.event = torch.cuda.Event()
        self.batch = None           # (jobs, dst offsets, arena start, pairs) of the batch in flight
        self.cv = threading.Condition()

    @staticmethod
    def fixed_bytes(cap_pairs, cap_jobs) -> int:
        return cap_jobs * 8 + (cap_jobs + 1) * 8 + 48 * cap_jobs + SCRATCH_BYTES_PER_PAIR * cap_pairs


class Server:
    def __init__(self, A, B, pa, pb, device: int = 0, slots: int = 3, max_batch_pairs: int = 1 << 19,
                 max_batch_jobs: int = 1024, mem_budget_bytes: int = 8 << 30, arena_pairs: int | None = None,
                 params: dict | None = None):
        """A, B: prepared DevicePolySets; pa, pb: resident candidate pairs (int32 device tensors).
        mem_budget_bytes bounds the slots' fixed memory plus the pair arena; arena_pairs (default:
        the rest of the budget, at most slots x max_batch_pairs) sets the arena explicitly."""
        import torch
        self.A, self.B, self.pa, self.pb = A, B, pa, pb
        self.cap_pairs, self.cap_jobs = int(max_batch_pairs), int(max_batch_jobs)
        fixed = slots * _Slot.fixed_bytes(self.cap_pairs, self.cap_jobs)
        room = (mem_budget_bytes - fixed) // ARENA_BYTES_PER_PAIR
        if arena_pairs is None:
            arena_pairs = min(room, slots * self.cap_pairs)
        if fixed > mem_budget_bytes or arena_pairs > room or arena_pairs < 1:
            raise ValueError(f"{slots} slots of {max_batch_pairs} pairs and an arena of {arena_pairs} pairs do not "
                             f"fit a budget of {mem_budget_bytes} bytes")
        self.mem_budget_bytes = int(mem_budget_bytes)
        dev = torch.device("cuda", device)
        self.arena = Arena(arena_pairs)
        self.a_pa = torch.empty(arena_pairs, dtype=torch.int32, device=dev)
        self.a_pb = torch.empty(arena_pairs, dtype=torch.int32, device=dev)
        self.a_inter = torch.empty(arena_pairs, dtype=torch.int64, device=dev)
        self.a_uni = torch.empty(arena_pairs, dtype=torch.int64, device=dev)
        self.slots = [_Slot(device, params, self.cap_pairs, self.cap_jobs) for _ in range(slots)]
        self.free = collections.deque(range(slots))
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.done_cv = threading.Condition()     # notified whenever a batch's tickets complete
        self.stop = False
        self.batches = 0
        self.batched_jobs = 0
        self.waited_for_memory = 0       # batch formations cut short because the arena was full
        self.batcher = threading.Thread(target=self._batch_loop, daemon=True)
        self.completers = [threading.Thread(target=self._complete_loop, args=(k,), daemon=True)
                           for k in range(slots)]
        self.batcher.start()
        for t in self.completers:
            t.start()

    @property
    def arena_pairs(self) -> int:
        return self.arena.capacity

    def device_bytes(self) -> int:
        return (len(self.slots) * _Slot.fixed_bytes(self.cap_pairs, self.cap_jobs) +
                self.arena.capacity * ARENA_BYTES_PER_PAIR)

    # ------------------------------------------------------------------ client side
    def _check(self, job: Job):
        n = job.p1 - job.p0
        if n <= 0 or n > self.cap_pairs or n > self.arena.capacity or job.p0 < 0 or job.p1 > self.pa.numel():
            raise ValueError(f"job of {n} pairs at [{job.p0}, {job.p1}) does not fit a batch slot or the pair arena")

    def submit(self, job: Job) -> Ticket:
        return self.submit_many([job])[0]

    def submit_many(self, jobs) -> list:
        """Queue jobs in the given order (one lock acquisition); jobs without a scheduled arrival
        time get the submit time. Returns one Ticket per job."""
        for j in jobs:
            self._check(j)
        now = time.perf_counter()
        tickets = [Ticket(j, self) for j in jobs]
        with self.cv:
            for j in jobs:
                if not j.t_arrival:
                    j.t_arrival = now
            self.pending.extend(tickets)
            self.cv.notify()
        return tickets

    def drain(self, timeout: float | None = None) -> bool:
        """Wait until no job is queued and no batch is in flight (the results of every submitted job
        are then ready; reading them costs the caller, not the server). False on timeout."""
        def idle():
            with self.cv:
                return not self.pending and len(self.free) == len(self.slots)
        with self.done_cv:
            return self.done_cv.wait_for(idle, timeout)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        with self.done_cv:
            self.done_cv.notify_all()
        for s in self.slots:
            with s.cv:
                s.cv.notify_all()
        self.batcher.join(timeout=10)
        for t in self.completers:
            t.join(timeout=10)

    # ------------------------------------------------------------------ server side
    def _form(self):
        """Pending jobs in arrival order that fit one batch and the arena's largest free range
        (called with self.cv held), admitted to one batch record. Cancelled jobs are dropped."""
        jobs, npairs = [], 0
        bo = _BatchOut()
        room = min(self.cap_pairs, self.arena.largest())
        while self.pending and len(jobs) < self.cap_jobs:
            t = self.pending[0]
            if t._state == 3:                    # cancelled by the client before admission
                self.pending.popleft()
                continue
            n = t.job.p1 - t.job.p0
            if npairs + n > room:
                if npairs + n <= self.cap_pairs:
                    self.waited_for_memory += 1
                break
            self.pending.popleft()
            t._bo, t._j = bo, len(jobs)
            t._state = 1
            jobs.append(t)
            npairs += n
        return jobs, npairs, bo

    def _batch_loop(self):
        import torch
        while True:
            with self.cv:
                while True:
                    if self.stop:
                        return
                    if self.pending and self.free:
                        jobs, npairs, bo = self._form()
                        if jobs:
                            break
                    self.cv.wait(timeout=0.01)
                slot_id = self.free.popleft()
                start = self.arena.take(npairs)
            slot = self.slots[slot_id]
            k = len(jobs)
            src = np.array([t.job.p0 for t in jobs], dtype=np.int64)
            dst = np.zeros(k + 1, dtype=np.int64)
            np.cumsum([t.job.p1 - t.job.p0 for t in jobs], out=dst[1:])
            slot.h_src[:k].copy_(torch.from_numpy(src))
            slot.h_dst[:k + 1].copy_(torch.from_numpy(dst))
            rng = slice(start, start + npairs)
            with torch.cuda.stream(slot.stream):
                c = slot.ctx
                # host <-> device copies by the SMs (sccg_copy), like the pipelined front end's
                c.copy(slot.seg_src[:k], slot.h_src[:k], stream=slot.stream)
                c.copy(slot.seg_dst[:k + 1], slot.h_dst[:k + 1], stream=slot.stream)
                c.gather_pairs(self.pa, self.pb, slot.seg_src[:k], slot.seg_dst[:k + 1], self.a_pa[rng],
                               self.a_pb[rng], stream=slot.stream)
                c.pair_areas(self.A, self.B, self.a_pa[rng], self.a_pb[rng], mode=MODE_PERSISTENT,
                             out=(self.a_inter[rng], self.a_uni[rng]), stream=slot.stream)
                c.jaccard_segments(self.a_inter[rng], self.a_uni[rng], slot.seg_dst[:k + 1], slot.jres,
                                   stream=slot.stream)
                c.copy(slot.h_inter[:npairs], self.a_inter[rng], stream=slot.stream)
                c.copy(slot.h_uni[:npairs], self.a_uni[rng], stream=slot.stream)
                c.copy(slot.h_jres[:48 * k], slot.jres[:48 * k], stream=slot.stream)
                slot.event.record(slot.stream)
            with slot.cv:
                slot.batch = (jobs, dst, start, npairs, bo)
                slot.cv.notify()
            with self.cv:
                self.batches += 1
                self.batched_jobs += k

    def _complete_loop(self, slot_id: int):
        slot = self.slots[slot_id]
        while True:
            with slot.cv:
                while slot.batch is None and not self.stop:
                    slot.cv.wait(timeout=0.01)
                if slot.batch is None:
                    return
                jobs, dst, start, npairs, bo = slot.batch
            slot.event.synchronize()
            now = time.perf_counter()
            k = len(jobs)
            # out of the slot's pinned staging before the slot is reused (torch's copy runs on several
            # cores and without the interpreter lock)
            bo.inter = slot.h_inter[:npairs].clone().numpy()
            bo.uni = slot.h_uni[:npairs].clone().numpy()
            bo.jac = Context.decode_jaccard_array(slot.h_jres[:48 * k].numpy())
            bo.dst, bo.t_done, bo.k = dst, now, k
            with slot.cv:
                slot.batch = None
            with self.cv:
                self.arena.give(start, npairs)
                self.free.append(slot_id)
                self.cv.notify()
            bo.ready = True                      # every ticket of the batch is done (no per-job work here)
            with self.done_cv:
                self.done_cv.notify_all()


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
    """Replay a Poisson arrival trace at rate_jobs_s: every job is stamped with its scheduled arrival
    time and submitted once that time has passed (all jobs that are due go in one call, so a slow
    client delays submission, which then counts in the latency, instead of thinning the load; between
    calls the client sleeps up to 1 ms instead of spinning). Returns (results, wall seconds from the
    first scheduled arrival to the last completion)."""
    arrivals = np.cumsum(rng.exponential(1.0 / rate_jobs_s, len(jobs)))
    futs = []
    k = 0
    t0 = time.perf_counter() + 0.002
    while k < len(jobs):
        now = time.perf_counter() - t0
        j = int(np.searchsorted(arrivals, now, side="right"))
        if j > k:
            for i in range(k, j):
                jobs[i].t_arrival = t0 + float(arrivals[i])
            futs += server.submit_many(jobs[k:j])
            k = j
        if k < len(jobs):
            # sleep (releasing the interpreter to the server's threads) rather than spin: jobs that
            # fall due meanwhile go in with the next call, stamped with their scheduled arrival
            wait = float(arrivals[k]) - (time.perf_counter() - t0)
            time.sleep(min(max(wait, 0.0002), 0.001))
    server.drain()                       # every job served before any result is cut out of its batch
    res = [f.result() for f in futs]
    return res, max(r.t_done for r in res) - (t0 + float(arrivals[0]))


def latency_summary(results, wall_s: float, offered_jobs_per_s: float | None = None) -> dict:
    lat = np.array([r.latency_ms for r in results])
    pairs = sum(len(r.inter) for r in results)
    out = {"jobs": len(results), "pairs": int(pairs), "pairs_per_s": pairs / wall_s,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_batch_jobs": float(np.mean([r.batch_jobs for r in results]))}
    if offered_jobs_per_s:
        out["offered_pairs_per_s"] = offered_jobs_per_s * pairs / len(results)
        out["achieved_over_offered"] = out["pairs_per_s"] / out["offered_pairs_per_s"]
    return out
