"""Tile tasks admitted to GPU streams by the state of their input buffers.

The paper balances its pipeline by watching the aggregator's input buffer (Sec. 4.2): a full buffer
means the GPU is congested, an empty one that it is idle, and tasks migrate accordingly, the
smallest first (Sec. 5.6 evaluates it). Here every task runs on the GPU (there is no CPU execution
path); what is scheduled is which CUDA stream a tile task is admitted to. Each stream has a bounded
host-side input buffer of tasks not yet launched and a window of tasks launched but not finished.

Policies:
  static   tile t goes to stream t mod n_streams; when that stream's buffer is full the producer
           waits for it, whatever the other streams are doing.
  dynamic  a new task goes to the stream whose buffer holds the least work (pairs); whenever a
           stream is idle (empty buffer, nothing in flight) while another's buffer is full, the
           smallest tasks of the full buffer move to the idle stream (the full/empty triggers of
           Sec. 4.2, with GPU streams in the place of CPU workers).

The executor is abstract (launch a task on a stream, ask whether it finished), so the scheduling
logic runs on the host alone in tests with synthetic task durations and injected stalls; the GPU
executor launches the per-tile pair-area kernel of `sccg_pair_areas` (PLAIN) on the tile's slice of
the candidate pairs and records an event.
"""
from __future__ import annotations

import collections
import dataclasses
import time


@dataclasses.dataclass
class Task:
    tile: int
    p0: int          # candidate pairs p0 .. p1 - 1
    p1: int

    @property
    def size(self) -> int:
        return self.p1 - self.p0


class Scheduler:
    def __init__(self, executor, n_streams: int = 4, depth: int = 4, window: int = 2, policy: str = "dynamic"):
        if policy not in ("static", "dynamic"):
            raise ValueError(policy)
        self.ex = executor
        self.n = int(n_streams)
        self.depth = int(depth)          # input buffer capacity per stream (tasks not yet launched)
        self.window = int(window)        # tasks launched and not finished per stream
        self.policy = policy
        self.buf = [collections.deque() for _ in range(self.n)]
        self.flight = [collections.deque() for _ in range(self.n)]
        self.done = []                   # (task, stream) in completion order
        self.migrations = 0
        self.producer_waits = 0

    # ------------------------------------------------------------------ buffer state
    def _pending_work(self, s: int) -> int:
        return sum(t.size for t in self.buf[s])

    def _retire(self):
        for s in range(self.n):
            while self.flight[s] and self.ex.finished(self.flight[s][0][1]):
                t, _ = self.flight[s].popleft()
                self.done.append((t, s))

    def _launch_ready(self):
        for s in range(self.n):
            while self.buf[s] and len(self.flight[s]) < self.window:
                t = self.buf[s].popleft()
                self.flight[s].append((t, self.ex.launch(s, t)))

    def _migrate(self):
        if self.policy != "dynamic":
            return
        for idle in range(self.n):
            if self.buf[idle] or self.flight[idle]:
                continue
            full = max(range(self.n), key=lambda s: len(self.buf[s]))
            if len(self.buf[full]) < self.depth:
                continue
            # the smallest tasks of the congested buffer, up to half of it
            moved = sorted(self.buf[full], key=lambda t: t.size)[: max(1, len(self.buf[full]) // 2)]
            keep = [t for t in self.buf[full] if not any(t is m for m in moved)]
            self.buf[full] = collections.deque(keep)
            self.buf[idle].extend(moved)
            self.migrations += len(moved)

    def _step(self):
        self._retire()
        self._migrate()
        self._launch_ready()

    # ------------------------------------------------------------------ driver
    def run(self, tasks):
        """Admit every task in order and wait for all of them; returns (elapsed seconds on the
        executor's clock, completion list of (task, stream)). The executor's idle() is called when
        nothing can move until a launched task finishes."""
        t0 = self.ex.now()
        for k, task in enumerate(tasks):
            while True:
                self._step()
                if self.policy == "static":
                    s = k % self.n
                else:
                    s = min(range(self.n), key=lambda j: (self._pending_work(j) +
                                                          sum(t.size for t, _ in self.flight[j]), j))
                if len(self.buf[s]) < self.depth:
                    self.buf[s].append(task)
                    break
                self.producer_waits += 1
                self.ex.idle()
        while any(self.buf) or any(self.flight):
            n_done = len(self.done)
            self._step()
            if len(self.done) == n_done:
                self.ex.idle()
        return self.ex.now() - t0, self.done


class SimExecutor:
    """Host-only executor for tests: stream s runs its launched tasks one after another, a task taking
    size * cost[s] units of a simulated clock; idle() advances the clock to the next completion.
    Raising a stream's cost injects a stall (a congested stream)."""

    def __init__(self, cost):
        self.cost = list(cost)
        self.clock = 0.0
        self.free_at = [0.0] * len(self.cost)
        self.ends = []

    def now(self) -> float:
        return self.clock

    def launch(self, s: int, task: Task):
        end = max(self.clock, self.free_at[s]) + task.size * self.cost[s]
        self.free_at[s] = end
        self.ends.append(end)
        return end

    def finished(self, handle) -> bool:
        return handle <= self.clock

    def idle(self):
        later = [e for e in self.ends if e > self.clock]
        if later:
            self.clock = min(later)
        self.ends = later


def tile_tasks(tile_pair_off) -> list:
    """One task per tile with candidate pairs, in tile order."""
    return [Task(t, int(tile_pair_off[t]), int(tile_pair_off[t + 1])) for t in range(len(tile_pair_off) - 1)
            if tile_pair_off[t + 1] > tile_pair_off[t]]


class GpuExecutor:
    """Launches a tile task's pair areas (one warp per pair, one kernel launch: the per-tile form of
    Sec. 4.1) on CUDA stream s and records an event after it."""

    def __init__(self, ctx, A, B, pa, pb, inter, uni, n_streams: int, device: int = 0):
        import torch
        self.ctx, self.A, self.B, self.pa, self.pb, self.inter, self.uni = ctx, A, B, pa, pb, inter, uni
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]

    def launch(self, s: int, task: Task):
        import torch
        from . import MODE_PLAIN
        st = self.streams[s]
        sl = slice(task.p0, task.p1)
        self.ctx.pair_areas(self.A, self.B, self.pa[sl], self.pb[sl], mode=MODE_PLAIN,
                            out=(self.inter[sl], self.uni[sl]), stream=st)
        ev = torch.cuda.Event()
        ev.record(st)
        return ev

    @staticmethod
    def finished(handle) -> bool:
        return handle.query()

    @staticmethod
    def now() -> float:
        return time.perf_counter()

    @staticmethod
    def idle():
        time.sleep(0)
