"""Host-to-host cross-comparison with the copies overlapped (the pipelined front end of Sec. 4.1,
Fig. 6: while the GPU works on one batch of tiles, the next batch is being moved to it).

The two polygon sets live in pinned host memory, grouped by tile. They are cut into chunks of
consecutive tiles; chunk k+1 is copied host -> device on a copy stream while chunk k is prepared,
filtered and compared on the compute stream, into two alternating device buffers. Chunk sizes (in
vertices, at tile boundaries) grow by a constant factor, so that the first copy, which nothing
overlaps, is short while each later copy still ends before the work on the chunk before it (the
copy moves a vertex faster than the kernels consume one). Results go back to pinned host memory on
a third stream as each chunk finishes. The copies are made by the SMs (sccg_copy: a few CTAs that
read or write the pinned host buffers directly, on high-priority streams so that they start beside
the comparison kernels); copy="engine" uses the DMA copy engines instead (cudaMemcpyAsync), whose
host-to-device rate on the measured boxes dropped to about an eighth for 0.1-0.2 s at a time while
the SM copies held the link's full rate. Each chunk's
candidate pairs and areas land in one device result array (and are copied back to pinned host memory
as they finish); the Jaccard reduction runs once over all pairs at the end, so J and J' are the same
bits as for one call over the whole sets. Every step runs in the library's kernels (chunk-local pair
indices are rebased on the device by sccg_rebase_pairs); the chunks' vertex offset and tile arrays
are rebased once, when the pipeline is built, into pinned buffers of their own, so that a run only
issues copies and launches.
"""
from __future__ import annotations

import numpy as np

from . import MODE_PERSISTENT, SccgError, SCCG_ECAPACITY


def _pin(a, dtype):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=dtype))
    return t.pin_memory()


class HostSet:
    """A polygon set in pinned host memory (CSR, tiles non-decreasing), ready for chunked copies."""

    def __init__(self, off, xy, tile):
        self.off = _pin(off, np.int64)
        self.xy = _pin(xy, np.int32)
        self.tile = _pin(tile, np.int32)
        self.n = self.off.numel() - 1
        self.off_np = self.off.numpy()
        self.tile_np = self.tile.numpy()

    @classmethod
    def from_polyset(cls, ps):
        return cls(ps.off, ps.xy, ps.tile)

    def range_of_tiles(self, t0: int, t1: int):
        """Polygons [i0, i1) of tiles [t0, t1)."""
        return (int(np.searchsorted(self.tile_np, t0, "left")), int(np.searchsorted(self.tile_np, t1, "left")))

    def bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.off, self.xy, self.tile))


class _Side:
    """Device buffers of one set for one of the two alternating chunk slots."""

    def __init__(self, dev, max_n: int, max_v: int):
        import torch
        self.off = torch.empty(max_n + 1, dtype=torch.int64, device=dev)
        self.xy = torch.empty(max(2 * max_v, 2), dtype=torch.int32, device=dev)
        self.tile = torch.empty(max(max_n, 1), dtype=torch.int32, device=dev)
        self.mbr = torch.empty((max(max_n, 1), 4), dtype=torch.int32, device=dev)
        self.area = torch.empty(max(max_n, 1), dtype=torch.int64, device=dev)
        self.raster = None      # pixel rasters of the chunk, grown to the largest chunk by the first run


class Pipeline:
    """Chunked, copy-overlapped cross comparison of two HostSets on one device.

    chunks: number of tile chunks (the copy of chunk k+1 overlaps the work on chunk k).
    growth: size ratio of consecutive chunks (1: equal chunks)."""

    def __init__(self, ctx, A: HostSet, B: HostSet, n_tiles: int, chunks: int = 3, mode: int = MODE_PERSISTENT,
                 initial_pairs: int | None = None, growth: float = 1.5, copy: str = "sm"):
        import torch
        if copy not in ("sm", "engine"):
            raise ValueError("copy: 'sm' or 'engine'")
        self.ctx, self.A, self.B, self.mode, self.copy = ctx, A, B, mode, copy
        self.dev = torch.device("cuda", ctx.device)
        self.chunks = self._cut(A, B, n_tiles, max(1, min(chunks, n_tiles)), growth)
        self.ranges = [(A.range_of_tiles(t0, t1), B.range_of_tiles(t0, t1)) for t0, t1 in self.chunks]
        max_na = max(a1 - a0 for (a0, a1), _ in self.ranges)
        max_nb = max(b1 - b0 for _, (b0, b1) in self.ranges)
        max_va = max(int(A.off_np[a1] - A.off_np[a0]) for (a0, a1), _ in self.ranges)
        max_vb = max(int(B.off_np[b1] - B.off_np[b0]) for _, (b0, b1) in self.ranges)
        self.slots = [(_Side(self.dev, max_na, max_va), _Side(self.dev, max_nb, max_vb)) for _ in range(2)]
        # the copy streams at the highest priority: their few CTAs are scheduled as soon as an SM has room
        self.copy_stream = torch.cuda.Stream(device=self.dev, priority=-1)
        self.compute_stream = torch.cuda.Stream(device=self.dev)
        self.d2h_stream = torch.cuda.Stream(device=self.dev, priority=-1)
        self.done = torch.cuda.Event()
        self.copied = [torch.cuda.Event() for _ in range(2)]
        self.freed = [torch.cuda.Event() for _ in range(2)]
        self._alloc_results(initial_pairs if initial_pairs else max(A.n + B.n, 1 << 16))
        # chunk-local offsets (from 0) and tiles (from the chunk's first tile), pinned, per chunk
        self.staged = []
        for k, ((a0, a1), (b0, b1)) in enumerate(self.ranges):
            t0 = self.chunks[k][0]
            per = []
            for S, i0, i1 in ((A, a0, a1), (B, b0, b1)):
                off = _pin(S.off_np[i0:i1 + 1] - S.off_np[i0], np.int64)
                tile = _pin(S.tile_np[i0:i1] - t0, np.int32)
                per.append((off, tile, int(S.off_np[i0]), int(S.off_np[i1])))
            self.staged.append(per)
        self.h2d_bytes = sum(off.numel() * 8 + tile.numel() * 4 + (v1 - v0) * 8
                             for per in self.staged for off, tile, v0, v1 in per)

    @staticmethod
    def _cut(A: HostSet, B: HostSet, n_tiles: int, k: int, growth: float):
        """Tile ranges of k chunks whose vertex counts grow by `growth` (cut at tile boundaries)."""
        verts = np.zeros(n_tiles, dtype=np.float64)
        for S in (A, B):
            if S.n:
                np.add.at(verts, S.tile_np, np.diff(S.off_np).astype(np.float64))
        cum = np.concatenate([[0.0], np.cumsum(verts)])
        w = np.power(float(growth), np.arange(k))
        targets = np.cumsum(w) / w.sum() * cum[-1]
        edges = [0]
        for t in targets[:-1]:
            e = int(np.searchsorted(cum, t, "left"))
            edges.append(min(max(e, edges[-1] + 1), n_tiles))
        edges.append(n_tiles)
        return [(edges[i], edges[i + 1]) for i in range(k) if edges[i + 1] > edges[i]]

    def _alloc_results(self, cap: int, keep: int = 0):
        import torch
        old = getattr(self, "res", None)
        if old is not None:
            self.d2h_stream.synchronize()    # the old pinned buffers are complete before they are copied
        res = {"pa": torch.empty(cap, dtype=torch.int32, device=self.dev),
               "pb": torch.empty(cap, dtype=torch.int32, device=self.dev),
               "inter": torch.empty(cap, dtype=torch.int64, device=self.dev),
               "uni": torch.empty(cap, dtype=torch.int64, device=self.dev)}
        host = {k: torch.empty(cap, dtype=v.dtype).pin_memory() for k, v in res.items()}
        if old is not None and keep:
            for k in res:
                res[k][:keep].copy_(old[k][:keep])
                host[k][:keep].copy_(self.host[k][:keep])
        self.res, self.host, self.cap = res, host, cap

    def _copy_in(self, slot: int, k: int):
        """Host -> device copies of chunk k into `slot` on the copy stream (after the work that last
        used the slot's device buffers)."""
        import torch
        with torch.cuda.stream(self.copy_stream):
            self.copy_stream.wait_event(self.freed[slot])
            for side, S, (off, tile, v0, v1) in zip(self.slots[slot], (self.A, self.B), self.staged[k]):
                n = tile.numel()
                self._copy(side.off[:n + 1], off, self.copy_stream)
                self._copy(side.tile[:n], tile, self.copy_stream)
                self._copy(side.xy[:2 * (v1 - v0)], S.xy[2 * v0:2 * v1], self.copy_stream)
            self.copied[slot].record(self.copy_stream)

    def _copy(self, dst, src, stream):
        if self.copy == "sm":
            self.ctx.copy(dst, src, stream=stream)
        else:
            dst.copy_(src, non_blocking=True)

    def run(self):
        """All candidate pairs (indices into the whole sets), their areas and the Jaccard result, in
        host memory: (pa, pb, inter, uni) numpy views of pinned buffers that the next run overwrites
        (copy them to keep them), and the Jaccard dict."""
        import torch
        ctx = self.ctx
        cs = self.compute_stream
        P = 0
        self._copy_in(0, 0)
        for k in range(len(self.chunks)):
            slot = k % 2
            if k + 1 < len(self.chunks):
                self._copy_in(1 - slot, k + 1)
            cs.wait_event(self.copied[slot])
            sa, sb = self.slots[slot]
            (a0, a1), (b0, b1) = self.ranges[k]
            with torch.cuda.stream(cs):
                A, B = ctx.prepare_sets(
                    [(sa.off[:a1 - a0 + 1], sa.xy, sa.tile[:a1 - a0], (sa.mbr, sa.area, sa.raster)),
                     (sb.off[:b1 - b0 + 1], sb.xy, sb.tile[:b1 - b0], (sb.mbr, sb.area, sb.raster))], stream=cs)
                sa.raster = A.raster if A.raster is not None else sa.raster
                sb.raster = B.raster if B.raster is not None else sb.raster
                while True:
                    try:
                        pa, pb = ctx.candidate_pairs(A, B, capacity=self.cap - P, stream=cs,
                                                     out=(self.res["pa"][P:], self.res["pb"][P:]))
                        break
                    except SccgError as e:
                        if e.status != SCCG_ECAPACITY:
                            raise
                        need = ctx.candidate_pairs(A, B, stream=cs)[0].numel()
                        self._alloc_results(int((P + need) * 1.5) + 1, keep=P)
                n = pa.numel()
                if n:
                    ctx.pair_areas(A, B, pa, pb, mode=self.mode, stream=cs,
                                   out=(self.res["inter"][P:P + n], self.res["uni"][P:P + n]))
                    ctx.rebase_pairs(pa, pb, a0, b0, stream=cs)
                self.freed[slot].record(cs)
            if n:
                self.done.record(cs)
                self.d2h_stream.wait_event(self.done)
                with torch.cuda.stream(self.d2h_stream):
                    for key in ("pa", "pb", "inter", "uni"):
                        self._copy(self.host[key][P:P + n], self.res[key][P:P + n], self.d2h_stream)
            P += n
        with torch.cuda.stream(cs):
            J = ctx.jaccard(self.res["inter"][:P], self.res["uni"][:P], stream=cs)
        cs.synchronize()
        self.d2h_stream.synchronize()
        self.d2h_bytes = P * (4 + 4 + 8 + 8) + 48
        return (self.host["pa"][:P].numpy(), self.host["pb"][:P].numpy(), self.host["inter"][:P].numpy(),
                self.host["uni"][:P].numpy(), J)
