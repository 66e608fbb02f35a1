"""Seeded synthetic polygon sets that stand in for the paper's segmentation results.

The paper's 18 brain-tumour datasets (Sec. 5.1) are not available, so every input here is drawn
from a numpy ``Generator(PCG64(seed))`` with the shapes of the paper's workloads: nucleus-sized
polygons (mean ~150 px, Sec. 5.1), half a million to millions of polygons per result set, polygons
grouped per image tile (Sec. 2.1, Sec. 4.1), and a second result set that resembles the first
(Sec. 2.1: two segmentations of the same image).

This module only *draws* inputs. It holds none of the cross-comparison arithmetic (no MBRs, no
point-in-polygon, no areas): both the CUDA path and the CPU oracle read the arrays it returns.

A polygon set is stored as CSR:
  off  int64[n+1]  vertex offsets; polygon i owns vertices off[i] .. off[i+1]-1
  xy   int32[2*V]  interleaved (x, y) vertex coordinates; the ring is closed implicitly
  tile int32[n]    tile id of the polygon's generating centre, non-decreasing
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np


@dataclasses.dataclass
class PolySet:
    off: np.ndarray   # int64 [n+1]
    xy: np.ndarray    # int32 [2*V]
    tile: np.ndarray  # int32 [n]

    @property
    def n(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def n_vertices(self) -> int:
        return int(self.off[-1])

    def polygon(self, i: int) -> np.ndarray:
        """Vertices of polygon i as an int32 [k, 2] array."""
        return self.xy[2 * self.off[i]: 2 * self.off[i + 1]].reshape(-1, 2)

    def sha256(self) -> str:
        h = hashlib.sha256()
        for a in (self.off, self.xy, self.tile):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


@dataclasses.dataclass
class Workload:
    name: str
    A: PolySet
    B: PolySet
    n_tiles: int
    tile_px: int
    seed: int


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def from_rings(rings, tiles=None) -> PolySet:
    """Build a PolySet from a list of [k, 2] integer vertex rings (used by tests and examples)."""
    rings = [np.asarray(r, dtype=np.int64).reshape(-1, 2) for r in rings]
    counts = np.array([len(r) for r in rings], dtype=np.int64)
    off = np.zeros(len(rings) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    xy = (np.concatenate(rings).astype(np.int32).reshape(-1) if rings
          else np.zeros(0, dtype=np.int32))
    tile = (np.zeros(len(rings), dtype=np.int32) if tiles is None
            else np.asarray(tiles, dtype=np.int32))
    return PolySet(off=off, xy=xy, tile=tile)


# ----------------------------------------------------------------------------------------------
# ring construction helpers (vectorised over many polygons)
# ----------------------------------------------------------------------------------------------

def _segment_ids(counts: np.ndarray):
    """For a CSR count vector return (owner polygon of each element, index within its polygon)."""
    counts = counts.astype(np.int64)
    tot = int(counts.sum())
    owner = np.repeat(np.arange(counts.shape[0], dtype=np.int64), counts)
    start = np.cumsum(counts) - counts
    k = np.arange(tot, dtype=np.int64) - np.repeat(start, counts)
    return owner, k


def _dedup_rings(x: np.ndarray, y: np.ndarray, counts: np.ndarray):
    """Drop vertices equal to their cyclic predecessor; return (x, y, new counts)."""
    owner, k = _segment_ids(counts)
    start = np.cumsum(counts) - counts
    prev = np.arange(x.shape[0], dtype=np.int64) - 1
    first = k == 0
    prev[first] = (start + counts - 1)[owner[first]]
    keep = (x != x[prev]) | (y != y[prev])
    new_counts = np.bincount(owner[keep], minlength=counts.shape[0]).astype(np.int64)
    return x[keep], y[keep], new_counts


def _pack(x, y, counts, tiles) -> PolySet:
    off = np.zeros(counts.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    xy = np.empty(2 * x.shape[0], dtype=np.int32)
    xy[0::2] = x
    xy[1::2] = y
    return PolySet(off=off, xy=xy, tile=np.asarray(tiles, dtype=np.int32))


def star_rings(rng, cx, cy, s, nv, kind="nucleus"):
    """Star-shaped integer rings around centres (cx, cy) with MBR target s and nv vertices.

    Angles theta_k = 2*pi*(k + u_k)/nv with u_k ~ U[0, 1) are strictly increasing, so the real ring is
    star-shaped. Radii: 'nucleus' r_k = (s/2)*U(0.75, 1); 'tissue' r_k = (s/2)*(0.55 + 0.45*h(theta_k))
    with h a sum of 3..6 random low-frequency harmonics normalised to [0, 1] (strongly concave).
    Vertices are rounded to integers and cyclic duplicates dropped; a ring left with fewer than 3
    vertices is rejected and drawn again (new angles and radii, same centre, size and vertex count).
    Returns (x int64, y int64, counts int64).
    """
    x, y, counts = _star_draw(rng, cx, cy, s, nv, kind)
    for _ in range(100):
        bad = np.nonzero(counts < 3)[0]
        if bad.size == 0:
            return x, y, counts
        bx, by, bc = _star_draw(rng, np.asarray(cx, dtype=np.float64)[bad], np.asarray(cy, dtype=np.float64)[bad],
                                np.asarray(s, dtype=np.float64)[bad], np.asarray(nv, dtype=np.int64)[bad], kind)
        x, y, counts = _replace_rings(x, y, counts, bad, bx, by, bc)
    raise ValueError("star polygons keep collapsing below 3 vertices (sizes too small for integer rounding)")


def _replace_rings(x, y, counts, idx, nx, ny, ncounts):
    """Rings idx[k] of (x, y, counts) replaced by the k-th ring of (nx, ny, ncounts)."""
    starts = np.concatenate([[0], np.cumsum(counts)])
    nstarts = np.concatenate([[0], np.cumsum(ncounts)])
    new_counts = counts.copy()
    new_counts[idx] = ncounts
    src = {int(i): k for k, i in enumerate(idx)}
    parts_x, parts_y = [], []
    for i in range(counts.shape[0]):
        k = src.get(i)
        if k is None:
            parts_x.append(x[starts[i]:starts[i + 1]])
            parts_y.append(y[starts[i]:starts[i + 1]])
        else:
            parts_x.append(nx[nstarts[k]:nstarts[k + 1]])
            parts_y.append(ny[nstarts[k]:nstarts[k + 1]])
    return np.concatenate(parts_x), np.concatenate(parts_y), new_counts


def _star_draw(rng, cx, cy, s, nv, kind):
    """One draw of star_rings' rings (before rejection of collapsed rings)."""
    cx = np.asarray(cx, dtype=np.float64)
    cy = np.asarray(cy, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    nv = np.asarray(nv, dtype=np.int64)
    owner, k = _segment_ids(nv)
    tot = owner.shape[0]
    theta = 2.0 * np.pi * (k + rng.random(tot)) / nv[owner]
    R = 0.5 * s
    if kind == "nucleus":
        r = R[owner] * rng.uniform(0.75, 1.0, tot)
    elif kind == "tissue":
        n = nv.shape[0]
        m = rng.integers(3, 7, n)                       # harmonics per polygon
        h = np.zeros(tot)
        for j in range(6):
            f = rng.integers(2, 8, n).astype(np.float64)
            a = rng.uniform(0.3, 1.0, n) * (j < m)
            ph = rng.uniform(0.0, 2.0 * np.pi, n)
            h += a[owner] * np.cos(f[owner] * theta + ph[owner])
        hmin = np.full(n, np.inf)
        hmax = np.full(n, -np.inf)
        np.minimum.at(hmin, owner, h)
        np.maximum.at(hmax, owner, h)
        span = np.maximum(hmax - hmin, 1e-12)
        h = (h - hmin[owner]) / span[owner]
        r = R[owner] * (0.55 + 0.45 * h)
    else:
        raise ValueError(kind)
    x = np.rint(cx[owner] + r * np.cos(theta)).astype(np.int64)
    y = np.rint(cy[owner] + r * np.sin(theta)).astype(np.int64)
    return _dedup_rings(x, y, nv)


def staircase_rings(rng, n, max_cols=12, max_h=15, origin_span=200):
    """Simple rectilinear (axis-aligned, integer) polygons, the paper's raster-boundary shape (Fig. 3).

    Each polygon is a run of unit-width columns i = 0..w-1 covering rows [bot_i, top_i), adjacent
    columns overlapping, traced bottom-left -> right along the bottom steps and back along the top.
    Returns (rings, column_heights) where sum(column_heights[j]) is polygon j's exact area.
    """
    rings, heights = [], []
    for _ in range(n):
        w = int(rng.integers(1, max_cols + 1))
        x0 = int(rng.integers(-origin_span, origin_span))
        y0 = int(rng.integers(-origin_span, origin_span))
        bot = np.empty(w, dtype=np.int64)
        top = np.empty(w, dtype=np.int64)
        bot[0] = 0
        top[0] = int(rng.integers(1, max_h + 1))
        for i in range(1, w):
            # keep [bot_i, top_i) overlapping [bot_{i-1}, top_{i-1}) by at least one row
            b = int(rng.integers(bot[i - 1] - max_h // 2, top[i - 1]))
            t = int(rng.integers(max(b + 1, bot[i - 1] + 1), max(b + 1, bot[i - 1] + 1) + max_h))
            bot[i], top[i] = b, t
        pts = []
        # bottom boundary, left to right
        pts.append((0, bot[0]))
        for i in range(w):
            pts.append((i + 1, bot[i]))
            if i + 1 < w and bot[i + 1] != bot[i]:
                pts.append((i + 1, bot[i + 1]))
        # right side up, then top boundary right to left
        pts.append((w, top[w - 1]))
        for i in range(w - 1, -1, -1):
            pts.append((i, top[i]))
            if i - 1 >= 0 and top[i - 1] != top[i]:
                pts.append((i, top[i - 1]))
        ring = np.array(pts, dtype=np.int64)
        # drop collinear duplicates produced by equal consecutive points
        keep = np.ones(len(ring), dtype=bool)
        for j in range(len(ring)):
            if np.array_equal(ring[j], ring[j - 1]):
                keep[j] = False
        ring = ring[keep]
        ring[:, 0] += x0
        ring[:, 1] += y0
        rings.append(ring)
        heights.append(top - bot)
    return rings, heights


# ----------------------------------------------------------------------------------------------
# result-set B from result-set A (Sec. 2.1: two segmentations of the same image)
# ----------------------------------------------------------------------------------------------

def _derive_b(rng, A: PolySet, kinds: np.ndarray, shift_nuc: int, shift_tissue: int, jitter: int,
              drop_frac: float, new_fn):
    """B = A with floor(drop_frac*n) nuclei dropped, each kept polygon shifted by U{-shift..shift}^2
    and each vertex jittered by U{-jitter..jitter}^2, plus floor(drop_frac*n) fresh nuclei from new_fn.
    Tissue polygons (kinds == 1) are never dropped; they are shifted by U{-shift_tissue..shift_tissue}."""
    n = A.n
    nuc = np.nonzero(kinds == 0)[0]
    n_drop = int(math.floor(drop_frac * nuc.shape[0]))
    dropped = rng.permutation(nuc)[:n_drop]
    keep = np.ones(n, dtype=bool)
    keep[dropped] = False
    kept = np.nonzero(keep)[0]
    counts = np.diff(A.off)[kept]
    owner, k = _segment_ids(counts)
    src = A.off[kept][owner] + k
    x = A.xy[2 * src].astype(np.int64)
    y = A.xy[2 * src + 1].astype(np.int64)
    span = np.where(kinds[kept] == 1, shift_tissue, shift_nuc)
    sx = rng.integers(-span, span + 1)
    sy = rng.integers(-span, span + 1)
    x = x + sx[owner] + rng.integers(-jitter, jitter + 1, x.shape[0])
    y = y + sy[owner] + rng.integers(-jitter, jitter + 1, y.shape[0])
    x, y, counts = _dedup_rings(x, y, counts)
    tiles = A.tile[kept]
    bad = counts < 3
    if bad.any():
        # jitter collapsed a ring: fall back to the shifted copy without jitter
        parts_x, parts_y = [], []
        starts = np.cumsum(counts) - counts
        for i in range(counts.shape[0]):
            if not bad[i]:
                parts_x.append(x[starts[i]:starts[i] + counts[i]])
                parts_y.append(y[starts[i]:starts[i] + counts[i]])
            else:
                p = A.polygon(int(kept[i])).astype(np.int64)
                parts_x.append(p[:, 0] + sx[i])
                parts_y.append(p[:, 1] + sy[i])
                counts[i] = p.shape[0]
        x, y = np.concatenate(parts_x), np.concatenate(parts_y)
    nx, ny, ncounts, ntiles = new_fn(rng, n_drop)
    x = np.concatenate([x, nx])
    y = np.concatenate([y, ny])
    counts = np.concatenate([counts, ncounts])
    tiles = np.concatenate([tiles, ntiles]).astype(np.int32)
    return _sort_by_tile(x, y, counts, tiles)


def _sort_by_tile(x, y, counts, tiles) -> PolySet:
    order = np.argsort(tiles, kind="stable")
    if np.all(order == np.arange(order.shape[0])):
        return _pack(x, y, counts, tiles)
    starts = np.cumsum(counts) - counts
    c2 = counts[order]
    owner, k = _segment_ids(c2)
    src = starts[order][owner] + k
    return _pack(x[src], y[src], c2, tiles[order])


# ----------------------------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------------------------

def _nuclei(rng, n, x_lo, x_hi, y_lo, y_hi, s_lo=10.0, s_hi=40.0, nv_lo=8, nv_hi=64):
    cx = rng.uniform(x_lo, x_hi)
    cy = rng.uniform(y_lo, y_hi)
    s = rng.uniform(s_lo, s_hi, n)
    nv = rng.integers(nv_lo, nv_hi + 1, n)
    if np.ndim(cx) == 0:
        cx = rng.uniform(x_lo, x_hi, n)
        cy = rng.uniform(y_lo, y_hi, n)
    return cx, cy, s, nv


def single_tile(seed: int = 1, n: int = 1000, tile_px: int = 2048) -> Workload:
    """One 2048 x 2048 px tile: A = n star polygons (8..64 vertices, MBR 10..40 px, centres uniform);
    B = A jittered +-3 px per vertex, shifted +-5 px, 10% dropped and 10% fresh."""
    rng = _rng(seed)
    cx = rng.uniform(0, tile_px, n)
    cy = rng.uniform(0, tile_px, n)
    s = rng.uniform(10.0, 40.0, n)
    nv = rng.integers(8, 65, n)
    x, y, c = star_rings(rng, cx, cy, s, nv)
    A = _pack(x, y, c, np.zeros(n, dtype=np.int32))

    def new_fn(r, m):
        ncx = r.uniform(0, tile_px, m)
        ncy = r.uniform(0, tile_px, m)
        ns = r.uniform(10.0, 40.0, m)
        nnv = r.integers(8, 65, m)
        a, b, cc = star_rings(r, ncx, ncy, ns, nnv)
        return a, b, cc, np.zeros(m, dtype=np.int32)

    B = _derive_b(rng, A, np.zeros(n, dtype=np.int8), 5, 8, 3, 0.1, new_fn)
    return Workload("single_tile_2048", A, B, 1, tile_px, seed)


def _grid_tiles(rng, image_px, tile_px, density_per_px2):
    """Poisson polygon centres per tile of an image_px^2 image cut into tile_px tiles."""
    nt = (image_px + tile_px - 1) // tile_px
    cxs, cys, tiles = [], [], []
    for ty in range(nt):
        for tx in range(nt):
            x_lo, y_lo = tx * tile_px, ty * tile_px
            x_hi, y_hi = min(image_px, x_lo + tile_px), min(image_px, y_lo + tile_px)
            lam = density_per_px2 * (x_hi - x_lo) * (y_hi - y_lo)
            m = int(rng.poisson(lam))
            cxs.append(rng.uniform(x_lo, x_hi, m))
            cys.append(rng.uniform(y_lo, y_hi, m))
            tiles.append(np.full(m, ty * nt + tx, dtype=np.int32))
    return np.concatenate(cxs), np.concatenate(cys), np.concatenate(tiles), nt * nt


def whole_slide(seed: int = 1, image_px: int = 100_000, tile_px: int = 4096,
                density_per_mpx: float = 100.0) -> Workload:
    """A 100,000^2 px slide cut into 4096^2 tiles (25 x 25; edge tiles narrower); nucleus centres
    Poisson at density_per_mpx per 10^6 px^2 per tile; same star generator and B rule as the single
    tile."""
    rng = _rng(seed)
    dens = density_per_mpx / 1e6
    cx, cy, tiles, n_tiles = _grid_tiles(rng, image_px, tile_px, dens)
    n = cx.shape[0]
    s = rng.uniform(10.0, 40.0, n)
    nv = rng.integers(8, 65, n)
    x, y, c = star_rings(rng, cx, cy, s, nv)
    A = _pack(x, y, c, tiles)
    nt_side = (image_px + tile_px - 1) // tile_px

    def new_fn(r, m):
        ncx = r.uniform(0, image_px, m)
        ncy = r.uniform(0, image_px, m)
        ns = r.uniform(10.0, 40.0, m)
        nnv = r.integers(8, 65, m)
        a, b, cc = star_rings(r, ncx, ncy, ns, nnv)
        t = (np.floor(ncy / tile_px) * nt_side + np.floor(ncx / tile_px)).astype(np.int32)
        return a, b, cc, t

    B = _derive_b(rng, A, np.zeros(n, dtype=np.int8), 5, 8, 3, 0.1, new_fn)
    return Workload(f"whole_slide_{image_px}", A, B, n_tiles, tile_px, seed)


def _loguniform_int(rng, lo, hi, size):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size))).astype(np.int64)


def _concat(parts) -> PolySet:
    """Concatenate PolySets (tiles already in increasing order across parts)."""
    offs, xys, tiles, base = [np.zeros(1, dtype=np.int64)], [], [], 0
    for P in parts:
        offs.append(P.off[1:] + base)
        base += P.n_vertices
        xys.append(P.xy)
        tiles.append(P.tile)
    return PolySet(off=np.concatenate(offs), xy=np.concatenate(xys), tile=np.concatenate(tiles).astype(np.int32))


def _blocks(fn, seed: int, n_tiles: int, block: int, workers: int | None, **kw):
    """Draw tile blocks [t0, t0 + block) independently, block k from SeedSequence([seed, k]), in a
    thread pool (numpy releases the GIL on large array operations). The result does not depend on
    the number of workers."""
    import concurrent.futures as cf
    import os
    jobs = [(k, t0, min(t0 + block, n_tiles)) for k, t0 in enumerate(range(0, n_tiles, block))]
    workers = workers or min(len(jobs), max(1, (os.cpu_count() or 1)))

    def run(job):
        k, t0, t1 = job
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, k])))
        return fn(rng, t0, t1, **kw)
    if workers == 1:
        out = [run(j) for j in jobs]
    else:
        with cf.ThreadPoolExecutor(workers) as ex:
            out = list(ex.map(run, jobs))
    return _concat([a for a, _ in out]), _concat([b for _, b in out])


def _uneven_block(rng, t0, t1, tile_px, count_lo, count_hi, tiles_per_row):
    counts = np.minimum(_loguniform_int(rng, count_lo, count_hi, t1 - t0), count_hi)
    tiles = np.repeat(np.arange(t0, t1, dtype=np.int32), counts)
    n = tiles.shape[0]

    def draw(r, m, t):
        tx = (t % tiles_per_row).astype(np.float64) * tile_px
        ty = (t // tiles_per_row).astype(np.float64) * tile_px
        cx = tx + r.uniform(0, tile_px, m)
        cy = ty + r.uniform(0, tile_px, m)
        s = np.clip(r.lognormal(math.log(20.0), 0.75, m), 8.0, 400.0)
        nv = _loguniform_int(r, 4, 512, m)
        nv = np.maximum(4, np.minimum(nv, np.floor(2 * np.pi * s).astype(np.int64)))
        return cx, cy, s, nv

    cx, cy, s, nv = draw(rng, n, tiles)
    x, y, c = star_rings(rng, cx, cy, s, nv)
    A = _pack(x, y, c, tiles)

    def new_fn(r, m):
        t = r.integers(t0, t1, m).astype(np.int32)
        ncx, ncy, ns, nnv = draw(r, m, t)
        a, b, cc = star_rings(r, ncx, ncy, ns, nnv)
        return a, b, cc, t

    B = _derive_b(rng, A, np.zeros(n, dtype=np.int8), 5, 8, 3, 0.1, new_fn)
    return A, B


def batched_uneven(seed: int = 1, n_tiles: int = 2000, tile_px: int = 4096,
                   count_lo: int = 50, count_hi: int = 20_000, tiles_per_row: int = 50,
                   workers: int | None = None) -> Workload:
    """n_tiles tiles of uneven load: polygons per tile log-uniform [50, 20000]; MBR size
    s = clip(lognormal(ln 20, 0.75), 8, 400); vertices log-uniform {4..512}, capped at 2*pi*s.
    Drawn in independent blocks of 50 tiles (B derived from A within each block)."""
    A, B = _blocks(_uneven_block, seed, n_tiles, 50, workers, tile_px=tile_px, count_lo=count_lo,
                   count_hi=count_hi, tiles_per_row=tiles_per_row)
    return Workload(f"batched_uneven_{n_tiles}", A, B, n_tiles, tile_px, seed)


def _heavy_block(rng, t0, t1, tile_px, nuclei_per_tile, tissue_lo, tissue_hi, tiles_per_row,
                 tissue_nv_lo, tissue_nv_hi, tissue_s_lo, tissue_s_hi):
    nt_ = t1 - t0
    n_tissue = rng.integers(tissue_lo, tissue_hi + 1, nt_)
    per_tile = nuclei_per_tile + n_tissue
    tiles = np.repeat(np.arange(t0, t1, dtype=np.int32), per_tile)
    n = tiles.shape[0]
    kinds = np.zeros(n, dtype=np.int8)
    starts = np.cumsum(per_tile) - per_tile
    for j in range(nt_):
        kinds[starts[j] + nuclei_per_tile: starts[j] + per_tile[j]] = 1
    tx = (tiles % tiles_per_row).astype(np.float64) * tile_px
    ty = (tiles // tiles_per_row).astype(np.float64) * tile_px
    cx = tx + rng.uniform(0, tile_px, n)
    cy = ty + rng.uniform(0, tile_px, n)
    s = rng.uniform(10.0, 40.0, n)
    nv = rng.integers(8, 65, n)
    tis = kinds == 1
    ntis = int(tis.sum())
    s[tis] = np.exp(rng.uniform(math.log(tissue_s_lo), math.log(tissue_s_hi), ntis))
    nv[tis] = rng.integers(tissue_nv_lo, tissue_nv_hi + 1, ntis)
    xn, yn, cn = star_rings(rng, cx[~tis], cy[~tis], s[~tis], nv[~tis], "nucleus")
    xt, yt, ct = star_rings(rng, cx[tis], cy[tis], s[tis], nv[tis], "tissue")
    counts = np.zeros(n, dtype=np.int64)
    counts[~tis] = cn
    counts[tis] = ct
    x = np.empty(int(counts.sum()), dtype=np.int64)
    y = np.empty_like(x)
    owner, _ = _segment_ids(counts)
    is_t = tis[owner]
    x[~is_t], y[~is_t] = xn, yn
    x[is_t], y[is_t] = xt, yt
    A = _pack(x, y, counts, tiles)

    def new_fn(r, m):
        t = r.integers(t0, t1, m).astype(np.int32)
        ntx = (t % tiles_per_row).astype(np.float64) * tile_px
        nty = (t // tiles_per_row).astype(np.float64) * tile_px
        ncx = ntx + r.uniform(0, tile_px, m)
        ncy = nty + r.uniform(0, tile_px, m)
        ns = r.uniform(10.0, 40.0, m)
        nnv = r.integers(8, 65, m)
        a, b, cc = star_rings(r, ncx, ncy, ns, nnv)
        return a, b, cc, t

    B = _derive_b(rng, A, kinds, 5, 8, 3, 0.1, new_fn)
    return A, B


def heavy_tail(seed: int = 1, n_tiles: int = 200, tile_px: int = 4096, nuclei_per_tile: int = 20_000,
               tissue_lo: int = 5, tissue_hi: int = 20, tiles_per_row: int = 20,
               tissue_nv_lo: int = 2000, tissue_nv_hi: int = 20_000,
               tissue_s_lo: float = 500.0, tissue_s_hi: float = 4000.0, workers: int | None = None) -> Workload:
    """n_tiles tiles each holding nuclei_per_tile nuclei (MBR 10..40 px, 8..64 vertices) plus
    U{5..20} concave tissue-region polygons (2,000..20,000 vertices, MBR log-uniform 500..4,000 px).
    B: nuclei by the single-tile rule; tissue polygons shifted +-8 px and jittered +-3 px.
    Drawn in independent blocks of 10 tiles."""
    A, B = _blocks(_heavy_block, seed, n_tiles, 10, workers, tile_px=tile_px, nuclei_per_tile=nuclei_per_tile,
                   tissue_lo=tissue_lo, tissue_hi=tissue_hi, tiles_per_row=tiles_per_row,
                   tissue_nv_lo=tissue_nv_lo, tissue_nv_hi=tissue_nv_hi, tissue_s_lo=tissue_s_lo,
                   tissue_s_hi=tissue_s_hi)
    return Workload(f"heavy_tail_{n_tiles}", A, B, n_tiles, tile_px, seed)


def subset_tiles(w: Workload, tiles) -> Workload:
    """Restrict a workload to the given tile ids (renumbered 0..k-1 in the given order)."""
    tiles = list(tiles)

    def sub(P: PolySet) -> PolySet:
        rings_idx = [np.nonzero(P.tile == t)[0] for t in tiles]
        idx = np.concatenate(rings_idx) if rings_idx else np.zeros(0, dtype=np.int64)
        counts = np.diff(P.off)[idx]
        owner, k = _segment_ids(counts)
        src = P.off[idx][owner] + k
        x = P.xy[2 * src].astype(np.int64)
        y = P.xy[2 * src + 1].astype(np.int64)
        newt = np.concatenate([np.full(len(r), j, dtype=np.int32) for j, r in enumerate(rings_idx)])
        return _pack(x, y, counts, newt)

    return Workload(w.name + f"_sub{len(tiles)}", sub(w.A), sub(w.B), len(tiles), w.tile_px, w.seed)


def scaled(w: Workload, factor: int) -> Workload:
    """Every vertex coordinate multiplied by an integer factor (the scale-factor experiment of
    Sec. 5.2, Fig. 8: polygons factor^2 times larger, same vertices, same MBR overlaps)."""
    def sc(P: PolySet) -> PolySet:
        xy = P.xy.astype(np.int64) * int(factor)
        if xy.size and np.abs(xy).max() > (1 << 28):
            raise ValueError("scaled coordinates exceed the +-2^28 limit")
        return PolySet(off=P.off.copy(), xy=xy.astype(np.int32), tile=P.tile.copy())

    return Workload(f"{w.name}_x{factor}", sc(w.A), sc(w.B), w.n_tiles, w.tile_px * int(factor), w.seed)


CONFIGS = {
    1: single_tile,
    2: whole_slide,
    3: batched_uneven,
    4: heavy_tail,
}


def make_config(k: int, seed: int = 1, **kw) -> Workload:
    return CONFIGS[k](seed=seed, **kw)
