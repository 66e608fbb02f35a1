"""CPU oracle for pair areas, candidate pairs and the Jaccard reduction (test infrastructure).

Only the tests, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product path (the CUDA library and its Python binding) never imports,
links or runs it, and this package imports nothing from the product package.

The brute-force C code in ``sccg_oracle.c`` defines the pixel areas (Sec. 3.1: pixelization and
ray casting, with the exact tie rule written out in that file's header). This module wraps it with
ctypes and adds the Jaccard reductions of Sec. 2.1 in plain Python:

  J  = sum(inter) / sum(union)          over pairs with inter > 0
  J' = (1/n) * sum(inter_i / union_i)   over the n pairs with inter > 0        (Eq. 1)

Each ratio is the IEEE double quotient of the two integer counts; the n ratios are summed exactly
and rounded once (``math.fsum``), then divided by n. That fixes a single, order-independent double
for J' (the paper leaves the summation order open).

Parity pins: every function here is checked by ``tests/test_oracle_pins.py`` against closed forms,
hand-derived counts and an independent method; no function is left unpinned.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sccg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liboracle.so (portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_pixel_in_polygon.argtypes = [P, I64, I64, I64]
            lib.oracle_pixel_in_polygon.restype = ctypes.c_int
            lib.oracle_polygon_area.argtypes = [P, I64]
            lib.oracle_polygon_area.restype = I64
            lib.oracle_rle_area.argtypes = [P, I64]
            lib.oracle_rle_area.restype = I64
            lib.oracle_pair.argtypes = [P, I64, P, I64, P, P]
            lib.oracle_pair.restype = None
            lib.oracle_rle_pair.argtypes = [P, I64, P, I64, P, P]
            lib.oracle_rle_pair.restype = None
            lib.oracle_pair_areas.argtypes = [P, P, P, P, P, P, I64, P, P, ctypes.c_int, ctypes.c_int]
            lib.oracle_pair_areas.restype = None
            lib.oracle_polygon_areas.argtypes = [P, P, I64, P, P, ctypes.c_int, ctypes.c_int]
            lib.oracle_polygon_areas.restype = None
            lib.oracle_candidate_pairs.argtypes = [P, P, I64, P, P, I64, P, P, I64]
            lib.oracle_candidate_pairs.restype = I64
            lib.oracle_polygon_mask.argtypes = [P, I64, P]
            lib.oracle_polygon_mask.restype = None
            lib.oracle_rle_mask.argtypes = [P, I64, P]
            lib.oracle_rle_mask.restype = None
            lib.oracle_touches.argtypes = [P, I64, P, I64]
            lib.oracle_touches.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ring(r) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(r, dtype=np.int32).reshape(-1))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------- single polygons

def pixel_in_polygon(ring, x: int, y: int) -> int:
    r = _ring(ring)
    return int(_load().oracle_pixel_in_polygon(_ptr(r), r.size // 2, int(x), int(y)))


def polygon_area(ring) -> int:
    """||p|| by brute force over MBR(p)'s pixel window."""
    r = _ring(ring)
    return int(_load().oracle_polygon_area(_ptr(r), r.size // 2))


def polygon_area_rle(ring) -> int:
    """||p|| by the independent row-interval method."""
    r = _ring(ring)
    return int(_load().oracle_rle_area(_ptr(r), r.size // 2))


def polygon_mask(ring, method: str = "brute") -> np.ndarray:
    """Membership of every pixel of MBR(p)'s window: bool [H, W], row y - min y, column x - min x
    (brute force per pixel, or "rle": the row intervals, for windows too large for the brute force)."""
    r = _ring(ring)
    xy = r.reshape(-1, 2)
    W = int(xy[:, 0].max()) - int(xy[:, 0].min())
    H = int(xy[:, 1].max()) - int(xy[:, 1].min())
    out = np.zeros(max(W, 0) * max(H, 0), dtype=np.uint8)
    if out.size:
        fn = _load().oracle_polygon_mask if method == "brute" else _load().oracle_rle_mask
        fn(_ptr(r), r.size // 2, _ptr(out))
    return out.reshape(max(H, 0), max(W, 0)).astype(bool)


def pair(ring_p, ring_q):
    """(||p n q||, ||p u q||) counted directly over the bounding box of both MBRs."""
    a, b = _ring(ring_p), _ring(ring_q)
    i = np.zeros(1, dtype=np.int64)
    u = np.zeros(1, dtype=np.int64)
    _load().oracle_pair(_ptr(a), a.size // 2, _ptr(b), b.size // 2, _ptr(i), _ptr(u))
    return int(i[0]), int(u[0])


def pair_rle(ring_p, ring_q):
    a, b = _ring(ring_p), _ring(ring_q)
    i = np.zeros(1, dtype=np.int64)
    u = np.zeros(1, dtype=np.int64)
    _load().oracle_rle_pair(_ptr(a), a.size // 2, _ptr(b), b.size // 2, _ptr(i), _ptr(u))
    return int(i[0]), int(u[0])


def shoelace_area2(ring) -> int:
    """Twice the signed shoelace area (Sec. 3.2, the POLYAREA formula), exact in integers."""
    r = np.asarray(ring, dtype=np.int64).reshape(-1, 2)
    x, y = r[:, 0], r[:, 1]
    return int(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


# ---------------------------------------------------------------------------- whole sets

def polygon_areas(off, xy, method: str = "brute", nthreads: int | None = None):
    """Per-polygon (area int64[n], mbr int32[n,4]) for a CSR polygon set."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = off.shape[0] - 1
    area = np.zeros(n, dtype=np.int64)
    mbr = np.zeros((n, 4), dtype=np.int32)
    _load().oracle_polygon_areas(_ptr(off), _ptr(xy), n, _ptr(area), _ptr(mbr),
                                 0 if method == "brute" else 1, nthreads or default_threads())
    return area, mbr


def pair_areas(A, B, pa, pb, method: str = "brute", nthreads: int | None = None):
    """Per-pair (inter int64[n], union int64[n]) for pairs (A polygon pa[i], B polygon pb[i])."""
    pa = np.ascontiguousarray(pa, dtype=np.int64)
    pb = np.ascontiguousarray(pb, dtype=np.int64)
    n = pa.shape[0]
    inter = np.zeros(n, dtype=np.int64)
    uni = np.zeros(n, dtype=np.int64)
    offa = np.ascontiguousarray(A.off, dtype=np.int64)
    xya = np.ascontiguousarray(A.xy, dtype=np.int32)
    offb = np.ascontiguousarray(B.off, dtype=np.int64)
    xyb = np.ascontiguousarray(B.xy, dtype=np.int32)
    _load().oracle_pair_areas(_ptr(offa), _ptr(xya), _ptr(offb), _ptr(xyb), _ptr(pa), _ptr(pb), n,
                              _ptr(inter), _ptr(uni), 0 if method == "brute" else 1,
                              nthreads or default_threads())
    return inter, uni


def candidate_pairs(mbr_a, tile_a, mbr_b, tile_b):
    """All same-tile (a, b) with overlapping closed MBRs, ascending (a, b). Returns (pa, pb) int64."""
    ma = np.ascontiguousarray(mbr_a, dtype=np.int32).reshape(-1, 4)
    mb = np.ascontiguousarray(mbr_b, dtype=np.int32).reshape(-1, 4)
    ta = np.ascontiguousarray(tile_a, dtype=np.int32)
    tb = np.ascontiguousarray(tile_b, dtype=np.int32)
    lib = _load()
    z = np.zeros(1, dtype=np.int64)
    cnt = lib.oracle_candidate_pairs(_ptr(ma), _ptr(ta), ma.shape[0], _ptr(mb), _ptr(tb), mb.shape[0],
                                     _ptr(z), _ptr(z), 0)
    if cnt < 0:
        raise ValueError("tile ids must be non-decreasing in both sets")
    pa = np.zeros(cnt, dtype=np.int64)
    pb = np.zeros(cnt, dtype=np.int64)
    lib.oracle_candidate_pairs(_ptr(ma), _ptr(ta), ma.shape[0], _ptr(mb), _ptr(tb), mb.shape[0],
                               _ptr(pa), _ptr(pb), cnt)
    return pa, pb


def jaccard(inter, uni):
    """Sec. 2.1 reductions over the pairs with inter > 0.

    Returns dict(sum_inter, sum_union, n_nonzero, J, Jprime): J = float(sum_inter)/float(sum_union);
    J' = fsum(float(inter_i)/float(union_i)) / n_nonzero. Both are 0.0 when no pair intersects."""
    inter = np.asarray(inter, dtype=np.int64)
    uni = np.asarray(uni, dtype=np.int64)
    nz = inter > 0
    si = int(inter[nz].sum())
    su = int(uni[nz].sum())
    n = int(nz.sum())
    if n == 0:
        return dict(sum_inter=0, sum_union=0, n_nonzero=0, J=0.0, Jprime=0.0)
    ratios = [float(a) / float(b) for a, b in zip(inter[nz].tolist(), uni[nz].tolist())]
    return dict(sum_inter=si, sum_union=su, n_nonzero=n, J=float(si) / float(su),
                Jprime=math.fsum(ratios) / n)


def cross_compare(A, B, method: str = "brute", nthreads: int | None = None):
    """The whole path on the CPU: areas, MBRs, candidate pairs, pair areas, Jaccard."""
    area_a, mbr_a = polygon_areas(A.off, A.xy, method, nthreads)
    area_b, mbr_b = polygon_areas(B.off, B.xy, method, nthreads)
    pa, pb = candidate_pairs(mbr_a, A.tile, mbr_b, B.tile)
    inter, uni = pair_areas(A, B, pa, pb, method, nthreads)
    return dict(area_a=area_a, area_b=area_b, mbr_a=mbr_a, mbr_b=mbr_b, pa=pa, pb=pb,
                inter=inter, uni=uni, jaccard=jaccard(inter, uni))


# ---------------------------------------------------------------------------- other operators

def touches(ring_p, ring_q) -> bool:
    """ST_Touches by the rule given with the other operators of Sec. 3.4: no edge crossing, no vertex
    of one strictly within the other, some vertex of one on an edge of the other."""
    a, b = _ring(ring_p), _ring(ring_q)
    return bool(_load().oracle_touches(_ptr(a), a.size // 2, _ptr(b), b.size // 2))


def touches_pairs(A, B, pa, pb):
    """touches() for every pair (A polygon pa[k], B polygon pb[k]) -> uint8 [n]."""
    out = np.zeros(len(pa), dtype=np.uint8)
    for k, (i, j) in enumerate(zip(np.asarray(pa), np.asarray(pb))):
        ra = A.xy[2 * A.off[i]: 2 * A.off[i + 1]]
        rb = B.xy[2 * B.off[j]: 2 * B.off[j + 1]]
        out[k] = touches(ra, rb)
    return out


def contains_flags(area_a, area_b, pa, pb, inter):
    """ST_Contains as Sec. 3.4 states it, on pixel areas: bit 0 = the A polygon contains the B polygon
    (||p n q|| = ||q|| > 0), bit 1 = the B polygon contains the A polygon (||p n q|| = ||p|| > 0)."""
    pa, pb, inter = (np.asarray(x, dtype=np.int64) for x in (pa, pb, inter))
    aa, ab = np.asarray(area_a)[pa], np.asarray(area_b)[pb]
    return (((inter == ab) & (ab > 0)).astype(np.uint8) | (((inter == aa) & (aa > 0)).astype(np.uint8) << 1))
