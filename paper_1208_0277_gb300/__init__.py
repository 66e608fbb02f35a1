"""GB300-native exact pixel-area cross-comparison of two polygon result sets.

Implements the aggregator path of Wang et al., "Accelerating Pathology Image Data Cross-Comparison
on CPU-GPU Hybrid Systems" (PVLDB 5(11), 2012): candidate pairs by MBR overlap within tiles
(Sec. 4.1, the && filter of Fig. 1b), exact intersection and union pixel areas by PixelBox
sampling-box subdivision with per-pixel ray casting (Sec. 3, Algorithm 1), and the Jaccard
similarities J and J' (Sec. 2.1, Eq. 1).

All computation runs in the CUDA library ``libsccg.so`` (hand-written sm_103a kernels behind the C
ABI in ``include/sccg.h``). This module only marshals arguments: torch supplies device memory and
streams. There is no CPU fallback; calls raise if the library or a GPU is missing.
"""
from __future__ import annotations

import ctypes
import dataclasses

from . import _native
from ._native import build  # noqa: F401

SCCG_OK = 0
SCCG_ECAPACITY = 3
MODE_PLAIN = 0
MODE_PERSISTENT = 1
MODE_NOSEP = 2         # PixelBox-NoSep (Sec. 5.2): union counted directly, for comparison
AREA_ROWS = 0          # sccg_prepare counts ||p|| row by row (default)
AREA_PIXELBOX = 1      # ... or by PixelBox on the polygon alone
AREA_SHOELACE = 2      # ... or, for sets flagged rectilinear and simple, by the shoelace formula


class SccgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        lib = _native.load()
        msg = lib.sccg_status_str(status).decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _hptr(a) -> int | None:
    return None if a is None else a.ctypes.data


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclasses.dataclass
class DevicePolySet:
    """A prepared polygon set resident in device memory (torch tensors) plus its C descriptor."""
    off: object
    xy: object
    tile: object
    mbr: object
    area: object
    c: _native.PolySetC
    bands: object = None        # uint8 device tensor holding the band index, if the set has one
    raster: object = None       # uint8 device tensor holding the pixel rasters, if the set has them

    @property
    def n(self) -> int:
        return int(self.c.n)


class Context:
    """An sccg context on one CUDA device (scratch memory, tunables)."""

    def __init__(self, device: int = 0, params: dict | None = None):
        import json
        self.lib = _native.load()
        self.device = device
        h = ctypes.c_void_p()
        js = json.dumps(params).encode() if params else None
        st = self.lib.sccg_ctx_create(device, js, ctypes.byref(h))
        if st != SCCG_OK:
            raise SccgError(st, "sccg_ctx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.sccg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, where: str):
        if st != SCCG_OK:
            raise SccgError(st, where, self.lib.sccg_last_error(self.h).decode())

    def set_param(self, name: str, value: int):
        self._check(self.lib.sccg_ctx_set_param(self.h, name.encode(), int(value)), "sccg_ctx_set_param")

    def reserve(self, max_pairs: int):
        """Size the context's scratch for up to max_pairs pairs now (no allocation, and no device
        synchronisation, in later pair-area and Jaccard calls up to that size)."""
        self._check(self.lib.sccg_ctx_reserve(self.h, int(max_pairs)), "sccg_ctx_reserve")

    def params(self) -> dict:
        p = _native.ParamsC()
        self._check(self.lib.sccg_ctx_get_params(self.h, ctypes.byref(p)), "sccg_ctx_get_params")
        return {k: getattr(p, k) for k, _ in p._fields_}

    # ------------------------------------------------------------------ sets
    def upload(self, ps, stream=None, bands: bool = True, raster: bool = True) -> DevicePolySet:
        """Copy a host PolySet (workload.PolySet) to the device and prepare it (MBRs, areas, and by
        default the pixel rasters)."""
        import torch
        dev = torch.device("cuda", self.device)
        off = torch.from_numpy(ps.off).to(dev)
        xy = torch.from_numpy(ps.xy).to(dev)
        tile = torch.from_numpy(ps.tile).to(dev)
        return self.prepare(off, xy, tile, stream, bands=bands, raster=raster)

    def _polyset(self, off, xy, tile, out):
        import torch
        n = off.numel() - 1
        if out is None:
            mbr = torch.empty((max(n, 1), 4), dtype=torch.int32, device=off.device)
            area = torch.empty(max(n, 1), dtype=torch.int64, device=off.device)
            rbuf = None
        else:
            mbr, area = out[0], out[1]
            rbuf = out[2] if len(out) > 2 else None
        if xy.numel() == 0:
            xy = torch.zeros(2, dtype=torch.int32, device=off.device)
        c = _native.PolySetC(n=n, off=off.data_ptr(), xy=xy.data_ptr(), tile=_ptr(tile),
                             mbr=mbr.data_ptr(), area=area.data_ptr())
        return c, xy, mbr, area, rbuf

    def raster_bytes(self, c: _native.PolySetC, stream=None) -> int:
        """Device bytes the pixel rasters of the set described by c take (sccg_raster_bytes)."""
        nb = ctypes.c_int64()
        self._check(self.lib.sccg_raster_bytes(self.h, ctypes.byref(c), ctypes.byref(nb), _stream(stream)),
                    "sccg_raster_bytes")
        return int(nb.value)

    def _raster_buffer(self, c, rbuf, device, stream):
        """rbuf if it holds the set's rasters, else a new buffer of the exact size."""
        import torch
        if rbuf is None or rbuf.numel() < int(c.raster_bytes or 0):
            nb = self.raster_bytes(c, stream) if rbuf is None else int(c.raster_bytes)
            rbuf = torch.empty(max(nb, 16), dtype=torch.uint8, device=device)
        c.raster = rbuf.data_ptr()
        c.raster_cap = rbuf.numel()
        return rbuf

    def prepare(self, off, xy, tile=None, stream=None, out=None, bands: bool = True,
                raster: bool = True) -> DevicePolySet:
        """MBRs, validation and pixel areas of a device-resident CSR set (off int64, xy int32 pairs,
        tile int32 or None). out = (mbr int32 [n,4], area int64 [n][, raster uint8]) reuses caller
        buffers. With raster (default) the set's pixel rasters are written too (into out's raster
        buffer when it is large enough, else into a new one of the exact size), and the pair-area
        calls on two such sets AND rasters instead of pixelizing pair windows. With bands (default)
        the band index of polygons with >= 1024 vertices is built when there are any."""
        c, xy, mbr, area, rbuf = self._polyset(off, xy, tile, out)
        if raster and c.n > 0:
            rbuf = self._raster_buffer(c, rbuf, off.device, stream)
        self._check(self.lib.sccg_prepare(self.h, ctypes.byref(c), _stream(stream)), "sccg_prepare")
        if raster and c.n > 0 and not c.raster_ok:
            # the buffer given was too small for these rasters: once more into one of the exact size
            rbuf = self._raster_buffer(c, None if rbuf is None else rbuf[:0], off.device, stream)
            self._check(self.lib.sccg_prepare(self.h, ctypes.byref(c), _stream(stream)), "sccg_prepare")
        d = DevicePolySet(off, xy, tile, mbr, area, c, raster=rbuf if c.raster_ok else None)
        if bands and c.band_bytes > 0:
            self.build_bands(d, stream=stream)
        return d

    def prepare_sets(self, specs, stream=None, bands: bool = True, raster: bool = True) -> list:
        """prepare() for several sets with one synchronisation: specs = [(off, xy, tile, out), ...]
        (tile and out may be None; out as in prepare())."""
        k = len(specs)
        arr = (_native.PolySetC * k)()
        keep = []
        for j, (off, xy, tile, out) in enumerate(specs):
            c, xy2, mbr, area, rbuf = self._polyset(off, xy, tile, out)
            if raster and c.n > 0:
                rbuf = self._raster_buffer(c, rbuf, off.device, stream)
            arr[j] = c
            keep.append((off, xy2, tile, mbr, area, rbuf))
        self._check(self.lib.sccg_prepare_sets(self.h, arr, k, _stream(stream)), "sccg_prepare_sets")
        if raster and any(arr[j].n > 0 and not arr[j].raster_ok for j in range(k)):
            for j in range(k):
                if arr[j].n > 0 and not arr[j].raster_ok:
                    off, xy2, tile, mbr, area, rbuf = keep[j]
                    rbuf = self._raster_buffer(arr[j], None if rbuf is None else rbuf[:0], off.device, stream)
                    keep[j] = (off, xy2, tile, mbr, area, rbuf)
            self._check(self.lib.sccg_prepare_sets(self.h, arr, k, _stream(stream)), "sccg_prepare_sets")
        out = []
        for j, (off, xy2, tile, mbr, area, rbuf) in enumerate(keep):
            c = _native.PolySetC()
            ctypes.pointer(c)[0] = arr[j]
            d = DevicePolySet(off, xy2, tile, mbr, area, c, raster=rbuf if c.raster_ok else None)
            if bands and c.band_bytes > 0:
                self.build_bands(d, stream=stream)
            out.append(d)
        return out

    def build_bands(self, d: DevicePolySet, stream=None):
        """Build (or rebuild) the band index of a prepared set into a new device buffer."""
        import torch
        buf = torch.empty(max(int(d.c.band_bytes), 16), dtype=torch.uint8, device=d.off.device)
        self._check(self.lib.sccg_build_bands(self.h, ctypes.byref(d.c), ctypes.c_void_p(buf.data_ptr()),
                                              buf.numel(), _stream(stream)), "sccg_build_bands")
        d.bands = buf if d.c.bands else None

    # ------------------------------------------------------------------ hot path
    def candidate_pairs(self, A: DevicePolySet, B: DevicePolySet, capacity: int | None = None,
                        stream=None, with_tile_offsets: bool = False, out=None):
        """(pa, pb) int32 device tensors of all same-tile MBR-overlapping pairs; with
        with_tile_offsets also the host int64 array of per-tile pair offsets [n_tiles + 1]."""
        import numpy as np
        import torch
        dev = A.off.device
        n = ctypes.c_int64(0)
        n_tiles = max(A.c.n_tiles, B.c.n_tiles, 1)
        tpo = np.zeros(n_tiles + 1, dtype=np.int64) if with_tile_offsets else None
        if capacity is None:
            st = self.lib.sccg_candidate_pairs(self.h, ctypes.byref(A.c), ctypes.byref(B.c), None, None, 0,
                                               ctypes.byref(n), _hptr(tpo), _stream(stream))
            if st not in (SCCG_OK, SCCG_ECAPACITY):
                self._check(st, "sccg_candidate_pairs")
            capacity = int(n.value)
        if out is None:
            pa = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
            pb = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
        else:
            pa, pb = out
            capacity = min(capacity, pa.numel(), pb.numel())
        self._check(self.lib.sccg_candidate_pairs(self.h, ctypes.byref(A.c), ctypes.byref(B.c), pa.data_ptr(),
                                                  pb.data_ptr(), capacity, ctypes.byref(n), _hptr(tpo),
                                                  _stream(stream)), "sccg_candidate_pairs")
        k = int(n.value)
        if with_tile_offsets:
            return pa[:k], pb[:k], tpo
        return pa[:k], pb[:k]

    def pair_areas(self, A: DevicePolySet, B: DevicePolySet, pa, pb, mode: int = MODE_PLAIN,
                   out=None, stream=None):
        """(inter, uni) int64 device tensors: ||p n q|| and ||p|| + ||q|| - ||p n q|| per pair."""
        import torch
        n = pa.numel()
        if out is None:
            inter = torch.empty(max(n, 1), dtype=torch.int64, device=pa.device)
            uni = torch.empty(max(n, 1), dtype=torch.int64, device=pa.device)
        else:
            inter, uni = out
        self._check(self.lib.sccg_pair_areas(self.h, ctypes.byref(A.c), ctypes.byref(B.c), pa.data_ptr(),
                                             pb.data_ptr(), n, inter.data_ptr(), uni.data_ptr(), int(mode),
                                             _stream(stream)), "sccg_pair_areas")
        return inter[:n], uni[:n]

    def pair_areas_tiles(self, A: DevicePolySet, B: DevicePolySet, pa, pb, tile_pair_off, out=None, stream=None):
        """One kernel launch per tile (tile_pair_off: host int64 [n_tiles + 1])."""
        import numpy as np
        import torch
        n = pa.numel()
        tpo = np.ascontiguousarray(tile_pair_off, dtype=np.int64)
        if out is None:
            inter = torch.empty(max(n, 1), dtype=torch.int64, device=pa.device)
            uni = torch.empty(max(n, 1), dtype=torch.int64, device=pa.device)
        else:
            inter, uni = out
        self._check(self.lib.sccg_pair_areas_tiles(self.h, ctypes.byref(A.c), ctypes.byref(B.c), pa.data_ptr(),
                                                   pb.data_ptr(), tpo.ctypes.data, len(tpo) - 1, inter.data_ptr(),
                                                   uni.data_ptr(), _stream(stream)), "sccg_pair_areas_tiles")
        return inter[:n], uni[:n]

    def batch_run(self, A: DevicePolySet, B: DevicePolySet, pa, pb, out, result, stream=None):
        """Persistent pair areas + Jaccard replayed as one CUDA graph. out = (inter, uni) int64 device
        tensors; result = device uint8 tensor of 48 bytes receiving the Jaccard struct."""
        inter, uni = out
        n = pa.numel()
        self._check(self.lib.sccg_batch_run(self.h, ctypes.byref(A.c), ctypes.byref(B.c), pa.data_ptr(),
                                            pb.data_ptr(), n, inter.data_ptr(), uni.data_ptr(), result.data_ptr(),
                                            _stream(stream)), "sccg_batch_run")
        return inter[:n], uni[:n]

    @staticmethod
    def read_jaccard(result) -> dict:
        """Decode the 48-byte device Jaccard struct (copies it to the host)."""
        r = _native.JaccardC.from_buffer_copy(result.cpu().numpy().tobytes())
        return {k: getattr(r, k) for k, _ in r._fields_}

    def gather_pairs(self, src_pa, src_pb, seg_src, seg_dst, dst_pa, dst_pb, stream=None):
        """Copy pair slices (segment s: seg_src[s], length seg_dst[s+1]-seg_dst[s]) into dst."""
        self._check(self.lib.sccg_gather_pairs(self.h, src_pa.data_ptr(), src_pb.data_ptr(), seg_src.data_ptr(),
                                               seg_dst.data_ptr(), seg_src.numel(), dst_pa.data_ptr(),
                                               dst_pb.data_ptr(), _stream(stream)), "sccg_gather_pairs")

    def jaccard_segments(self, inter, uni, seg_off, out, stream=None):
        """Per-segment Jaccard into `out` (device uint8 tensor of 48 * n_segments bytes)."""
        self._check(self.lib.sccg_jaccard_segments(self.h, inter.data_ptr(), uni.data_ptr(), seg_off.data_ptr(),
                                                   seg_off.numel() - 1, out.data_ptr(), _stream(stream)),
                    "sccg_jaccard_segments")

    @staticmethod
    def decode_jaccard_array(raw) -> list:
        """Decode a host bytes/uint8 array of 48-byte Jaccard structs."""
        import numpy as np
        names = [k for k, _ in _native.JaccardC._fields_]
        dt = np.dtype([(k, "<i8") for k in names[:4]] + [(k, "<f8") for k in names[4:]])
        buf = np.ascontiguousarray(np.asarray(raw, dtype=np.uint8))
        return [dict(zip(names, r)) for r in np.frombuffer(buf.tobytes(), dtype=dt).tolist()]

    def launch_count(self) -> int:
        c = ctypes.c_uint64(0)
        self._check(self.lib.sccg_launch_count(self.h, ctypes.byref(c)), "sccg_launch_count")
        return int(c.value)

    def pair_areas_raw(self, A, B, pa_ptr: int, pb_ptr: int, n: int, inter_ptr: int, uni_ptr: int,
                       mode: int = MODE_PLAIN, stream=None):
        """Pointer-level variant of pair_areas (used for per-tile slices)."""
        self._check(self.lib.sccg_pair_areas(self.h, ctypes.byref(A.c), ctypes.byref(B.c), pa_ptr, pb_ptr, n,
                                             inter_ptr, uni_ptr, int(mode), _stream(stream)), "sccg_pair_areas")

    def jaccard(self, inter, uni, stream=None) -> dict:
        r = _native.JaccardC()
        n = inter.numel()
        self._check(self.lib.sccg_jaccard(self.h, _ptr(inter) if n else None, _ptr(uni) if n else None, n,
                                          ctypes.byref(r), _stream(stream)), "sccg_jaccard")
        return {k: getattr(r, k) for k, _ in r._fields_}

    def jaccard_device(self, inter, uni, out, stream=None):
        """Asynchronous Jaccard into a device buffer `out` (uint8 tensor of 48 bytes)."""
        n = inter.numel()
        self._check(self.lib.sccg_jaccard(self.h, _ptr(inter) if n else None, _ptr(uni) if n else None, n,
                                          ctypes.c_void_p(out.data_ptr()), _stream(stream)), "sccg_jaccard")

    def contains(self, A: DevicePolySet, B: DevicePolySet, pa, pb, inter, stream=None):
        """ST_Contains flags (uint8 device tensor): bit 0 A contains B, bit 1 B contains A."""
        import torch
        n = pa.numel()
        out = torch.empty(max(n, 1), dtype=torch.uint8, device=pa.device)
        self._check(self.lib.sccg_contains(self.h, ctypes.byref(A.c), ctypes.byref(B.c), _ptr(pa), _ptr(pb),
                                           _ptr(inter), n, _ptr(out), _stream(stream)), "sccg_contains")
        return out[:n]

    def touches(self, A: DevicePolySet, B: DevicePolySet, pa, pb, stream=None):
        """ST_Touches (uint8 device tensor, 1 = touch) by the rule of Sec. 5."""
        import torch
        n = pa.numel()
        out = torch.empty(max(n, 1), dtype=torch.uint8, device=pa.device)
        self._check(self.lib.sccg_touches(self.h, ctypes.byref(A.c), ctypes.byref(B.c), _ptr(pa), _ptr(pb), n,
                                          _ptr(out), _stream(stream)), "sccg_touches")
        return out[:n]

    def rebase_pairs(self, pa, pb, base_a: int, base_b: int, stream=None):
        """In place on the device: pa += base_a, pb += base_b."""
        n = pa.numel()
        self._check(self.lib.sccg_rebase_pairs(self.h, _ptr(pa) if n else None, _ptr(pb) if n else None, n,
                                               int(base_a), int(base_b), _stream(stream)), "sccg_rebase_pairs")

    def copy(self, dst, src, stream=None):
        """dst.copy_(src) by the SMs (sccg_copy): contiguous tensors of equal byte size, each on this
        context's device or in page-locked host memory."""
        nb = src.numel() * src.element_size()
        if dst.numel() * dst.element_size() != nb or not (dst.is_contiguous() and src.is_contiguous()):
            raise ValueError("copy: contiguous tensors of equal byte size")
        if nb:
            self._check(self.lib.sccg_copy(self.h, ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src.data_ptr()),
                                           nb, _stream(stream)), "sccg_copy")

    def work_counters(self, reset: bool = True) -> dict:
        a = (ctypes.c_uint64 * 12)()
        self._check(self.lib.sccg_work_counters(self.h, a, int(reset)), "sccg_work_counters")
        return dict(strip_edges=a[0], pixel_edges=a[1], box_edges=a[2], boxes=a[3], row_entries=a[4],
                    row_edges=a[5], scan_entries=a[6], scan_pairs=a[7], leaf_pixels=a[8], window_pixels=a[9],
                    raster_out=a[10], raster_and=a[11])


def alu_probe(device: int = 0, iters: int = 4096) -> tuple[float, float]:
    """(ms, int32 lane operations) of one run of the library's integer ALU issue-rate kernel."""
    lib = _native.load()
    ms, ops = ctypes.c_double(), ctypes.c_double()
    st = lib.sccg_alu_probe(int(device), int(iters), ctypes.byref(ms), ctypes.byref(ops))
    if st != SCCG_OK:
        raise SccgError(st, "sccg_alu_probe")
    return ms.value, ops.value


def cross_compare(ctx: Context, A: DevicePolySet, B: DevicePolySet, mode: int = MODE_PLAIN, stream=None):
    """The whole path on prepared sets: candidate pairs, pair areas, Jaccard."""
    pa, pb = ctx.candidate_pairs(A, B, stream=stream)
    inter, uni = ctx.pair_areas(A, B, pa, pb, mode=mode, stream=stream)
    return dict(pa=pa, pb=pb, inter=inter, uni=uni, jaccard=ctx.jaccard(inter, uni, stream=stream))
