"""Build and load the CUDA library libsccg.so (sm_103a) and declare its C ABI for ctypes.

The library is compiled in-tree with nvcc into ``paper_1208_0277_gb300/_build/``. Loading it needs
no GPU; calling into it does. There is no fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
CSRC = os.path.join(_PKG, "csrc")
INCLUDE = os.path.join(_ROOT, "include")
BUILD_DIR = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsccg.so")
SOURCES = ["sccg_api.cu"]
HEADERS = ["leaf64.cuh", "pixelbox.cuh", "scanline.cuh", "kernels.cuh", "raster.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

# Every symbol include/sccg.h declares (checked by the CPU test suite).
EXPORTS = [
    "sccg_status_str", "sccg_ctx_create", "sccg_ctx_destroy", "sccg_ctx_set_param",
    "sccg_ctx_get_params", "sccg_last_error", "sccg_prepare", "sccg_candidate_pairs",
    "sccg_pair_areas", "sccg_pair_areas_tiles", "sccg_batch_run", "sccg_launch_count", "sccg_jaccard",
    "sccg_jaccard_static", "sccg_work_counters", "sccg_build_bands", "sccg_gather_pairs",
    "sccg_jaccard_segments", "sccg_rebase_pairs", "sccg_prepare_sets", "sccg_contains", "sccg_touches",
    "sccg_alu_probe", "sccg_ctx_reserve", "sccg_raster_bytes", "sccg_copy",
]

_lock = threading.Lock()
_lib = None


def nvcc_command(out: str) -> list[str]:
    nvcc = os.environ.get("NVCC", "nvcc")
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    return [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            f"-I{INCLUDE}", "-o", out] + srcs


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "sccg.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libsccg.so for sm_103a (no GPU needed)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or _stale():
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        cmd = nvcc_command(tmp)
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class PolySetC(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("off", ctypes.c_void_p),
        ("xy", ctypes.c_void_p),
        ("tile", ctypes.c_void_p),
        ("mbr", ctypes.c_void_p),
        ("area", ctypes.c_void_p),
        ("max_nv", ctypes.c_int32),
        ("max_extent", ctypes.c_int32),
        ("n_tiles", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("band_bytes", ctypes.c_int64),
        ("bands", ctypes.c_void_p),
        ("raster", ctypes.c_void_p),
        ("raster_cap", ctypes.c_int64),
        ("raster_bytes", ctypes.c_int64),
        ("raster_ok", ctypes.c_int32),
        ("raster_pad", ctypes.c_int32),
    ]


class ParamsC(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("split_pixels", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("area_method", ctypes.c_int32), ("leaf_words", ctypes.c_int32), ("pair_lanes", ctypes.c_int32),
                ("area_T", ctypes.c_int32), ("rasters", ctypes.c_int32), ("raster_heavy", ctypes.c_int32),
                ("raster_lanes", ctypes.c_int32)]


class JaccardC(ctypes.Structure):
    _fields_ = [("sum_inter", ctypes.c_int64), ("sum_union", ctypes.c_int64),
                ("n_nonzero", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("J", ctypes.c_double), ("Jprime", ctypes.c_double)]


def load(path: str | None = None):
    """Load libsccg.so and declare argument types. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libsccg.so not found at {p}: build it with "
                               "paper_1208_0277_gb300.build() (nvcc, sm_103a)")
        lib = ctypes.CDLL(p)
        V, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        PS = ctypes.POINTER(PolySetC)
        sig = {
            "sccg_status_str": ([I], ctypes.c_char_p),
            "sccg_ctx_create": ([I, ctypes.c_char_p, ctypes.POINTER(V)], I),
            "sccg_ctx_destroy": ([V], I),
            "sccg_ctx_set_param": ([V, ctypes.c_char_p, I64], I),
            "sccg_ctx_get_params": ([V, ctypes.POINTER(ParamsC)], I),
            "sccg_ctx_reserve": ([V, I64], I),
            "sccg_last_error": ([V], ctypes.c_char_p),
            "sccg_prepare": ([V, PS, V], I),
            "sccg_prepare_sets": ([V, PS, I, V], I),
            "sccg_raster_bytes": ([V, PS, ctypes.POINTER(I64), V], I),
            "sccg_candidate_pairs": ([V, PS, PS, V, V, I64, ctypes.POINTER(I64), V, V], I),
            "sccg_pair_areas": ([V, PS, PS, V, V, I64, V, V, I, V], I),
            "sccg_pair_areas_tiles": ([V, PS, PS, V, V, V, ctypes.c_int32, V, V, V], I),
            "sccg_batch_run": ([V, PS, PS, V, V, I64, V, V, V, V], I),
            "sccg_gather_pairs": ([V, V, V, V, V, ctypes.c_int32, V, V, V], I),
            "sccg_jaccard_segments": ([V, V, V, V, ctypes.c_int32, V, V], I),
            "sccg_launch_count": ([V, ctypes.POINTER(ctypes.c_uint64)], I),
            "sccg_jaccard": ([V, V, V, I64, V, V], I),
            "sccg_jaccard_static": ([V, V, I64, V, V], I),
            "sccg_build_bands": ([V, PS, V, I64, V], I),
            "sccg_rebase_pairs": ([V, V, V, I64, I64, I64, V], I),
            "sccg_contains": ([V, PS, PS, V, V, V, I64, V, V], I),
            "sccg_touches": ([V, PS, PS, V, V, I64, V, V], I),
            "sccg_work_counters": ([V, ctypes.POINTER(ctypes.c_uint64), I], I),
            "sccg_copy": ([V, V, V, I64, V], I),
            "sccg_alu_probe": ([I, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                               I),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        if path is None:
            _lib = lib
        return lib
