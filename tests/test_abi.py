"""CPU checks of the boundary: the library builds for sm_103a, loads without a GPU and exports every
entry point include/sccg.h declares; the binding's structs match the header's layout."""
import ctypes
import os
import re

import pytest

from paper_1208_0277_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _native.build()
    return ctypes.CDLL(_native.LIB_PATH)


def header_functions():
    src = open(os.path.join(ROOT, "include", "sccg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sccg_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_what_the_binding_lists():
    assert header_functions() == sorted(_native.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    f = lib.sccg_status_str
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"ok"
    assert f(3) == b"output capacity too small"
    assert f(99) == b"unknown status"


def test_struct_sizes_match_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives the header's structs."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"sccg_polyset": _native.PolySetC, "sccg_params": _native.ParamsC,
               "sccg_jaccard_result": _native.JaccardC}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sccg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0; }"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_ctx_create_without_gpu_reports_not_supported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    f = lib.sccg_ctx_create
    f.argtypes = [ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    st = f(0, None, ctypes.byref(h))
    assert st != 0 and not h.value


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1208_0277_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "sccg_oracle" not in txt, fn


def test_copy_refuses_a_missing_context_and_bad_sizes(lib):
    """sccg_copy's host-side checks, before any CUDA call: no context, a negative size."""
    f = lib.sccg_copy
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    buf = (ctypes.c_uint32 * 16)()
    assert f(None, ctypes.addressof(buf), ctypes.addressof(buf), 64, None) != 0
    assert f(None, ctypes.addressof(buf), ctypes.addressof(buf), -4, None) != 0
