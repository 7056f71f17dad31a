"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/tms.h, and the ctypes mirrors match the C struct layouts."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2109_14814_gb300 as tms
from paper_2109_14814_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tms.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    libbuild.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tms_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 12
    lib = ctypes.CDLL(tms._binding.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_ctypes(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tms.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(tms_params), sizeof(tms_hit),"
        " sizeof(tms_stats), offsetof(tms_hit, P), offsetof(tms_params, tau)); return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    p, h, s, off_p, off_tau = map(int, out)
    assert p == ctypes.sizeof(tms.Params)
    assert h == tms.HIT_BYTES == 128
    assert s == ctypes.sizeof(tms.Stats)
    assert off_p == 6 * 8          # P at float64 column 6 of the record view
    assert off_tau == tms.Params.tau.offset


def test_defaults_and_status_strings():
    p = tms.params()
    assert (p.precision, p.face_level, p.cell_filter, p.narrow_filter, p.use_graph) == (1, 1, 1, 1, 1)
    assert abs(p.tau - 1e-12) < 1e-30 and p.cell_mult > 1.0
    assert tms.status_str(tms.TMS_ERR_CAPACITY) == "capacity exceeded"
    assert "sm_103a" in tms.version()


def test_null_arguments_rejected_without_gpu():
    lib = tms.lib()
    out = ctypes.c_void_p()
    assert lib.tms_build_mesh(None, None, None, None, 4, 4, 0, 4, None, 1, None,
                              ctypes.byref(out)) == tms.TMS_ERR_ARG
    assert lib.tms_destroy_mesh(None) == tms.TMS_ERR_STATE
    n = ctypes.c_longlong()
    assert lib.tms_search(None, None, None, None, 0, ctypes.byref(n), None) != tms.TMS_OK
    best = tms.Params()
    assert lib.tms_autotune(None, None, 1, None, ctypes.byref(best), None, None,
                            None) == tms.TMS_ERR_ARG
    assert lib.tms_autotune(None, None, 0, None, ctypes.byref(best), None, None,
                            None) == tms.TMS_ERR_ARG


def test_noalloc_layout_fits_its_static_array():
    lib = tms.lib()
    needed, reserved = ctypes.c_ulonglong(), ctypes.c_ulonglong()
    lib.tms_noalloc_footprint.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.tms_noalloc_footprint(ctypes.byref(needed), ctypes.byref(reserved)) == tms.TMS_OK
    assert reserved.value == 64 << 20
    assert 0 < needed.value <= reserved.value
