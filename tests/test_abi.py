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
        " sizeof(tms_stats), offsetof(tms_hit, P), offsetof(tms_params, tau));"
        " printf(\"%zu %zu %zu\\n\", offsetof(tms_params, patch), offsetof(tms_params, spin_limit),"
        " offsetof(tms_params, autotune_cache)); return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    p, h, s, off_p, off_tau, off_patch, off_spin, off_cache = map(int, out)
    assert (off_patch, off_spin, off_cache) == (tms.Params.patch.offset, tms.Params.spin_limit.offset,
                                                tms.Params.autotune_cache.offset)
    assert p == ctypes.sizeof(tms.Params)
    assert h == tms.HIT_BYTES == 128
    assert s == ctypes.sizeof(tms.Stats)
    assert off_p == 6 * 8          # P at float64 column 6 of the record view
    assert off_tau == tms.Params.tau.offset


def test_defaults_and_status_strings():
    p = tms.params()
    assert (p.precision, p.face_level, p.cell_filter, p.narrow_filter, p.use_graph, p.patch) == (1, 1, 1, 1, 1, 1)
    assert p.spin_limit == 0 and p.autotune_cache is None
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
    assert reserved.value == 72 << 20
    assert 0 < needed.value <= reserved.value


def test_refine_struct_layouts_match_ctypes(tmp_path):
    prog = tmp_path / "rsizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tms.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(tms_surface_pair),"
        " sizeof(tms_refine_params), offsetof(tms_surface_pair, alpha_s),"
        " offsetof(tms_surface_pair, c0), offsetof(tms_surface_pair, reg),"
        " offsetof(tms_refine_params, max_iter)); return 0;}\n")
    exe = tmp_path / "rsizes"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    S, R = tms.SurfacePair, tms.RefineParams
    assert vals == [ctypes.sizeof(S), ctypes.sizeof(R), S.alpha_s.offset, S.c0.offset,
                    S.reg.offset, R.max_iter.offset]


def test_refine_arguments_checked_without_gpu():
    import synth
    lib = tms.lib()
    sp = tms.surface_pair(synth.config1().surface)
    assert sp.n_harmonics == 6 and sp.n_folds == 0 and sp.stretch == 0
    p = tms.refine_params()
    assert (p.alpha0, p.alpha1, p.tol, p.max_iter) == (0.5, 0.5, 1e-10, 200)
    B = ctypes.byref
    # n == 0 is a no-op; everything below is rejected before any device call
    assert lib.tms_refine(B(sp), B(p), None, 4, 0, None, None, None, None, None, None) == tms.TMS_OK
    assert lib.tms_refine(None, B(p), None, 4, 0, None, None, None, None, None, None) == tms.TMS_ERR_ARG
    assert lib.tms_refine(B(sp), B(p), None, 4, -1, None, None, None, None, None, None) == tms.TMS_ERR_ARG
    for field, bad in (("alpha0", 0.0), ("alpha1", 1.5), ("tol", -1.0), ("max_iter", -1),
                       ("s_hi", -1.0), ("rho_min", float("nan"))):
        q = tms.refine_params(**{field: bad})
        assert lib.tms_refine(B(sp), B(q), None, 4, 0, None, None, None, None, None,
                              None) == tms.TMS_ERR_ARG, field
    bad = tms.surface_pair(synth.config1().surface)
    bad.n_harmonics = 9
    assert lib.tms_refine(B(bad), B(p), None, 4, 0, None, None, None, None, None, None) == tms.TMS_ERR_ARG
    bad = tms.surface_pair(synth.config1().surface)
    bad.h_amp = float("inf")
    assert lib.tms_refine(B(bad), B(p), None, 4, 0, None, None, None, None, None, None) == tms.TMS_ERR_ARG
    assert "non-finite" in tms.last_error()
    # seeds must be given for n > 0 (rejected before the pointer query)
    assert lib.tms_refine(B(sp), B(p), None, 4, 3, None, None, None, None, None, None) == tms.TMS_ERR_ARG
    assert lib.tms_refine(B(sp), B(p), None, 3, 3, None, None, None, None, None, None) == tms.TMS_ERR_ARG


def test_layer_pairs_host_enumeration_matches_oracle():
    import synth
    from oracle import layers as L
    p = synth.layered_pair(NA=96, NB=128, n_max=3, per_layer=8, sites=(8, 6), n_hits=12)
    lay = p.meta["layers"]
    args = (lay["D_u"], lay["lam_u"])
    got = tms.layer_pairs(p.A.s, *args, p.B.s, lay["D_s"], lay["lam_s"], lay["n_max"])
    want = L.layer_pairs(p.A.s.numpy(), *args, p.B.s.numpy(), lay["D_s"], lay["lam_s"], lay["n_max"])
    assert got == want and len(got) == 24
    lib = tms.lib()
    a, b = p.A.s.contiguous(), p.B.s.contiguous()
    buf = (tms.LayerPair * 4)()
    cnt = ctypes.c_int(0)
    rc = lib.tms_layer_pairs(a.data_ptr(), a.numel(), *args, b.data_ptr(), b.numel(), lay["D_s"],
                             lay["lam_s"], 3, 1e-9, buf, 4, ctypes.byref(cnt))
    assert rc == tms.TMS_ERR_CAPACITY and cnt.value == 24
    assert buf[3].as_dict() == want[3]
    with pytest.raises(tms.TmsError):
        tms.layer_pairs(p.A.s, lay["D_u"] * 1.3, lay["lam_u"], p.B.s, lay["D_s"], lay["lam_s"], 3)
    with pytest.raises(tms.TmsError):
        tms.layer_pairs(p.A.s, lay["D_u"], 0.5, p.B.s, lay["D_s"], lay["lam_s"], 3)
    with pytest.raises(tms.TmsError):                     # more layers than the mesh holds
        tms.layer_pairs(p.A.s, lay["D_u"], lay["lam_u"], p.B.s, lay["D_s"], lay["lam_s"], 4)


def test_theta_arguments_checked_without_gpu():
    lib = tms.lib()
    # sizes are checked before any device call; an empty batch is a no-op
    assert lib.tms_theta_translate(None, None, 12, 4, 4, 48, None, 0.0, 0, None) == tms.TMS_ERR_ARG
    assert lib.tms_theta_translate(None, None, 16384, 4, 4, 65536, None, 0.0, 0, None) == tms.TMS_ERR_ARG
    assert lib.tms_theta_translate(None, None, 64, 0, 4, 0, None, 0.0, 0, None) == tms.TMS_OK
    assert lib.tms_theta_translate(None, None, 64, 4, 4, 64, None, 0.0, 0, None) == tms.TMS_ERR_ARG
    assert lib.tms_theta_translate(None, None, 64, 4, 4, 256, None, float("nan"), 0, None) == tms.TMS_ERR_ARG
    assert lib.tms_phase_align(None, None, 64, 9, 1, None, None, None) == tms.TMS_ERR_ARG
    assert lib.tms_phase_align(None, None, 64, 4, 0, None, None, None) == tms.TMS_OK
