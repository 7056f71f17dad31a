"""Thin Python binding of libtms.so (include/tms.h): argument marshalling only.

PyTorch supplies device memory and the current stream; every step of the
search runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is not built, or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtms.so")
HIT_BYTES = 128

TMS_OK, TMS_ERR_ARG, TMS_ERR_CAPACITY, TMS_ERR_TIMEOUT, TMS_ERR_CUDA, TMS_ERR_STATE = range(6)

_c = ctypes
_lib = None


class TmsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({last_error()})")


class Params(ctypes.Structure):
    """Mirror of tms_params."""
    _fields_ = [
        ("precision", _c.c_int),
        ("face_level", _c.c_int),
        ("moller", _c.c_int),
        ("cell_filter", _c.c_int),
        ("narrow_filter", _c.c_int),
        ("cell_mult", _c.c_float),
        ("tau", _c.c_double),
        ("entry_capacity", _c.c_longlong),
        ("cand_capacity", _c.c_longlong),
        ("hit_capacity", _c.c_longlong),
        ("use_graph", _c.c_int),
        ("inject", _c.c_uint),
        ("block_faces", _c.c_int),
        ("tile_rows", _c.c_int),
        ("timing", _c.c_int),
        ("patch", _c.c_int),
        ("pad0", _c.c_int),
        ("spin_limit", _c.c_longlong),
        ("autotune_cache", _c.c_char_p),
    ]


class Stats(ctypes.Structure):
    """Mirror of tms_stats."""
    _fields_ = [
        ("entries", _c.c_longlong),
        ("cells", _c.c_longlong),
        ("pair_slots", _c.c_longlong),
        ("candidates", _c.c_longlong),
        ("fp64_solves", _c.c_longlong),
        ("raw_hits", _c.c_longlong),
        ("hits", _c.c_longlong),
        ("grid_n", _c.c_int * 4),
        ("empty", _c.c_int),
        ("retries", _c.c_int),
        ("kernels", _c.c_int),
        ("pad", _c.c_int),
        ("fp32_solves", _c.c_longlong),
        ("sat_tests", _c.c_longlong),
        ("quad_tests", _c.c_longlong),
        ("patch_pairs", _c.c_longlong),
        ("patch_tests", _c.c_longlong),
        ("quad_kept", _c.c_longlong),
        ("patch_kept", _c.c_longlong),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "grid_n"}
        d["grid_n"] = list(self.grid_n)
        return d


class LayerPair(ctypes.Structure):
    """Mirror of tms_layer_pair."""
    _fields_ = [(f, _c.c_int) for f in ("n", "m", "sign_u", "sign_s", "a_k0", "a_k1", "b_k0", "b_k1")]

    def as_dict(self):
        return dict(n=self.n, m=self.m, sign_u=self.sign_u, sign_s=self.sign_s,
                    a=(self.a_k0, self.a_k1), b=(self.b_k0, self.b_k1))


class SurfacePair(ctypes.Structure):
    """Mirror of tms_surface_pair (the closed-form sheet pair refined on)."""
    _fields_ = [
        ("n_harmonics", _c.c_int), ("n_folds", _c.c_int), ("stretch", _c.c_int), ("pad", _c.c_int),
        ("ca", (_c.c_double * 4) * 8), ("cb", (_c.c_double * 4) * 8),
        ("dca", (_c.c_double * 4) * 8), ("dcb", (_c.c_double * 4) * 8),
        ("alpha_u", _c.c_double), ("alpha_s", _c.c_double), ("alpha_ref", _c.c_double),
        ("lam", _c.c_double),
        ("fold_amp", _c.c_double * 4), ("fold_root", (_c.c_double * 3) * 4),
        ("fold_dir", (_c.c_double * 4) * 4),
        ("c0", _c.c_double), ("h_amp", _c.c_double), ("P", _c.c_double), ("Q", _c.c_double),
        ("theta0", _c.c_double), ("s0", _c.c_double),
        ("v1", _c.c_double * 4), ("v2", _c.c_double * 4), ("reg", _c.c_double),
    ]


class RefineParams(ctypes.Structure):
    """Mirror of tms_refine_params."""
    _fields_ = [
        ("alpha0", _c.c_double), ("alpha1", _c.c_double), ("switch_below", _c.c_double),
        ("tol", _c.c_double), ("s_lo", _c.c_double), ("s_hi", _c.c_double),
        ("rho_min", _c.c_double), ("max_iter", _c.c_int), ("pad", _c.c_int),
    ]


class ContinueParams(ctypes.Structure):
    """Mirror of tms_continue_params."""
    _fields_ = [("corrector", RefineParams), ("rho_turn", _c.c_double), ("max_jump", _c.c_double),
                ("param", _c.c_int), ("pad", _c.c_int)]


REFINE_STATUS = ("converged", "max_iter", "singular", "escaped", "non_finite")
CONTINUE_STATUS = REFINE_STATUS + ("turning", "jumped", "stopped")


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2109_14814_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, LL, D = _c.c_void_p, _c.c_int, _c.c_longlong, _c.c_double
    L.tms_params_default.argtypes = [_c.POINTER(Params)]
    L.tms_params_default.restype = None
    L.tms_build_mesh.argtypes = [P, P, P, P, I, I, I, I, P, I, P, _c.POINTER(P)]
    L.tms_build_mesh.restype = I
    L.tms_destroy_mesh.argtypes = [P]
    L.tms_destroy_mesh.restype = I
    L.tms_search.argtypes = [P, P, _c.POINTER(Params), P, LL, _c.POINTER(LL), P]
    L.tms_search.restype = I
    L.tms_search_batched.argtypes = [P, P, I, _c.POINTER(Params), P, LL, P, _c.POINTER(LL), P]
    L.tms_search_host.argtypes = [P, P, P, P, _c.POINTER(Params), P, LL, _c.POINTER(LL), P]
    L.tms_search_host.restype = I
    L.tms_search_batched.restype = I
    L.tms_backward.argtypes = [P, P, P, LL, P, P, P, P, P, P, P, P]
    L.tms_backward.restype = I
    L.tms_last_stats.argtypes = [P, _c.POINTER(Stats)]
    L.tms_last_stats.restype = I
    L.tms_last_stage_ms.argtypes = [P, _c.POINTER(_c.c_float), I, _c.POINTER(I)]
    L.tms_last_stage_ms.restype = I
    L.tms_release_workspace.argtypes = [P]
    L.tms_release_workspace.restype = I
    L.tms_last_patch_frames.argtypes = [P, I, _c.POINTER(_c.c_float), LL, _c.POINTER(LL), _c.POINTER(I)]
    L.tms_last_patch_frames.restype = I
    L.tms_status_str.argtypes = [I]
    L.tms_status_str.restype = _c.c_char_p
    L.tms_version.argtypes = []
    L.tms_version.restype = _c.c_char_p
    L.tms_last_error.argtypes = []
    L.tms_last_error.restype = _c.c_char_p
    L.tms_probe_fp64.argtypes = [_c.POINTER(D), P]
    L.tms_probe_fp64.restype = I
    L.tms_search_noalloc.argtypes = [P, P, _c.POINTER(Params), P, LL, _c.POINTER(LL), P]
    L.tms_search_noalloc.restype = I
    L.tms_noalloc_last_error.argtypes = []
    L.tms_noalloc_last_error.restype = _c.c_char_p
    L.tms_autotune.argtypes = [P, P, I, _c.POINTER(Params), _c.POINTER(Params), _c.c_char_p,
                               _c.POINTER(D), P]
    L.tms_autotune.restype = I
    L.tms_refine_params_default.argtypes = [_c.POINTER(RefineParams)]
    L.tms_refine_params_default.restype = None
    L.tms_refine.argtypes = [_c.POINTER(SurfacePair), _c.POINTER(RefineParams), P, LL, LL, P, P, P,
                             P, P, P]
    L.tms_refine.restype = I
    L.tms_continue_params_default.argtypes = [_c.POINTER(ContinueParams)]
    L.tms_continue_params_default.restype = None
    L.tms_continue.argtypes = [_c.POINTER(SurfacePair), _c.POINTER(ContinueParams), P, I, P, LL, LL,
                               P, P, P, P, P, P]
    L.tms_continue.restype = I
    L.tms_layer_pairs.argtypes = [P, I, D, D, P, I, D, D, I, D, P, I, _c.POINTER(I)]
    L.tms_layer_pairs.restype = I
    L.tms_layer_plan_create.argtypes = [P, P, P, I, P, _c.POINTER(P)]
    L.tms_layer_plan_create.restype = I
    L.tms_layer_plan_destroy.argtypes = [P]
    L.tms_layer_plan_destroy.restype = I
    L.tms_layer_search.argtypes = [P, _c.POINTER(Params), P, LL, P, _c.POINTER(LL), P]
    L.tms_layer_search.restype = I
    L.tms_theta_translate.argtypes = [P, P, I, I, I, LL, P, D, I, P]
    L.tms_theta_translate.restype = I
    L.tms_phase_align.argtypes = [P, P, I, I, I, P, P, P]
    L.tms_phase_align.restype = I
    _lib = L
    return L


def search_noalloc(A: "Mesh", B: "Mesh", out: torch.Tensor, stream=None, **kw) -> "Hits":
    """tms_search_noalloc: the search with every scratch buffer in the library's
    static device array, for callers that must not allocate device memory
    (software that fixes its device footprint at start-up, or services whose
    device memory is all held by a pool allocator).  The caller passes the
    output buffer `out` ((capacity, 128) uint8, on the device); nothing is
    allocated.  Limits and sharing rules: see include/tms.h."""
    p = params(**kw)
    n = _c.c_longlong(0)
    rc = lib().tms_search_noalloc(A.handle, B.handle, _c.byref(p), out.data_ptr(), out.shape[0],
                                  _c.byref(n), _stream(stream))
    if rc != TMS_OK:
        msg = lib().tms_noalloc_last_error().decode()
        err = TmsError.__new__(TmsError)
        err.status = rc
        RuntimeError.__init__(err, f"tms_search_noalloc: {status_str(rc)} ({msg})")
        raise err
    return Hits(out[: n.value])


def autotune(As: Sequence["Mesh"], Bs: Sequence["Mesh"], cache_path: Optional[str] = None,
             stream=None, **kw):
    """tms_autotune: the fastest (face_level, cell_mult, block_faces) for these
    mesh pairs (one pair: tms_search; several: tms_search_batched), the other
    parameters taken from **kw.  Returns (params dict, median ms)."""
    if len(As) != len(Bs) or not As:
        raise ValueError("As and Bs must be non-empty and of equal length")
    base = params(**kw)
    best = Params()
    ms = _c.c_double(0.0)
    ha = (_c.c_void_p * len(As))(*[m.handle.value for m in As])
    hb = (_c.c_void_p * len(Bs))(*[m.handle.value for m in Bs])
    rc = lib().tms_autotune(ha, hb, len(As), _c.byref(base), _c.byref(best),
                            cache_path.encode() if cache_path else None, _c.byref(ms),
                            _stream(stream))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_autotune")
    return {f: getattr(best, f) for f, _ in Params._fields_}, float(ms.value)


def probe_fp64_tflops(stream=None) -> float:
    """tms_probe_fp64: measured FP64 FMA throughput of the current GPU."""
    v = _c.c_double(0.0)
    rc = lib().tms_probe_fp64(_c.byref(v), _stream(stream))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_probe_fp64")
    return float(v.value)


def status_str(s: int) -> str:
    return lib().tms_status_str(s).decode()


def last_error() -> str:
    return lib().tms_last_error().decode()


def version() -> str:
    return lib().tms_version().decode()


def params(**kw) -> Params:
    p = Params()
    lib().tms_params_default(_c.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k) or k == "pad0":
            raise KeyError(f"unknown search parameter {k!r}")
        if k == "autotune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(p, k, v)
    return p


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


class Mesh:
    """A mesh view (tms_build_mesh): X is a CUDA float64 tensor (4, M, N),
    coordinate c of vertex (theta_i, s_k) at X[c, k, i]; s holds the M s_k."""

    def __init__(self, X: torch.Tensor, s, periodic: bool = True, k0: int = 0,
                 k1: Optional[int] = None, stream=None):
        if not (X.is_cuda and X.dtype == torch.float64 and X.dim() == 3 and X.shape[0] == 4):
            raise ValueError("X must be a CUDA float64 tensor of shape (4, M, N)")
        self.X = X.contiguous()
        self.M, self.N = int(X.shape[1]), int(X.shape[2])
        if isinstance(s, torch.Tensor):
            s_t = s.detach().to(torch.float64).contiguous()
        else:
            s_t = torch.as_tensor(s, dtype=torch.float64).contiguous()
        self.s = s_t
        self.periodic = bool(periodic)
        self.k0 = int(k0)
        self.k1 = int(self.M if k1 is None else k1)
        h = _c.c_void_p()
        rc = lib().tms_build_mesh(self.X[0].data_ptr(), self.X[1].data_ptr(), self.X[2].data_ptr(),
                                  self.X[3].data_ptr(), self.N, self.M, self.k0, self.k1,
                                  self.s.data_ptr(), int(self.periodic), _stream(stream),
                                  _c.byref(h))
        if rc != TMS_OK:
            raise TmsError(rc, "tms_build_mesh")
        self.handle = h

    @classmethod
    def from_grid(cls, g, device="cuda", **kw):
        """From a synth.MeshGrid."""
        return cls(g.X.to(device).contiguous(), g.s.cpu(), g.periodic, **kw)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.tms_destroy_mesh(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Hits:
    """Search output on the device (views of the raw tms_hit records)."""
    raw: torch.Tensor          # (n, 128) uint8
    offsets: Optional[torch.Tensor] = None

    def __len__(self):
        return int(self.raw.shape[0])

    @property
    def _i32(self):
        return self.raw.view(torch.int32)

    @property
    def _f64(self):
        return self.raw.view(torch.float64)

    @property
    def triA(self):
        return self._i32[:, 0].to(torch.int64)

    @property
    def triB(self):
        return self._i32[:, 1].to(torch.int64)

    @property
    def pair(self):
        return self._i32[:, 2].to(torch.int64)

    @property
    def flags(self):
        return self._i32[:, 3].to(torch.int64)

    @property
    def z(self):
        return self._f64[:, 2:6]

    @property
    def P(self):
        return self._f64[:, 6:10]

    @property
    def params(self):
        return self._f64[:, 10:14]

    @property
    def rho(self):
        return self._f64[:, 14]

    @property
    def margin(self):
        return self._f64[:, 15]

    def to_dict(self):
        return dict(triA=self.triA, triB=self.triB, pair=self.pair, flags=self.flags, z=self.z,
                    P=self.P, params=self.params, rho=self.rho, margin=self.margin)


def _alloc_hits(cap: int, device) -> torch.Tensor:
    return torch.empty((max(cap, 1), HIT_BYTES), dtype=torch.uint8, device=device)


def search(A: Mesh, B: Mesh, hit_capacity: int = 1 << 16, stream=None, out=None, **kw) -> Hits:
    """tms_search: all intersecting triangle pairs of A against B."""
    p = params(**kw)
    st = _stream(stream)
    buf = out if out is not None else _alloc_hits(hit_capacity, A.X.device)
    n = _c.c_longlong(0)
    rc = lib().tms_search(A.handle, B.handle, _c.byref(p), buf.data_ptr(), buf.shape[0],
                          _c.byref(n), st)
    if rc == TMS_ERR_CAPACITY and out is None and n.value > buf.shape[0] and not (p.inject & 2):
        buf = _alloc_hits(int(n.value), A.X.device)
        rc = lib().tms_search(A.handle, B.handle, _c.byref(p), buf.data_ptr(), buf.shape[0],
                              _c.byref(n), st)
    if rc != TMS_OK:
        raise TmsError(rc, "tms_search")
    return Hits(buf[: n.value])


def search_host(A: Mesh, B: Mesh, XA: torch.Tensor, XB: torch.Tensor, out: torch.Tensor = None,
                hit_capacity: int = 1 << 16, stream=None, **kw) -> Hits:
    """tms_search_host: the search from host coordinates.  XA, XB: CPU float64
    tensors of the meshes' full (4, M, N) shape (pinned memory copies fastest),
    copied into the meshes' device arrays; the hits land in `out` (a CPU uint8
    tensor of hit records, pinned for speed) or a new one."""
    for X, m in ((XA, A), (XB, B)):
        if X.device.type != "cpu" or X.dtype != torch.float64 or tuple(X.shape) != tuple(m.X.shape) \
                or not X.is_contiguous():
            raise ValueError("host coordinates must be contiguous CPU float64 of the mesh's shape")
    p = params(**kw)
    st = _stream(stream)
    buf = out if out is not None else torch.empty((max(hit_capacity, 1), HIT_BYTES), dtype=torch.uint8)
    ha = (_c.c_void_p * 4)(*[XA[c].data_ptr() for c in range(4)])
    hb = (_c.c_void_p * 4)(*[XB[c].data_ptr() for c in range(4)])
    n = _c.c_longlong(0)
    rc = lib().tms_search_host(A.handle, ha, B.handle, hb, _c.byref(p), buf.data_ptr(), buf.shape[0],
                               _c.byref(n), st)
    if rc != TMS_OK:
        raise TmsError(rc, "tms_search_host")
    return Hits(buf[: n.value])


def search_batched(As: Sequence[Mesh], Bs: Sequence[Mesh], hit_capacity: int = 1 << 18,
                   stream=None, out=None, offsets=None, **kw) -> Hits:
    """tms_search_batched: independent searches of many mesh pairs in one graph."""
    if len(As) != len(Bs) or not As:
        raise ValueError("As and Bs must be non-empty and of equal length")
    p = params(**kw)
    st = _stream(stream)
    dev = As[0].X.device
    ha = (_c.c_void_p * len(As))(*[m.handle.value for m in As])
    hb = (_c.c_void_p * len(Bs))(*[m.handle.value for m in Bs])
    buf = out if out is not None else _alloc_hits(hit_capacity, dev)
    offs = offsets if offsets is not None else torch.empty(len(As) + 1, dtype=torch.int64, device=dev)
    n = _c.c_longlong(0)
    rc = lib().tms_search_batched(ha, hb, len(As), _c.byref(p), buf.data_ptr(), buf.shape[0],
                                  offs.data_ptr(), _c.byref(n), st)
    if rc == TMS_ERR_CAPACITY and out is None and n.value > buf.shape[0]:
        buf = _alloc_hits(int(n.value), dev)
        rc = lib().tms_search_batched(ha, hb, len(As), _c.byref(p), buf.data_ptr(), buf.shape[0],
                                      offs.data_ptr(), _c.byref(n), st)
    if rc != TMS_OK:
        raise TmsError(rc, "tms_search_batched")
    return Hits(buf[: n.value], offs)


def backward(A: Mesh, B: Mesh, hits: Hits, gP=None, gZ=None, gradA=None, gradB=None,
             dA_dalpha=None, dB_dalpha=None, galpha=None, stream=None):
    """tms_backward: accumulates vertex gradients into gradA/gradB (4, M, N) and
    writes per-hit alpha derivatives into galpha (n,)."""
    n = len(hits)
    for t in (gP, gZ):
        if t is not None and (t.dtype != torch.float64 or not t.is_contiguous()):
            raise ValueError("upstream gradients must be contiguous float64 (n, 4)")
    rc = lib().tms_backward(A.handle, B.handle, hits.raw.data_ptr() if n else None, n,
                            _dptr(gP), _dptr(gZ), _dptr(gradA), _dptr(gradB), _dptr(dA_dalpha),
                            _dptr(dB_dalpha), _dptr(galpha), _stream(stream))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_backward")


def last_stats(stream=None) -> dict:
    s = Stats()
    rc = lib().tms_last_stats(_stream(stream), _c.byref(s))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_last_stats")
    return s.as_dict()


STAGES = ["init", "face_bounds", "grid_params", "bitmap_clear", "face_mark_A", "face_probe_B",
          "face_probe_A", "group_count", "group_cells", "emit", "patch_quads", "narrow",
          "sort_hits", "merge_output", "readback"]


def last_stage_ms(stream=None) -> dict:
    """Per-stage device time of the last search made with timing=1."""
    buf = (_c.c_float * 32)()
    n = _c.c_int(0)
    rc = lib().tms_last_stage_ms(_stream(stream), buf, 32, _c.byref(n))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_last_stage_ms")
    return {STAGES[i]: float(buf[i]) for i in range(min(n.value, len(STAGES)))}


def last_patch_frames(side: int = 0, stream=None):
    """The patch frames of the last search on `stream` (mesh A for side 0, B
    for side 1) as a float32 array (patch rows, patches per row, 28): c, e_0..e_3,
    h_0..h_3, rho, L, n_2, n_3 (tms_last_patch_frames)."""
    import numpy as np
    n = _c.c_longlong(0)
    npi = _c.c_int(0)
    rc = lib().tms_last_patch_frames(_stream(stream), side, None, 0, _c.byref(n), _c.byref(npi))
    if rc not in (TMS_OK, TMS_ERR_CAPACITY):
        raise TmsError(rc, "tms_last_patch_frames")
    out = np.zeros((max(n.value, 1), 28), dtype=np.float32)
    rc = lib().tms_last_patch_frames(_stream(stream), side, out.ctypes.data_as(_c.POINTER(_c.c_float)),
                                     out.size, _c.byref(n), _c.byref(npi))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_last_patch_frames")
    return out[:n.value].reshape(-1, max(npi.value, 1), 28)


def surface_pair(sp, alpha_u=None, alpha_s=None) -> SurfacePair:
    """tms_surface_pair from a description with the fields of synth.SurfacePair
    (coefficient tables (K, 4), fold tables (F, 3) and (F, 4), scalars).  W_A is
    taken at alpha_u and B's sheet at alpha_s; each defaults to the
    description's alpha_u / alpha_s attribute, else its alpha."""
    def rows(t):
        return [[float(v) for v in r] for r in (t.tolist() if hasattr(t, "tolist") else t)]
    out = SurfacePair()
    ca, cb, dca, dcb = rows(sp.ca), rows(sp.cb), rows(sp.dca), rows(sp.dcb)
    if not 1 <= len(ca) <= 8:
        raise ValueError("1..8 harmonics supported")
    out.n_harmonics = len(ca)
    for dst, src in ((out.ca, ca), (out.cb, cb), (out.dca, dca), (out.dcb, dcb)):
        for k, r in enumerate(src):
            for c in range(4):
                dst[k][c] = r[c]
    amp = [float(v) for v in (sp.fold_amp.tolist() if hasattr(sp.fold_amp, "tolist") else sp.fold_amp)]
    if len(amp) > 4:
        raise ValueError("at most 4 folds supported")
    out.n_folds = len(amp)
    roots, dirs = rows(sp.fold_roots), rows(sp.fold_dir)
    for f in range(len(amp)):
        out.fold_amp[f] = amp[f]
        for j in range(3):
            out.fold_root[f][j] = roots[f][j]
        for c in range(4):
            out.fold_dir[f][c] = dirs[f][c]
    out.stretch = {"linear": 0, "exp": 1}[sp.stretch]
    out.lam = float(sp.lam)
    for name in ("alpha_ref", "c0", "h_amp", "P", "Q", "theta0", "s0", "reg"):
        setattr(out, name, float(getattr(sp, name)))
    out.alpha_u = float(alpha_u if alpha_u is not None else getattr(sp, "alpha_u", sp.alpha))
    out.alpha_s = float(alpha_s if alpha_s is not None else getattr(sp, "alpha_s", sp.alpha))
    v1 = sp.v1.tolist() if hasattr(sp.v1, "tolist") else sp.v1
    v2 = sp.v2.tolist() if hasattr(sp.v2, "tolist") else sp.v2
    for c in range(4):
        out.v1[c], out.v2[c] = float(v1[c]), float(v2[c])
    return out


def refine_params(**kw) -> RefineParams:
    p = RefineParams()
    lib().tms_refine_params_default(_c.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k) or k == "pad":
            raise KeyError(f"unknown refinement parameter {k!r}")
        setattr(p, k, v)
    return p


@dataclass
class Refined:
    """tms_refine output on the device."""
    x: torch.Tensor        # (n, 4) float64: theta_u, s_u, theta_s, s_s
    fnorm: torch.Tensor    # (n,) float64
    rho: torch.Tensor      # (n,) float64, det Df / prod of column norms
    iters: torch.Tensor    # (n,) int32
    status: torch.Tensor   # (n,) int32, index into REFINE_STATUS


def refine(surface, seeds, stream=None, out: Optional[Refined] = None, **kw) -> Refined:
    """tms_refine: damped Newton (Sec. 7) from each seed on the sheet pair
    `surface` (a SurfacePair mirror or anything surface_pair() accepts).
    seeds: a Hits (their parameter estimates are read in place) or a CUDA
    float64 tensor (n, 4) with unit column stride."""
    sp = surface if isinstance(surface, SurfacePair) else surface_pair(surface)
    p = refine_params(**kw)
    if isinstance(seeds, Hits):
        n = len(seeds)
        dev = seeds.raw.device
        ptr = seeds.raw.data_ptr() + 10 * 8 if n else None
        ld = HIT_BYTES // 8
    else:
        if not (seeds.is_cuda and seeds.dtype == torch.float64 and seeds.dim() == 2
                and seeds.shape[1] == 4 and seeds.stride(1) == 1):
            raise ValueError("seeds must be a CUDA float64 (n, 4) tensor with unit column stride")
        n = int(seeds.shape[0])
        dev = seeds.device
        ptr = seeds.data_ptr() if n else None
        ld = max(int(seeds.stride(0)), 4)
    if out is None:
        out = Refined(torch.empty((n, 4), dtype=torch.float64, device=dev),
                      torch.empty(n, dtype=torch.float64, device=dev),
                      torch.empty(n, dtype=torch.float64, device=dev),
                      torch.empty(n, dtype=torch.int32, device=dev),
                      torch.empty(n, dtype=torch.int32, device=dev))
    rc = lib().tms_refine(_c.byref(sp), _c.byref(p), ptr, ld, n, _dptr(out.x) if n else None,
                          _dptr(out.fnorm) if n else None, _dptr(out.rho) if n else None,
                          _dptr(out.iters) if n else None, _dptr(out.status) if n else None,
                          _stream(stream))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_refine")
    return out


@dataclass
class Continued:
    """tms_continue output on the device; step j of branch b at [b, j]."""
    x: torch.Tensor        # (n, K+1, 4) float64
    status: torch.Tensor   # (n, K+1) int32, index into CONTINUE_STATUS
    iters: torch.Tensor    # (n, K+1) int32
    rho: torch.Tensor      # (n, K+1) float64
    fnorm: torch.Tensor    # (n, K+1) float64
    alphas: torch.Tensor   # (K+1,) float64: the start value, then the steps


def continue_branches(surface, seeds, alphas, param: str = "u", stream=None, rho_turn=None,
                      max_jump=None, **kw) -> Continued:
    """tms_continue: continuation (Sec. 8) of each seed's connection through the
    parameter values `alphas` (K,) of alpha_u (param "u") or alpha_s ("s").
    seeds: CUDA float64 (n, 4) with unit column stride, or a Hits.  **kw are
    corrector (tms_refine_params) fields."""
    sp = surface if isinstance(surface, SurfacePair) else surface_pair(surface)
    p = ContinueParams()
    lib().tms_continue_params_default(_c.byref(p))
    p.corrector = refine_params(**kw)
    p.param = {"u": 0, "s": 1}[param]
    if rho_turn is not None:
        p.rho_turn = rho_turn
    if max_jump is not None:
        p.max_jump = max_jump
    if isinstance(seeds, Hits):
        n, dev = len(seeds), seeds.raw.device
        ptr, ld = (seeds.raw.data_ptr() + 10 * 8 if n else None), HIT_BYTES // 8
    else:
        if not (seeds.is_cuda and seeds.dtype == torch.float64 and seeds.dim() == 2
                and seeds.shape[1] == 4 and seeds.stride(1) == 1):
            raise ValueError("seeds must be a CUDA float64 (n, 4) tensor with unit column stride")
        n, dev = int(seeds.shape[0]), seeds.device
        ptr, ld = (seeds.data_ptr() if n else None), max(int(seeds.stride(0)), 4)
    a = torch.as_tensor(alphas, dtype=torch.float64).reshape(-1).to(dev).contiguous()
    K = int(a.numel())
    start = sp.alpha_u if p.param == 0 else sp.alpha_s
    out = Continued(torch.empty((n, K + 1, 4), dtype=torch.float64, device=dev),
                    torch.empty((n, K + 1), dtype=torch.int32, device=dev),
                    torch.empty((n, K + 1), dtype=torch.int32, device=dev),
                    torch.empty((n, K + 1), dtype=torch.float64, device=dev),
                    torch.empty((n, K + 1), dtype=torch.float64, device=dev),
                    torch.cat([torch.tensor([start], dtype=torch.float64, device=dev), a]))
    rc = lib().tms_continue(_c.byref(sp), _c.byref(p), a.data_ptr() if K else None, K, ptr, ld, n,
                            _dptr(out.x) if n else None, _dptr(out.status) if n else None,
                            _dptr(out.iters) if n else None, _dptr(out.rho) if n else None,
                            _dptr(out.fnorm) if n else None, _stream(stream))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_continue")
    return out


def layer_pairs(sA, D_u: float, lam_u: float, sB, D_s: float, lam_s: float, n_max: int,
                rel_tol: float = 1e-9) -> list:
    """tms_layer_pairs: the 8 n_max half-layer pairs (Sec. 5, Sec. 6.2) of the
    full meshes with s values sA, sB, as dicts (n, m, sign_u, sign_s, a, b)."""
    def host(v):
        arr = (v.detach().cpu() if isinstance(v, torch.Tensor) else torch.as_tensor(v))
        return arr.to(torch.float64).contiguous()
    a, b = host(sA), host(sB)
    cnt = _c.c_int(0)
    buf = (LayerPair * (8 * n_max))()
    rc = lib().tms_layer_pairs(a.data_ptr(), a.numel(), D_u, lam_u, b.data_ptr(), b.numel(), D_s,
                               lam_s, n_max, rel_tol, buf, 8 * n_max, _c.byref(cnt))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_layer_pairs")
    return [buf[i].as_dict() for i in range(cnt.value)]


class LayerSweep:
    """tms_layer_plan: the half-layer pairs of two full meshes searched as one
    batched search; hits carry the pair index and full-mesh triangle ids."""

    def __init__(self, A: "Mesh", B: "Mesh", pairs, stream=None):
        self.A, self.B, self.pairs = A, B, list(pairs)
        arr = (LayerPair * len(self.pairs))()
        for i, p in enumerate(self.pairs):
            arr[i] = LayerPair(p["n"], p["m"], p["sign_u"], p["sign_s"], p["a"][0], p["a"][1],
                               p["b"][0], p["b"][1])
        h = _c.c_void_p()
        rc = lib().tms_layer_plan_create(A.handle, B.handle, arr, len(self.pairs), _stream(stream),
                                         _c.byref(h))
        if rc != TMS_OK:
            raise TmsError(rc, "tms_layer_plan_create")
        self.handle = h

    def search(self, hit_capacity: int = 1 << 16, stream=None, out=None, offsets=None, **kw) -> "Hits":
        p = params(**kw)
        st = _stream(stream)
        dev = self.A.X.device
        buf = out if out is not None else _alloc_hits(hit_capacity, dev)
        offs = offsets if offsets is not None else torch.empty(len(self.pairs) + 1, dtype=torch.int64,
                                                              device=dev)
        n = _c.c_longlong(0)
        rc = lib().tms_layer_search(self.handle, _c.byref(p), buf.data_ptr(), buf.shape[0],
                                    offs.data_ptr(), _c.byref(n), st)
        if rc == TMS_ERR_CAPACITY and out is None and n.value > buf.shape[0]:
            buf = _alloc_hits(int(n.value), dev)
            rc = lib().tms_layer_search(self.handle, _c.byref(p), buf.data_ptr(), buf.shape[0],
                                        offs.data_ptr(), _c.byref(n), st)
        if rc != TMS_OK:
            raise TmsError(rc, "tms_layer_search")
        return Hits(buf[: n.value], offs)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.tms_layer_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def theta_translate(X: torch.Tensor, rho, derivative: bool = False, out=None, stream=None):
    """tms_theta_translate: each theta column of X (CUDA float64, (C, M, N) or
    (M, N), theta fastest) moved to theta + rho (Eq. translate) or, with
    `derivative`, its theta-derivative there (Eq. translate2).  rho: a float,
    or a CUDA float64 tensor of M per-column shifts.  Returns `out` (a new
    tensor unless given; may be X itself)."""
    if not (X.is_cuda and X.dtype == torch.float64 and X.is_contiguous() and X.dim() in (2, 3)):
        raise ValueError("X must be a contiguous CUDA float64 tensor (C, M, N) or (M, N)")
    C = 1 if X.dim() == 2 else int(X.shape[0])
    M, N = int(X.shape[-2]), int(X.shape[-1])
    out = torch.empty_like(X) if out is None else out
    if isinstance(rho, torch.Tensor):
        r = rho.to(device=X.device, dtype=torch.float64).contiguous()
        if r.numel() != M:
            raise ValueError("rho must hold one shift per column")
        rp, r0 = r.data_ptr(), 0.0
    else:
        r, rp, r0 = None, None, float(rho)
    rc = lib().tms_theta_translate(X.data_ptr(), out.data_ptr(), N, M, C, M * N, rp, r0,
                                   int(bool(derivative)), _stream(stream))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_theta_translate")
    return out


def phase_align(Wr: torch.Tensor, Wprev: torch.Tensor, stream=None):
    """tms_phase_align: the grid shift m minimising Eq. (rhoEquationDiscrete)
    for each pair of circles.  Wr, Wprev: CUDA float64 (A, C, N) or (C, N).
    Returns (shift int32 (A,), cost float64 (A, N))."""
    single = Wr.dim() == 2
    a, b = (Wr[None], Wprev[None]) if single else (Wr, Wprev)
    if a.shape != b.shape or not (a.is_cuda and a.dtype == torch.float64):
        raise ValueError("Wr and Wprev must be CUDA float64 tensors of one shape")
    a, b = a.contiguous(), b.contiguous()
    A, C, N = (int(v) for v in a.shape)
    cost = torch.empty((A, N), dtype=torch.float64, device=a.device)
    shift = torch.empty(A, dtype=torch.int32, device=a.device)
    rc = lib().tms_phase_align(a.data_ptr(), b.data_ptr(), N, C, A, cost.data_ptr(),
                               shift.data_ptr(), _stream(stream))
    if rc != TMS_OK:
        raise TmsError(rc, "tms_phase_align")
    return (shift[0], cost[0]) if single else (shift, cost)


def release_workspace(stream=None):
    lib().tms_release_workspace(_stream(stream) if stream is not None else None)


class HitPoint(torch.autograd.Function):
    """(P, z) of each hit as differentiable functions of the mesh vertices and,
    optionally, of a family parameter alpha on which both meshes depend.

    HitPoint.apply(XA, XB, meshA, meshB, hits[, alpha, dXA_dalpha, dXB_dalpha])
    returns the hit points P (n, 4) and barycentric pairs z = (a, b, c, d)
    (n, 4) found by the search; backward runs the library's FP64 adjoint
    (implicit differentiation of the 4x4 solve of Eq. (precise)) and returns
    vertex gradients shaped like XA and XB.  XA and XB must be the tensors the
    meshes were built from.  With alpha (a float64 tensor with one element) and
    dXA_dalpha, dXB_dalpha (CUDA float64, shaped like XA and XB: the vertices'
    derivatives in alpha; either may be None for a mesh that does not move),
    alpha's gradient is the sum over hits of the adjoint's per-hit alpha
    derivative, sum_v grad_v . dv/dalpha over each hit's six vertices.
    """

    @staticmethod
    def forward(ctx, XA, XB, meshA, meshB, hits, alpha=None, dXA_dalpha=None, dXB_dalpha=None):
        ctx.meshA, ctx.meshB, ctx.hits = meshA, meshB, hits
        ctx.alpha_shape = None if alpha is None else alpha.shape
        ctx.dA = None if dXA_dalpha is None else dXA_dalpha.to(torch.float64).contiguous()
        ctx.dB = None if dXB_dalpha is None else dXB_dalpha.to(torch.float64).contiguous()
        return hits.P.clone(), hits.z.clone()

    @staticmethod
    def backward(ctx, gP, gZ):
        A, B, hits = ctx.meshA, ctx.meshB, ctx.hits
        gA = torch.zeros_like(A.X)
        gB = torch.zeros_like(B.X)
        gP = None if gP is None else gP.to(torch.float64).contiguous()
        gZ = None if gZ is None else gZ.to(torch.float64).contiguous()
        want_alpha = ctx.alpha_shape is not None and ctx.needs_input_grad[5] and \
            (ctx.dA is not None or ctx.dB is not None)
        galpha = torch.zeros(len(hits), dtype=torch.float64, device=A.X.device) if want_alpha else None
        backward(A, B, hits, gP=gP, gZ=gZ, gradA=gA, gradB=gB,
                 dA_dalpha=ctx.dA if want_alpha else None,
                 dB_dalpha=ctx.dB if want_alpha else None, galpha=galpha)
        g_alpha = galpha.sum().reshape(ctx.alpha_shape) if want_alpha else None
        return gA, gB, None, None, None, g_alpha, None, None
