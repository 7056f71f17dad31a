"""CPU oracle for the mesh-vs-mesh intersection search -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package's smoke check and the benchmark's CPU-baseline leg
may import this package.  The CUDA search path never calls it, and it shares no
code with that path: the arithmetic lives in tms_oracle.c (plain C99, FP64,
compiled without fused multiply-add); this module only loads it, runs it over
mesh pairs and applies the post-processing rules written out below.

Post-processing (no counterpart in the paper, which stores every hit of every
triangle pair, Sec. 6.2.4 and Sec. 6.3):
  * merging of duplicate hits: a hit whose point lies on a shared edge or vertex
    of a mesh is found by every triangle pair incident to that feature.  Each
    side's feature is read off its barycentric weights (w1, w2, w3) =
    (a, 1-a-b, b) for (x1, x2, x3): no weight below tau -> the triangle itself;
    one weight below tau -> the edge joining the other two vertices; two ->
    the remaining vertex.  Hits with equal (feature A, feature B) are merged,
    keeping the smallest (triA, triB);
  * output order: sorted by (triA, triB).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tms_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_tms.so")
_lock = threading.Lock()
_lib = None

TAU = 1e-12
BAND = 1e-12

REC_DTYPE = np.dtype([
    ("triA", np.int64), ("triB", np.int64),
    ("z", np.float64, 4), ("P", np.float64, 4), ("params", np.float64, 4),
    ("rho", np.float64), ("margin", np.float64), ("det", np.float64), ("gap", np.float64),
    ("hit", np.int32), ("singular", np.int32),
])


def build(force: bool = False) -> str:
    """Compile tms_oracle.c with gcc (FP64, no FMA contraction, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    assert lib.oracle_sizeof_rec() == REC_DTYPE.itemsize, "record layout mismatch"
    P = ctypes.c_void_p
    I = ctypes.c_int
    L = ctypes.c_longlong
    D = ctypes.c_double
    mesh = [P, P, I, I, I]
    lib.oracle_bruteforce.argtypes = mesh + mesh + [D, P, L]
    lib.oracle_bruteforce.restype = L
    lib.oracle_pruned.argtypes = mesh + mesh + [D, P, L, P]
    lib.oracle_pruned.restype = L
    lib.oracle_hits_for_A.argtypes = mesh + mesh + [P, L, D, P, L]
    lib.oracle_hits_for_A.restype = L
    lib.oracle_box_pairs.argtypes = mesh + mesh + [P, L]
    lib.oracle_box_pairs.restype = L
    lib.oracle_eval_pairs.argtypes = mesh + mesh + [P, P, L, D, P]
    lib.oracle_eval_pairs.restype = None
    lib.oracle_tri_coords.argtypes = mesh + [P, L, P]
    lib.oracle_tri_coords.restype = None
    lib.oracle_tri_pair.argtypes = [P, P, D, P]
    lib.oracle_tri_pair.restype = None
    lib.oracle_solve4_flat.argtypes = [P, P, P, P]
    lib.oracle_solve4_flat.restype = I
    lib.oracle_pair_grad.argtypes = [P, P, P, P, P, P, P]
    lib.oracle_pair_grad.restype = I
    _lib = lib
    return lib


class OMesh:
    """A mesh as the oracle sees it: contiguous float64 numpy arrays."""

    def __init__(self, X, s, periodic: bool = True):
        self.X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
        self.s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
        assert self.X.ndim == 3 and self.X.shape[0] == 4
        self.M, self.N = int(self.X.shape[1]), int(self.X.shape[2])
        assert self.s.shape == (self.M,)
        self.periodic = bool(periodic)

    @classmethod
    def from_grid(cls, g):
        """From a synth.MeshGrid (torch tensors, any device)."""
        return cls(g.X.detach().cpu().numpy(), g.s.detach().cpu().numpy(), g.periodic)

    def args(self):
        return [self.X.ctypes.data, self.s.ctypes.data, self.N, self.M, int(self.periodic)]

    @property
    def n_tri_ids(self):
        return 2 * self.N * (self.M - 1)

    def tri_valid(self, t):
        t = np.asarray(t)
        i = (t // 2) % self.N
        ok = (t >= 0) & (t < self.n_tri_ids)
        return ok if self.periodic else ok & (i < self.N - 1)


def _run_collect(fn, est: int):
    cap = max(int(est), 1024)
    while True:
        out = np.zeros(cap, dtype=REC_DTYPE)
        n = fn(out, cap)
        if n <= cap:
            return out[:n]
        cap = int(n)


def bruteforce(A: OMesh, B: OMesh, tau: float = TAU) -> np.ndarray:
    """All-pairs narrow-phase test; raw hit records (unsorted, unmerged)."""
    lib = _load()
    return _run_collect(lambda out, cap: lib.oracle_bruteforce(
        *A.args(), *B.args(), tau, out.ctypes.data, cap), 4096)


def pruned(A: OMesh, B: OMesh, tau: float = TAU, return_overlaps: bool = False):
    """Exact pruning by closed box overlap (bounding-volume hierarchy over B),
    then the same narrow-phase test; raw hits."""
    lib = _load()
    nov = ctypes.c_longlong(0)
    recs = _run_collect(lambda out, cap: lib.oracle_pruned(
        *A.args(), *B.args(), tau, out.ctypes.data, cap, ctypes.byref(nov)), 1 << 16)
    return (recs, int(nov.value)) if return_overlaps else recs


def hits_for_A(A: OMesh, B: OMesh, trisA, tau: float = TAU) -> np.ndarray:
    lib = _load()
    trisA = np.ascontiguousarray(np.asarray(trisA, dtype=np.int64))
    return _run_collect(lambda out, cap: lib.oracle_hits_for_A(
        *A.args(), *B.args(), trisA.ctypes.data, trisA.size, tau, out.ctypes.data, cap), 4096)


def box_pairs(A: OMesh, B: OMesh) -> np.ndarray:
    """(n, 2) int64 array of triangle pairs whose closed boxes overlap."""
    lib = _load()
    cap = 1 << 16
    while True:
        pairs = np.zeros((cap, 2), dtype=np.int64)
        n = lib.oracle_box_pairs(*A.args(), *B.args(), pairs.ctypes.data, cap)
        if n <= cap:
            return pairs[:n]
        cap = int(n)


def eval_pairs(A: OMesh, B: OMesh, triA, triB, tau: float = TAU) -> np.ndarray:
    lib = _load()
    ta = np.ascontiguousarray(np.asarray(triA, dtype=np.int64))
    tb = np.ascontiguousarray(np.asarray(triB, dtype=np.int64))
    out = np.zeros(ta.size, dtype=REC_DTYPE)
    lib.oracle_eval_pairs(*A.args(), *B.args(), ta.ctypes.data, tb.ctypes.data, ta.size, tau,
                          out.ctypes.data)
    return out


def tri_coords(m: OMesh, tris) -> np.ndarray:
    """(n, 3, 4) vertex coordinates (x1, x2, x3) of the given triangles."""
    lib = _load()
    t = np.ascontiguousarray(np.asarray(tris, dtype=np.int64))
    out = np.zeros((t.size, 3, 4), dtype=np.float64)
    lib.oracle_tri_coords(*m.args(), t.ctypes.data, t.size, out.ctypes.data)
    return out


def tri_pair(x, y, tau: float = TAU) -> np.ndarray:
    """Narrow-phase record for explicit triangles x (3, 4) and y (3, 4)."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(12))
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(12))
    out = np.zeros(1, dtype=REC_DTYPE)
    lib.oracle_tri_pair(x.ctypes.data, y.ctypes.data, tau, out.ctypes.data)
    return out[0]


def solve4(A, r):
    """Gaussian elimination with partial pivoting: (z, det, ok)."""
    lib = _load()
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(16))
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(4))
    z = np.zeros(4)
    det = ctypes.c_double(0.0)
    ok = lib.oracle_solve4_flat(A.ctypes.data, r.ctypes.data, z.ctypes.data, ctypes.byref(det))
    return z, det.value, bool(ok)


def pair_grad(x, y, gP, gz):
    """Vertex gradients (gx (3, 4), gy (3, 4)) of one triangle pair and its z."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(12))
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(12))
    gP = np.ascontiguousarray(np.asarray(gP, dtype=np.float64).reshape(4))
    gz = np.ascontiguousarray(np.asarray(gz, dtype=np.float64).reshape(4))
    gx = np.zeros(12)
    gy = np.zeros(12)
    z = np.zeros(4)
    ok = lib.oracle_pair_grad(x.ctypes.data, y.ctypes.data, gP.ctypes.data, gz.ctypes.data,
                              gx.ctypes.data, gy.ctypes.data, z.ctypes.data)
    if not ok:
        raise ValueError("singular system")
    return gx.reshape(3, 4), gy.reshape(3, 4), z


# ----------------------------------------------------------------------------
# merging of duplicate hits and output order
# ----------------------------------------------------------------------------

def tri_vertex_ids(m: OMesh, t: int):
    """Vertex ids (k*N + i) of (x1, x2, x3) of triangle t (Sec. 6.2.4 orderings)."""
    q, tau = divmod(int(t), 2)
    k, i = divmod(q, m.N)
    ip = (i + 1) % m.N
    if tau == 0:
        ij = [(ip, k), (i, k), (i, k + 1)]
    else:
        ij = [(i, k + 1), (ip, k + 1), (ip, k)]
    return [kk * m.N + ii for (ii, kk) in ij]


def feature(m: OMesh, t: int, u: float, v: float, tau: float = TAU):
    """Feature of the hit point with weights (u, v) in triangle t (see module doc)."""
    w = [u, 1.0 - u - v, v]
    vid = tri_vertex_ids(m, t)
    small = [abs(x) < tau for x in w]
    ns = sum(small)
    if ns == 0:
        return ("T", int(t))
    if ns == 1:
        j = small.index(True)
        e = [vid[k] for k in range(3) if k != j]
        return ("E", min(e), max(e))
    if ns == 2:
        j = small.index(False)
        return ("V", vid[j])
    j = int(np.argmax(w))
    return ("V", vid[j])


def merge_and_sort(A: OMesh, B: OMesh, recs: np.ndarray, tau: float = TAU) -> np.ndarray:
    """Merge duplicate hits by (feature A, feature B), keep the smallest
    (triA, triB) of each group, return sorted by (triA, triB)."""
    if recs.size == 0:
        return recs
    order = np.lexsort((recs["triB"], recs["triA"]))
    recs = recs[order]
    seen = set()
    keep = np.zeros(recs.size, dtype=bool)
    for h in range(recs.size):
        r = recs[h]
        fa = feature(A, int(r["triA"]), float(r["z"][0]), float(r["z"][1]), tau)
        fb = feature(B, int(r["triB"]), float(r["z"][2]), float(r["z"][3]), tau)
        key = (fa, fb)
        if key in seen:
            continue
        seen.add(key)
        keep[h] = True
    return recs[keep]


def search(A: OMesh, B: OMesh, tau: float = TAU, method: str = "auto") -> np.ndarray:
    """The oracle's answer: merged, sorted hit records of mesh A against mesh B."""
    if method == "auto":
        method = "brute" if A.n_tri_ids * B.n_tri_ids <= 2e7 else "pruned"
    raw = bruteforce(A, B, tau) if method == "brute" else pruned(A, B, tau)
    return merge_and_sort(A, B, raw, tau)


def in_band(recs: np.ndarray, band: float = BAND) -> np.ndarray:
    """Near-degenerate pairs: rho < band or |margin| < band (or singular)."""
    return (recs["singular"] != 0) | (recs["rho"] < band) | (np.abs(recs["margin"]) < band)


# ----------------------------------------------------------------------------
# gradients of hits
# ----------------------------------------------------------------------------

def hit_grads(A: OMesh, B: OMesh, triA, triB, gP, gz, dA_dalpha=None, dB_dalpha=None):
    """Dense vertex gradients (4, M, N) for both meshes, accumulated over hits,
    and the per-hit alpha derivative when dX/dalpha is given."""
    triA = np.asarray(triA, dtype=np.int64)
    triB = np.asarray(triB, dtype=np.int64)
    gP = np.asarray(gP, dtype=np.float64).reshape(-1, 4)
    gz = np.asarray(gz, dtype=np.float64).reshape(-1, 4)
    GA = np.zeros_like(A.X)
    GB = np.zeros_like(B.X)
    galpha = np.zeros(triA.size)
    xs = tri_coords(A, triA)
    ys = tri_coords(B, triB)
    for h in range(triA.size):
        gx, gy, _ = pair_grad(xs[h], ys[h], gP[h], gz[h])
        va = tri_vertex_ids(A, int(triA[h]))
        vb = tri_vertex_ids(B, int(triB[h]))
        acc = 0.0
        for j in range(3):
            ka, ia = divmod(va[j], A.N)
            kb, ib = divmod(vb[j], B.N)
            GA[:, ka, ia] += gx[j]
            GB[:, kb, ib] += gy[j]
            if dA_dalpha is not None:
                acc += float(np.dot(gx[j], dA_dalpha[:, ka, ia]))
            if dB_dalpha is not None:
                acc += float(np.dot(gy[j], dB_dalpha[:, kb, ib]))
        galpha[h] = acc
    return GA, GB, galpha
