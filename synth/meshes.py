"""Seeded synthetic manifold-mesh pairs for the mesh-vs-mesh intersection search.

This module is the one input source shared by the CPU oracle and the CUDA path.
It builds vertex grids and planted intersection records; it contains none of the
search method's arithmetic (no bounding boxes, no grid cells, no 4x4 solve, no
margin test).  A planted record is built geometrically: a point is placed at
chosen barycentric weights inside a chosen triangle of mesh A, and the matching
triangle of mesh B is translated rigidly so that it contains that same point at
chosen weights.  The recorded (a, b, c, d), point P and (theta, s) parameters are
therefore known in closed form, independent of any solver.

Mesh storage follows the paper's vertex-grid layout (Sec. 6.1 and Sec. 6.3):
four N x M coordinate arrays x, y, px, py, theta fastest, here one float64
tensor X of shape (4, M, N) with X[c, k, i] = coordinate c of W(theta_i, s_k),
theta_i = 2*pi*i/N.  Quads are Q_ik for i in [0, N) (periodic in theta) and
k in [0, M-1); quad id q = k*N + i and triangle id t = 2*q + tau (tau = 0 for
T1, tau = 1 for T2), with the vertex orderings of Sec. 6.2.4:
  T1: x1 = W(i+1, k), x2 = W(i, k),   x3 = W(i, k+1)
  T2: x1 = W(i, k+1), x2 = W(i+1, k+1), x3 = W(i+1, k)

Surface family (stand-ins for the unstable/stable manifold half-layers, whose
Jupiter-Europa data are not available):
  A(theta, s; alpha) = g(s) * T(theta; alpha) + F(s)
      T  = sum_{k=1..6} (a_k(alpha) cos k theta + b_k(alpha) sin k theta) / k,
           a_k(alpha) = a_k + alpha a'_k, all coefficients N(0, I_4)
      g  = 1 + s (plain) or lambda**s (manifold-like stretching, lambda = 4)
      F  = sum over folds of amp * (s - r1)(s - r2)(s - r3) * e_f  (roots in (0,1))
  B(theta, s; alpha) = A(theta + c0, 1 - s; alpha) + H(theta, s)
      (reversed s gives the stable-manifold stretch lambda**(1-s))
      H  = h_amp * (sin(P (theta - theta0)) n1 + sin(Q pi (s - s0)) n2)
      with (n1, n2) an orthonormal normal frame of A (frozen at alpha_ref).
The two sheets cross transversally where H vanishes: a lattice of 2P x Q
"sites".  Planted hits and planted near-misses are placed at sites.
Both meshes are affine in alpha, so dX/dalpha is exact and returned.
"""
from __future__ import annotations

import math
from bisect import bisect_right
from dataclasses import dataclass, field
from typing import Optional

import torch

SEED_BASE = 210914814
TWO_PI = 2.0 * math.pi


@dataclass
class MeshGrid:
    """One manifold half-layer mesh: X (4, M, N) float64, s (M,) float64."""
    X: torch.Tensor
    s: torch.Tensor
    periodic: bool = True
    dXdalpha: Optional[torch.Tensor] = None

    @property
    def N(self) -> int:
        return int(self.X.shape[2])

    @property
    def M(self) -> int:
        return int(self.X.shape[1])

    @property
    def n_quads(self) -> int:
        return (self.N if self.periodic else self.N - 1) * (self.M - 1)

    @property
    def n_tri_ids(self) -> int:
        """Size of the triangle id space 2*N*(M-1) (open strips leave gaps)."""
        return 2 * self.N * (self.M - 1)

    def to(self, device) -> "MeshGrid":
        return MeshGrid(self.X.to(device), self.s.to(device), self.periodic,
                        None if self.dXdalpha is None else self.dXdalpha.to(device))


@dataclass
class Planted:
    """Planted records (all tensors length n, CPU).

    kind: 0 = planted hit (interior in both triangles, every weight >= 0.1),
          1 = planted near-miss (B weight c = -eta, so the planes meet outside
              triangle B at nominal distance `dist`).
    """
    kind: torch.Tensor
    triA: torch.Tensor
    triB: torch.Tensor
    abcd: torch.Tensor       # (n, 4) float64
    P: torch.Tensor          # (n, 4) float64 planted point
    params: torch.Tensor     # (n, 4) float64 (theta_u, s_u, theta_s, s_s)
    dist: torch.Tensor       # (n,) float64 nominal distance (0 for hits)

    def __len__(self):
        return int(self.kind.numel())

    def select(self, mask) -> "Planted":
        return Planted(*(getattr(self, f)[mask] for f in
                         ("kind", "triA", "triB", "abcd", "P", "params", "dist")))


@dataclass
class SurfacePair:
    """Closed form of the two analytic sheets a mesh pair samples (planted
    corrections excluded), for refinement on the true surfaces:

      W_A(theta, s) = g(s) T(theta; alpha) + F(s)
      W_B(theta, s) = W_A(theta + c0, 1 - s) + h_amp (sin(P (theta - theta0)) n1
                                                    + sin(Q pi (s - s0)) n2)
      T(theta; alpha) = sum_k ((ca_k + alpha dca_k) cos k theta
                               + (cb_k + alpha dcb_k) sin k theta) / k
      g = 1 + s ("linear") or lam**s ("exp");  F = sum_f amp_f prod_j (s - r_fj) e_f
      (n1, n2)(theta, s): v1, v2 minus their regularised least-squares projection
        on span(t1, t2), t1, t2 = the theta- and s-partials of the underlying
        sheet g(s') T(theta'; alpha_ref) + F(s') at theta' = theta + c0,
        s' = 1 - s; regulariser eps = reg (|t1|^2 + |t2|^2) / 2.
    sites: (n, 2) lattice points (theta, s) of B where both sines vanish; each
    is an exact crossing of the sheets at (theta + c0, 1 - s, theta, s)."""
    ca: torch.Tensor
    cb: torch.Tensor
    dca: torch.Tensor
    dcb: torch.Tensor
    alpha: float
    alpha_ref: float
    stretch: str
    lam: float
    fold_amp: torch.Tensor
    fold_roots: torch.Tensor
    fold_dir: torch.Tensor
    c0: float
    h_amp: float
    P: float
    Q: float
    theta0: float
    s0: float
    v1: torch.Tensor
    v2: torch.Tensor
    reg: float
    sites: torch.Tensor


@dataclass
class MeshPair:
    A: MeshGrid
    B: MeshGrid
    planted: Planted
    meta: dict = field(default_factory=dict)
    surface: Optional[SurfacePair] = None


# ----------------------------------------------------------------------------
# surface family
# ----------------------------------------------------------------------------

@dataclass
class _Family:
    ca: torch.Tensor      # (K, 4)
    cb: torch.Tensor
    dca: torch.Tensor     # alpha-derivative coefficients
    dcb: torch.Tensor
    stretch: str          # "linear" or "exp"
    lam: float
    fold_amp: torch.Tensor    # (F,)
    fold_roots: torch.Tensor  # (F, 3)
    fold_dir: torch.Tensor    # (F, 4)


def _make_family(gen: torch.Generator, stretch: str, lam: float, n_folds: int,
                 fold_scale: float) -> _Family:
    K = 6
    ca = torch.randn(K, 4, generator=gen, dtype=torch.float64)
    cb = torch.randn(K, 4, generator=gen, dtype=torch.float64)
    dca = torch.randn(K, 4, generator=gen, dtype=torch.float64) * 0.25
    dcb = torch.randn(K, 4, generator=gen, dtype=torch.float64) * 0.25
    roots = torch.rand(n_folds, 3, generator=gen, dtype=torch.float64) * 0.8 + 0.1
    d = torch.randn(n_folds, 4, generator=gen, dtype=torch.float64)
    d = d / d.norm(dim=1, keepdim=True).clamp_min(1e-12)
    amp = (torch.rand(n_folds, generator=gen, dtype=torch.float64) * 0.5 + 0.75) * fold_scale
    return _Family(ca, cb, dca, dcb, stretch, lam, amp, roots, d)


def _trig(fam: _Family, theta: torch.Tensor, alpha: float):
    """T(theta), dT/dtheta, dT/dalpha as (4, n) tensors."""
    dev = theta.device
    K = fam.ca.shape[0]
    k = torch.arange(1, K + 1, dtype=torch.float64, device=dev)
    kt = k[:, None] * theta[None, :]
    c, s = torch.cos(kt), torch.sin(kt)
    ca = (fam.ca + alpha * fam.dca).to(dev)
    cb = (fam.cb + alpha * fam.dcb).to(dev)
    T = (ca / k[:, None]).T @ c + (cb / k[:, None]).T @ s
    dT = -ca.T @ s + cb.T @ c
    Ta = (fam.dca.to(dev) / k[:, None]).T @ c + (fam.dcb.to(dev) / k[:, None]).T @ s
    return T, dT, Ta


def _g(fam: _Family, s: torch.Tensor):
    if fam.stretch == "linear":
        return 1.0 + s, torch.ones_like(s)
    ln = math.log(fam.lam)
    g = torch.exp(ln * s)
    return g, ln * g


def _folds(fam: _Family, s: torch.Tensor):
    """F(s), F'(s) as (4, m) tensors."""
    dev = s.device
    F = torch.zeros(4, s.numel(), dtype=torch.float64, device=dev)
    dF = torch.zeros_like(F)
    for f in range(fam.fold_amp.numel()):
        r = fam.fold_roots[f].tolist()
        p = (s - r[0]) * (s - r[1]) * (s - r[2])
        dp = (s - r[1]) * (s - r[2]) + (s - r[0]) * (s - r[2]) + (s - r[0]) * (s - r[1])
        e = fam.fold_dir[f].to(dev)[:, None]
        F += float(fam.fold_amp[f]) * p[None, :] * e
        dF += float(fam.fold_amp[f]) * dp[None, :] * e
    return F, dF


def _surface_A(fam, theta, s, alpha):
    """A on the tensor grid theta (n,), s (m,): value, d/dtheta, d/ds, d/dalpha (4, m, n)."""
    T, dT, Ta = _trig(fam, theta, alpha)
    g, dg = _g(fam, s)
    F, dF = _folds(fam, s)
    X = g[None, :, None] * T[:, None, :] + F[:, :, None]
    Xt = g[None, :, None] * dT[:, None, :]
    Xs = dg[None, :, None] * T[:, None, :] + dF[:, :, None]
    Xa = g[None, :, None] * Ta[:, None, :]
    return X, Xt, Xs, Xa


def _normal_frame(Xt, Xs, gen_dirs, reg: float = 0.25):
    """Smooth normal fields (n1, n2): the fixed directions gen_dirs with their
    component along the tangent plane span(Xt, Xs) removed by a regularised
    least-squares projection v - J (J^T J + eps I)^{-1} J^T v, J = [Xt, Xs],
    eps = reg * trace(J^T J) / 2.  The regularisation keeps the fields smooth
    where the tangent plane is nearly degenerate (folds)."""
    g11 = (Xt * Xt).sum(0)
    g12 = (Xt * Xs).sum(0)
    g22 = (Xs * Xs).sum(0)
    eps = reg * 0.5 * (g11 + g22)
    a, b, c = g11 + eps, g12, g22 + eps
    det = a * c - b * b
    out = []
    for r in gen_dirs:
        v = r.to(Xt.device).view(4, 1, 1)
        jt1 = (Xt * v).sum(0)
        jt2 = (Xs * v).sum(0)
        y1 = (c * jt1 - b * jt2) / det
        y2 = (-b * jt1 + a * jt2) / det
        out.append(v - Xt * y1 - Xs * y2)
    return out[0], out[1]


# ----------------------------------------------------------------------------
# mesh index helpers (generator-side: vertex lists of triangles)
# ----------------------------------------------------------------------------

def tri_vertex_ij(N: int, t: int):
    """(i, k) grid indices of (x1, x2, x3) of triangle t, Sec. 6.2.4 orderings."""
    q, tau = divmod(t, 2)
    k, i = divmod(q, N)
    ip = (i + 1) % N
    if tau == 0:
        return [(ip, k), (i, k), (i, k + 1)]
    return [(i, k + 1), (ip, k + 1), (ip, k)]


def _locate(theta, s_val, N, s_grid):
    """Triangle id and cell fractions of parameter point (theta, s) on a grid."""
    dth = TWO_PI / N
    th = theta % TWO_PI
    i = int(math.floor(th / dth)) % N
    ft = th / dth - math.floor(th / dth)
    sg = s_grid
    k = min(max(bisect_right(sg, s_val) - 1, 0), len(sg) - 2)
    fs = (s_val - sg[k]) / (sg[k + 1] - sg[k])
    fs = min(max(fs, 0.0), 1.0)
    tau = 0 if ft + fs <= 1.0 else 1
    return i, k, tau, ft, fs


def _to_weights(tau, ft, fs):
    """Barycentric (a, b) of the point at cell fractions (ft, fs) in T1 or T2."""
    return (ft, fs) if tau == 0 else (1.0 - ft, 1.0 - fs)


def _shrink(a, b, m):
    """Move (a, b) toward the centroid until a, b, 1-a-b are all >= m."""
    w = [a, b, 1.0 - a - b]
    t = 0.0
    for wi in w:
        if wi < m:
            t = max(t, (m - wi) / (1.0 / 3.0 - wi))
    t = min(t, 1.0)
    a2 = (1 - t) * a + t / 3.0
    b2 = (1 - t) * b + t / 3.0
    return a2, b2


def _point_params(N, s_grid, t, a, b):
    """Parameter (theta, s) of the point with weights (a, b) in triangle t:
    the weighted average of the vertex parameters (weights a, 1-a-b, b for
    x1, x2, x3), with theta taken unwrapped across the seam."""
    verts = tri_vertex_ij(N, t)
    q, _ = divmod(t, 2)
    i0 = q % N
    w = [a, 1.0 - a - b, b]
    th = 0.0
    sv = 0.0
    dth = TWO_PI / N
    for (vi, vk), wv in zip(verts, w):
        rel = (vi - i0) % N          # 0 or 1 (unwrapped neighbour)
        th += wv * (i0 + rel) * dth
        sv += wv * float(s_grid[vk])
    return th % TWO_PI, sv


# ----------------------------------------------------------------------------
# pair builder
# ----------------------------------------------------------------------------

def _plane_transversality(xv, yv) -> float:
    """Product of the sines of the two principal angles between the planes of
    triangle (x1, x2, x3) and triangle (y1, y2, y3): 0 when the planes share a
    direction, 1 when they are orthogonal."""
    QA, _ = torch.linalg.qr(torch.stack([xv[0] - xv[1], xv[2] - xv[1]], dim=1))
    QB, _ = torch.linalg.qr(torch.stack([yv[0] - yv[1], yv[2] - yv[1]], dim=1))
    cosines = torch.linalg.svdvals(QA.T @ QB).clamp(max=1.0)
    return float(torch.sqrt(1.0 - cosines ** 2).prod())


def _bump_weights(T: int):
    return [1.0] + [0.5 * (1.0 + math.cos(math.pi * d / (T + 1))) for d in range(1, T + 1)]


def build_pair(seed: int, NA: int, MA: int, NB: int, MB: int, *, stretch: str = "exp",
               lam: float = 4.0, n_folds: int = 3, fold_scale: float = 12.0,
               sites: tuple = (8, 4), n_hits: int = 64, n_near: int = 0,
               near_range: tuple = (1e-9, 1e-3), alpha: float = 0.0,
               alpha_ref: float = 0.5, with_dalpha: bool = False,
               h_scale: float = 1.0, device: str = "cpu",
               family_seed: Optional[int] = None,
               min_transversality: float = 0.01) -> MeshPair:
    """Build one seeded mesh pair.

    sites = (2P, Q): number of sign changes of the H lattice in theta and s.
    n_hits planted hits and n_near planted near-misses are placed at distinct
    sites (hits first); remaining sites are left as natural crossings.
    family_seed fixes the surface coefficients across a batch (alpha family);
    seed drives everything else.
    """
    gen = torch.Generator().manual_seed(seed)
    fgen = torch.Generator().manual_seed(seed if family_seed is None else family_seed)
    fam = _make_family(fgen, stretch, lam, n_folds, fold_scale)
    dirs = torch.randn(2, 4, generator=fgen, dtype=torch.float64)
    dirs = dirs / dirs.norm(dim=1, keepdim=True)
    c0 = float(torch.rand(1, generator=fgen, dtype=torch.float64)) * TWO_PI
    dev = torch.device(device)

    thA = torch.arange(NA, dtype=torch.float64, device=dev) * (TWO_PI / NA)
    sA = torch.linspace(0.0, 1.0, MA, dtype=torch.float64, device=dev)
    thB = torch.arange(NB, dtype=torch.float64, device=dev) * (TWO_PI / NB)
    sB = torch.linspace(0.0, 1.0, MB, dtype=torch.float64, device=dev)

    XA, _, _, XAa = _surface_A(fam, thA, sA, alpha)
    # B's underlying A-surface at (theta + c0, 1 - s)
    XB0, _, _, XBa = _surface_A(fam, thB + c0, 1.0 - sB, alpha)
    # H is frozen at alpha_ref so that both meshes stay affine in alpha
    _, XAt, XAs, _ = _surface_A(fam, thA, sA, alpha_ref)
    _, XBt, XBs, _ = _surface_A(fam, thB + c0, 1.0 - sB, alpha_ref)

    # H lattice amplitude from the typical mesh spacing of A
    n_th, n_s = sites
    P = n_th / 2.0
    Q = n_s
    w_th = (XAt.norm(dim=0).mean() * (TWO_PI / NA)).item()
    w_s = (XAs.norm(dim=0).mean() / max(MA - 1, 1)).item()
    w_typ = max(w_th, w_s)
    L_th = NB / n_th
    L_s = (MB - 1) / max(Q, 1)
    h_amp = h_scale * w_typ * min(L_th, L_s) / math.pi
    th0 = float(torch.rand(1, generator=fgen, dtype=torch.float64)) * (math.pi / max(P, 0.5)) * 0.5 \
        + 0.25 * (TWO_PI / NB)
    s0 = (0.5 + float(torch.rand(1, generator=fgen, dtype=torch.float64)) * 0.5) / max(Q, 1)
    n1, n2 = _normal_frame(XBt, XBs, [dirs[0], dirs[1]])
    u1 = torch.sin(P * (thB - th0))
    u2 = torch.sin(Q * math.pi * (sB - s0))
    H = h_amp * (u1[None, None, :] * n1 + u2[None, :, None] * n2)
    XB = XB0 + H
    dXB = XBa.clone()

    # lattice sites in B's parameter space
    site_th = [(th0 + m * math.pi / P) % TWO_PI for m in range(int(round(2 * P)))]
    site_s = [s0 + n / Q for n in range(int(Q) + 1) if 0.0 < s0 + n / Q < 1.0]
    site_list = [(a, b) for b in site_s for a in site_th]
    perm = torch.randperm(len(site_list), generator=fgen).tolist()
    site_list = [site_list[p] for p in perm]

    rec = dict(kind=[], triA=[], triB=[], abcd=[], P=[], params=[], dist=[])
    T_taper = 2
    wts = _bump_weights(T_taper)
    usedB = torch.zeros(MB, NB, dtype=torch.bool)
    XA_cpu = XA.cpu()
    XB_cpu = XB.cpu()
    # planting decisions (transversality) are taken on the alpha_ref surfaces in a
    # family, so that every member of the family plants the same sites
    if with_dalpha and alpha != alpha_ref:
        XA_dec = _surface_A(fam, thA, sA, alpha_ref)[0].cpu()
        XB_dec = (_surface_A(fam, thB + c0, 1.0 - sB, alpha_ref)[0] + H).cpu()
    else:
        XA_dec, XB_dec = XA_cpu, XB_cpu
    dXA_cpu = XAa.cpu()
    dXB_cpu = dXB.cpu()
    corr = torch.zeros(4, MB, NB, dtype=torch.float64)
    dcorr = torch.zeros(4, MB, NB, dtype=torch.float64)
    lo_near, hi_near = math.log(near_range[0]), math.log(near_range[1])
    sA_list = sA.cpu().tolist()
    sB_list = sB.cpu().tolist()
    want = [0] * n_hits + [1] * n_near
    for (sth, ss) in site_list:
        if not want:
            break
        kind = want[0]
        # A parameter of the site, and the triangle of A containing it
        ia, ka, taua, fta, fsa = _locate(sth + c0, 1.0 - ss, NA, sA_list)
        a, b = _to_weights(taua, fta, fsa)
        a, b = _shrink(a, b, 0.1)
        triA = 2 * (ka * NA + ia) + taua
        # B triangle containing the site
        ib, kb, taub, ftb, fsb = _locate(sth, ss, NB, sB_list)
        if kb + 1 >= MB:
            continue
        c, d = _to_weights(taub, ftb, fsb)
        c, d = _shrink(c, d, 0.1)
        dist = 0.0
        triB = 2 * (kb * NB + ib) + taub
        vb = tri_vertex_ij(NB, triB)
        yv = [XB_cpu[:, vk, vi] for (vi, vk) in vb]
        if kind == 1:
            dist = math.exp(lo_near + (hi_near - lo_near) *
                            float(torch.rand(1, generator=gen, dtype=torch.float64)))
            eta = dist / float((yv[0] - yv[1]).norm())
            c, d = -eta, min(max(d, 0.2), 0.7)
        va = tri_vertex_ij(NA, triA)
        xv = [XA_cpu[:, vk, vi] for (vi, vk) in va]
        if _plane_transversality([XA_dec[:, vk, vi] for (vi, vk) in va],
                                 [XB_dec[:, vk, vi] for (vi, vk) in vb]) < min_transversality:
            continue
        # disjoint supports on B
        rows = [kb + dk for dk in range(-T_taper, 2 + T_taper) if 0 <= kb + dk < MB]
        cols = [(ib + di) % NB for di in range(-T_taper, 2 + T_taper)]
        if usedB[rows][:, cols].any():
            continue
        for r in rows:
            usedB[r, cols] = True
        # planted point on A: weights (a, 1-a-b, b) on (x1, x2, x3)
        wA = [a, 1.0 - a - b, b]
        p = wA[0] * xv[0] + wA[1] * xv[1] + wA[2] * xv[2]
        wB = [c, 1.0 - c - d, d]
        qpt = wB[0] * yv[0] + wB[1] * yv[1] + wB[2] * yv[2]
        delta = p - qpt
        dxv = [dXA_cpu[:, vk, vi] for (vi, vk) in va]
        dyv = [dXB_cpu[:, vk, vi] for (vi, vk) in vb]
        ddelta = (wA[0] * dxv[0] + wA[1] * dxv[1] + wA[2] * dxv[2]) \
            - (wB[0] * dyv[0] + wB[1] * dyv[1] + wB[2] * dyv[2])
        for dk in range(-T_taper, 2 + T_taper):
            r = kb + dk
            if not (0 <= r < MB):
                continue
            wk = wts[0] if dk in (0, 1) else wts[(-dk) if dk < 0 else dk - 1]
            for di in range(-T_taper, 2 + T_taper):
                col = (ib + di) % NB
                wi = wts[0] if di in (0, 1) else wts[(-di) if di < 0 else di - 1]
                corr[:, r, col] += (wk * wi) * delta
                dcorr[:, r, col] += (wk * wi) * ddelta
        thu, su = _point_params(NA, sA_list, triA, a, b)
        ths, sss = _point_params(NB, sB_list, triB, c, d)
        rec["kind"].append(kind)
        rec["triA"].append(triA)
        rec["triB"].append(triB)
        rec["abcd"].append([a, b, c, d])
        rec["P"].append(p.tolist())
        rec["params"].append([thu, su, ths, sss])
        rec["dist"].append(dist)
        want.pop(0)

    XB = XB + corr.to(dev)
    dXB = dXB + dcorr.to(dev)
    planted = Planted(
        kind=torch.tensor(rec["kind"], dtype=torch.int32),
        triA=torch.tensor(rec["triA"], dtype=torch.int64),
        triB=torch.tensor(rec["triB"], dtype=torch.int64),
        abcd=torch.tensor(rec["abcd"], dtype=torch.float64).reshape(-1, 4),
        P=torch.tensor(rec["P"], dtype=torch.float64).reshape(-1, 4),
        params=torch.tensor(rec["params"], dtype=torch.float64).reshape(-1, 4),
        dist=torch.tensor(rec["dist"], dtype=torch.float64),
    )
    A = MeshGrid(XA.contiguous(), sA.contiguous(), True,
                 XAa.contiguous() if with_dalpha else None)
    B = MeshGrid(XB.contiguous(), sB.contiguous(), True,
                 dXB.contiguous() if with_dalpha else None)
    meta = dict(seed=seed, NA=NA, MA=MA, NB=NB, MB=MB, alpha=alpha, h_amp=h_amp,
                sites=len(site_list), stretch=stretch)
    surface = SurfacePair(
        ca=fam.ca.clone(), cb=fam.cb.clone(), dca=fam.dca.clone(), dcb=fam.dcb.clone(),
        alpha=float(alpha), alpha_ref=float(alpha_ref), stretch=stretch, lam=float(lam),
        fold_amp=fam.fold_amp.clone(), fold_roots=fam.fold_roots.clone(),
        fold_dir=fam.fold_dir.clone(), c0=c0, h_amp=float(h_amp), P=float(P), Q=float(Q),
        theta0=th0, s0=s0, v1=dirs[0].clone(), v2=dirs[1].clone(), reg=0.25,
        sites=torch.tensor(sorted(site_list), dtype=torch.float64).reshape(-1, 2))
    return MeshPair(A, B, planted, meta, surface)


# ----------------------------------------------------------------------------
# the five configurations
# ----------------------------------------------------------------------------

def independent_pair(seed: int, NA: int = 64, MA: int = 32, NB: int = 64, MB: int = 32,
                     n_hits: int = 5, stretch: str = "linear", n_folds: int = 0,
                     device: str = "cpu") -> MeshPair:
    """Mesh A and an independent second surface B of the same family form (its own
    seeded coefficients; no reparameterisation of A and no crossing term), bent
    to pass through n_hits planted points of A: for each, a point p at weights
    (a, b) (margins >= 0.1) in a random A triangle; among 64 random B triangles
    whose bump supports are still free, the one whose point q at its chosen
    weights (c, d) lies nearest to p; B's vertices get (p - q) times a bump that
    is exactly 1 on that triangle's 2 x 2 vertex block (the triangle moves
    rigidly and holds p at (c, d)) and tapers to 0 over two cells.  Pairs whose
    triangle planes are not transverse are skipped.  The planted records carry
    (a, b, c, d), P and (theta, s) in closed form."""
    gen = torch.Generator().manual_seed(seed)
    famA = _make_family(torch.Generator().manual_seed(seed), stretch, 4.0, n_folds, 12.0)
    famB = _make_family(torch.Generator().manual_seed(seed + 7919), stretch, 4.0, n_folds, 12.0)
    thA = torch.arange(NA, dtype=torch.float64) * (TWO_PI / NA)
    thB = torch.arange(NB, dtype=torch.float64) * (TWO_PI / NB)
    sA = torch.linspace(0.0, 1.0, MA, dtype=torch.float64)
    sB = torch.linspace(0.0, 1.0, MB, dtype=torch.float64)
    XA = _surface_A(famA, thA, sA, 0.0)[0]
    XB = _surface_A(famB, thB, sB, 0.0)[0].clone()
    sA_list, sB_list = sA.tolist(), sB.tolist()
    T_taper = 2
    wts = _bump_weights(T_taper)
    usedB = torch.zeros(MB, NB, dtype=torch.bool)
    rec = dict(kind=[], triA=[], triB=[], abcd=[], P=[], params=[], dist=[])
    attempts = 0
    while len(rec["triA"]) < n_hits and attempts < 200 * max(n_hits, 1):
        attempts += 1
        triA = int(torch.randint(0, 2 * NA * (MA - 1), (1,), generator=gen))
        a, b = _shrink(float(torch.rand(1, generator=gen)), float(torch.rand(1, generator=gen)) * 0.5, 0.1)
        va = tri_vertex_ij(NA, triA)
        xv = [XA[:, vk, vi] for (vi, vk) in va]
        p = a * xv[0] + (1.0 - a - b) * xv[1] + b * xv[2]
        best = None
        for _ in range(64):
            triB = int(torch.randint(0, 2 * NB * (MB - 1), (1,), generator=gen))
            q_, tau_b = divmod(triB, 2)
            kb, ib = divmod(q_, NB)
            rows = [kb + dk for dk in range(-T_taper, 2 + T_taper) if 0 <= kb + dk < MB]
            cols = [(ib + di) % NB for di in range(-T_taper, 2 + T_taper)]
            if usedB[rows][:, cols].any():
                continue
            c, d = _shrink(float(torch.rand(1, generator=gen)), float(torch.rand(1, generator=gen)) * 0.5, 0.1)
            yv = [XB[:, vk, vi] for (vi, vk) in tri_vertex_ij(NB, triB)]
            q = c * yv[0] + (1.0 - c - d) * yv[1] + d * yv[2]
            dist = float((p - q).norm())
            if best is None or dist < best[0]:
                best = (dist, triB, c, d, kb, ib, rows, cols, q, yv)
        if best is None:
            continue
        _, triB, c, d, kb, ib, rows, cols, q, yv = best
        if _plane_transversality(xv, yv) < 0.01:
            continue
        delta = p - q
        for r in rows:
            usedB[r, cols] = True
        for dk in range(-T_taper, 2 + T_taper):
            r = kb + dk
            if not (0 <= r < MB):
                continue
            wk = wts[0] if dk in (0, 1) else wts[(-dk) if dk < 0 else dk - 1]
            for di in range(-T_taper, 2 + T_taper):
                col = (ib + di) % NB
                wi = wts[0] if di in (0, 1) else wts[(-di) if di < 0 else di - 1]
                XB[:, r, col] += (wk * wi) * delta
        thu, su = _point_params(NA, sA_list, triA, a, b)
        ths, sss = _point_params(NB, sB_list, triB, c, d)
        rec["kind"].append(0)
        rec["triA"].append(triA)
        rec["triB"].append(triB)
        rec["abcd"].append([a, b, c, d])
        rec["P"].append(p.tolist())
        rec["params"].append([thu, su, ths, sss])
        rec["dist"].append(0.0)
    planted = Planted(
        kind=torch.tensor(rec["kind"], dtype=torch.int32),
        triA=torch.tensor(rec["triA"], dtype=torch.int64),
        triB=torch.tensor(rec["triB"], dtype=torch.int64),
        abcd=torch.tensor(rec["abcd"], dtype=torch.float64).reshape(-1, 4),
        P=torch.tensor(rec["P"], dtype=torch.float64).reshape(-1, 4),
        params=torch.tensor(rec["params"], dtype=torch.float64).reshape(-1, 4),
        dist=torch.tensor(rec["dist"], dtype=torch.float64),
    )
    dev = torch.device(device)
    A = MeshGrid(XA.contiguous().to(dev), sA.to(dev), True)
    B = MeshGrid(XB.contiguous().to(dev), sB.to(dev), True)
    meta = dict(seed=seed, NA=NA, MA=MA, NB=NB, MB=MB, independent=True, stretch=stretch)
    return MeshPair(A, B, planted, meta, None)


def config_seed(config: int, replica: int = 0) -> int:
    return SEED_BASE + 100 * config + replica


def config1(replica: int = 0, device: str = "cpu") -> MeshPair:
    """Plain FP64: 64 x 32 grids, (1 + s) trig surfaces, 5 planted hits."""
    return build_pair(config_seed(1, replica), 64, 32, 64, 32, stretch="linear",
                      n_folds=0, sites=(6, 1), n_hits=5, device=device)


def config1_independent(replica: int = 0, device: str = "cpu") -> MeshPair:
    """Plain FP64, 64 x 32 grids: (1 + s) trig surface A and an independent
    seeded trig surface B bent through 5 planted points of A."""
    return independent_pair(config_seed(1, replica) + 50, 64, 32, 64, 32, n_hits=5,
                            stretch="linear", n_folds=0, device=device)


def config2(replica: int = 0, device: str = "cpu") -> MeshPair:
    """Manifold-like stretching: 1024 x 256, lambda = 4, 3 folds, 64 planted hits."""
    return build_pair(config_seed(2, replica), 1024, 256, 1024, 256, stretch="exp",
                      lam=4.0, n_folds=3, sites=(16, 6), n_hits=64, device=device)


def config3(replica: int = 0, device: str = "cpu", N: int = 4096, M: int = 512,
            n_near: int = 10000) -> MeshPair:
    """Mixed precision: 4096 x 512, 256 planted hits + 1e4 planted near-misses."""
    n_th = max(2, (N // 16) & ~1)
    n_s = max(1, (M - 1) // 11)
    return build_pair(config_seed(3, replica), N, M, N, M, stretch="exp", lam=4.0,
                      n_folds=3, sites=(n_th, n_s), n_hits=256, n_near=n_near,
                      device=device)


def config4_sizes(replica: int = 0, n_pairs: int = 256):
    """Uneven per-mesh sizes: N ~ U{128..2048}, M ~ U{32..512}, independently."""
    g = torch.Generator().manual_seed(config_seed(4, replica))
    NA = torch.randint(128, 2049, (n_pairs,), generator=g).tolist()
    MA = torch.randint(32, 513, (n_pairs,), generator=g).tolist()
    NB = torch.randint(128, 2049, (n_pairs,), generator=g).tolist()
    MB = torch.randint(32, 513, (n_pairs,), generator=g).tolist()
    return list(zip(NA, MA, NB, MB))


def config4_pair(p: int, replica: int = 0, n_pairs: int = 256, device: str = "cpu",
                 sizes=None) -> MeshPair:
    """Pair p of the batched continuation sweep: alpha_p = p / (n_pairs - 1)."""
    if sizes is None:
        sizes = config4_sizes(replica, n_pairs)
    NA, MA, NB, MB = sizes[p]
    alpha = p / max(n_pairs - 1, 1)
    return build_pair(config_seed(4, replica) * 1000 + p, NA, MA, NB, MB, stretch="exp",
                      lam=4.0, n_folds=3, sites=(8, 2), n_hits=4, alpha=alpha,
                      with_dalpha=True, device=device,
                      family_seed=config_seed(4, replica))


def config5(replica: int = 0, device: str = "cpu") -> MeshPair:
    """Differentiation: 1024 x 256 at alpha = 0.5, 512 planted hits, dX/dalpha."""
    return build_pair(config_seed(5, replica), 1024, 256, 1024, 256, stretch="exp",
                      lam=4.0, n_folds=3, sites=(64, 10), n_hits=512, alpha=0.5,
                      with_dalpha=True, device=device)


def family_pair(seed: int, alpha: float, N: int = 96, M: int = 48, device: str = "cpu",
                n_hits: int = 8) -> MeshPair:
    """A small member of an alpha family (used for finite differences in alpha)."""
    return build_pair(seed, N, M, N, M, stretch="exp", lam=4.0, n_folds=3,
                      sites=(8, 2), n_hits=n_hits, alpha=alpha, with_dalpha=True,
                      device=device, family_seed=seed, alpha_ref=0.5)


# ----------------------------------------------------------------------------
# globalized meshes with layer structure (method of layers)
# ----------------------------------------------------------------------------

def layered_s_grid(D: float, lam: float, n_lo: int, n_hi: int, per_layer: int,
                   fund: int) -> torch.Tensor:
    """Sorted s values of a globalized mesh whose half-layers are
    [D lam^(n-1), D lam^n] (lam > 1) for n = n_lo..n_hi and their mirror images,
    each sampled by per_layer + 1 geometrically spaced columns (boundaries
    shared), plus fund - 1 evenly spaced columns strictly inside the innermost
    boundary.  A stable-manifold grid with multiplier mu < 1 is the same grid
    with lam = 1 / mu (its half-layer m spans [D / mu^(m-1), D / mu^m])."""
    pos = []
    for n in range(n_lo, n_hi + 1):
        for j in range(per_layer + (1 if n == n_hi else 0)):
            pos.append(D * lam ** (n - 1 + j / per_layer))
    inner = pos[0]
    mid = [inner * (2.0 * i / fund - 1.0) for i in range(1, fund)]
    vals = [-v for v in reversed(pos)] + mid + pos
    return torch.tensor(vals, dtype=torch.float64)


def layered_pair(seed: int = SEED_BASE + 600, NA: int = 1024, NB: int = 2048, n_max: int = 14,
                 per_layer: int = 34, D_u: float = 1e-2, lam_u: float = 2.0, D_s: float = 1e-2,
                 lam_s: float = 0.5, fund: int = 4, n_hits: int = 64, sites=(16, 12),
                 device: str = "cpu") -> MeshPair:
    """Globalized unstable and stable meshes for the method of layers: the
    surface geometry of build_pair (vertex columns in order), with s values
    relabelled so that the columns group into half-layers U_n^+-, n = 1..n_max,
    of per_layer quads ([D_u lam_u^(n-1), D_u lam_u^n]) and S_m^+-, m = 0..n_max
    ([D_s / lam_s^(m-1), D_s / lam_s^m]), with fund - 1 columns of the
    fundamental domain between the two signs.  With the defaults the meshes
    have the paper's benchmark shapes: N1 = 1024, N2 = 2048 and 35 columns per
    half-layer, 14 layers, 112 half-layer pairs."""
    sA = layered_s_grid(D_u, lam_u, 1, n_max, per_layer, fund)
    sB = layered_s_grid(D_s, 1.0 / lam_s, 0, n_max, per_layer, fund)
    pair = build_pair(seed, NA, sA.numel(), NB, sB.numel(), stretch="exp", lam=4.0, n_folds=3,
                      sites=sites, n_hits=n_hits, device=device)
    pair.A = MeshGrid(pair.A.X, sA.to(pair.A.X.device), True)
    pair.B = MeshGrid(pair.B.X, sB.to(pair.B.X.device), True)
    pair.meta.update(layers=dict(D_u=D_u, lam_u=lam_u, D_s=D_s, lam_s=lam_s, n_max=n_max,
                                 per_layer=per_layer, fund=fund))
    return pair
