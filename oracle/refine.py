"""CPU oracle of the refinement of approximate manifold intersections -- TEST
INFRASTRUCTURE ONLY (the tests, the package's smoke check and the benchmark's
CPU-baseline leg may call it; the CUDA path never does, and shares no code
with it).

Sec. 7 corrects each approximate intersection found by the mesh search by
solving Eq. (tosolve),
    f(x) = W_A(theta_u, s_u) - W_B(theta_s, s_s) = 0,   x = (theta_u, s_u, theta_s, s_s),
with the damped Newton iteration of Eq. (dampedNewtonEquation),
    x_{k+1} = x_k - alpha Df(x_k)^{-1} f(x_k),
    Df = [d f/d theta_u, d f/d s_u, d f/d theta_s, d f/d s_s],
iterating until f is within a tolerance.  W_A is taken at the family parameter
alpha_u and the sheet under W_B at alpha_s (both default to the pair's alpha),
standing in for the two tori's rotation numbers omega_u, omega_s of Sec. 8.
In the paper W and its partials come
from Fourier-Taylor series and the flow (Eqs. wuequation-dwsdsequation); here
the two manifolds are the closed-form synthetic sheets that the seeded meshes
sample (synth.SurfacePair), and the partials are their exact derivatives,
written out below term by term.  All arithmetic is float64 numpy, vectorised
over the seeds; the 4x4 solve and determinant are LAPACK's (numpy.linalg).

Readings of the paper taken here (the paper fixes none of them):
  * alpha: one value while ||f||_2 > switch_below and another below it (the
    paper changes alpha once during an iteration and uses values 0.01..0.5);
    alpha = 1 (the undamped limit) is allowed.
  * stopping: ||f(x_k)||_2 <= tol ends the iteration at x_k (converged);
    at most max_iter updates (else "max_iter"); a seed whose s_u or s_s leaves
    [s_lo, s_hi] stops ("escaped"); Df counts as singular when
    |det Df| / prod_j ||Df e_j|| < rho_min ("singular"); a non-finite iterate or
    residual stops ("non_finite").
  * theta_u, theta_s are returned reduced to [0, 2 pi).
"""
from __future__ import annotations

import copy
import math

import numpy as np

TWO_PI = 2.0 * math.pi

CONVERGED, MAX_ITER, SINGULAR, ESCAPED, NON_FINITE = range(5)
STATUS_NAMES = ("converged", "max_iter", "singular", "escaped", "non_finite")

DEFAULTS = dict(alpha0=0.5, alpha1=0.5, switch_below=0.0, tol=1e-10, max_iter=200,
                s_lo=-0.5, s_hi=1.5, rho_min=1e-14)


def _np(t):
    return np.asarray(t.detach().cpu().numpy() if hasattr(t, "detach") else t, dtype=np.float64)


def alphas(sp):
    """(alpha_u, alpha_s): the family parameters of W_A and of B's sheet."""
    return float(getattr(sp, "alpha_u", sp.alpha)), float(getattr(sp, "alpha_s", sp.alpha))


def _coeffs(sp, alpha):
    """(a_k, b_k) = (ca_k + alpha dca_k, cb_k + alpha dcb_k), shape (K, 4)."""
    return _np(sp.ca) + alpha * _np(sp.dca), _np(sp.cb) + alpha * _np(sp.dcb)


def _stretch(sp, s):
    """g(s), g'(s), g''(s)."""
    if sp.stretch == "linear":
        return 1.0 + s, np.ones_like(s), np.zeros_like(s)
    ln = math.log(sp.lam)
    g = np.exp(ln * s)
    return g, ln * g, ln * ln * g


def _folds(sp, s):
    """F(s), F'(s), F''(s) as (n, 4): sum_f amp_f p_f(s) e_f with
    p_f = (s - r1)(s - r2)(s - r3)."""
    amp, roots, dirs = _np(sp.fold_amp), _np(sp.fold_roots), _np(sp.fold_dir)
    F = np.zeros((s.size, 4))
    F1 = np.zeros((s.size, 4))
    F2 = np.zeros((s.size, 4))
    for f in range(amp.size):
        d0, d1, d2 = s - roots[f, 0], s - roots[f, 1], s - roots[f, 2]
        p = d0 * d1 * d2
        p1 = d1 * d2 + d0 * d2 + d0 * d1
        p2 = 2.0 * (d0 + d1 + d2)
        F += amp[f] * p[:, None] * dirs[f][None, :]
        F1 += amp[f] * p1[:, None] * dirs[f][None, :]
        F2 += amp[f] * p2[:, None] * dirs[f][None, :]
    return F, F1, F2


def sheet(sp, theta, s, alpha):
    """The underlying sheet S(theta, s) = g(s) T(theta; alpha) + F(s) and its
    first and second partials, each (n, 4): keys W, Wt, Ws, Wtt, Wts, Wss."""
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    a, b = _coeffs(sp, alpha)
    k = np.arange(1, a.shape[0] + 1, dtype=np.float64)
    kt = theta[:, None] * k[None, :]
    C, S = np.cos(kt), np.sin(kt)
    T = (C / k) @ a + (S / k) @ b            # sum (a_k cos + b_k sin) / k
    Tt = -S @ a + C @ b                      # d/dtheta
    Ttt = -(C * k) @ a - (S * k) @ b         # d2/dtheta2
    g, g1, g2 = _stretch(sp, s)
    F, F1, F2 = _folds(sp, s)
    return dict(W=g[:, None] * T + F, Wt=g[:, None] * Tt, Ws=g1[:, None] * T + F1,
                Wtt=g[:, None] * Ttt, Wts=g1[:, None] * Tt, Wss=g2[:, None] * T + F2)


def _dot(u, v):
    return np.sum(u * v, axis=1)


def frame(sp, theta, s):
    """Normal frame (n1, n2) of sheet B at B's (theta, s) and its partials in
    theta and s: returns {"n": [n1, n2], "n_t": [...], "n_s": [...]}, (n, 4)."""
    S = sheet(sp, np.asarray(theta) + sp.c0, 1.0 - np.asarray(s), sp.alpha_ref)
    t1, t2 = S["Wt"], S["Ws"]
    # partials of (t1, t2) in B's theta (d theta'/d theta = 1) and s (d s'/d s = -1)
    dirs = {"t": (S["Wtt"], S["Wts"]), "s": (-S["Wts"], -S["Wss"])}
    g11, g12, g22 = _dot(t1, t1), _dot(t1, t2), _dot(t2, t2)
    eps = sp.reg * 0.5 * (g11 + g22)
    G11, G12, G22 = g11 + eps, g12, g22 + eps
    det = G11 * G22 - G12 * G12

    def solve2(r1, r2):
        return (G22 * r1 - G12 * r2) / det, (-G12 * r1 + G11 * r2) / det

    out = {"n": [], "n_t": [], "n_s": []}
    for v in (_np(sp.v1), _np(sp.v2)):
        V = np.broadcast_to(v, t1.shape)
        j1, j2 = _dot(t1, V), _dot(t2, V)
        y1, y2 = solve2(j1, j2)
        out["n"].append(V - t1 * y1[:, None] - t2 * y2[:, None])
        for key, (d1, d2) in dirs.items():
            dg11, dg12, dg22 = 2.0 * _dot(t1, d1), _dot(t1, d2) + _dot(d1, t2), 2.0 * _dot(t2, d2)
            deps = sp.reg * 0.5 * (dg11 + dg22)
            dG11, dG12, dG22 = dg11 + deps, dg12, dg22 + deps
            # d y = G^{-1} (d(J^T v) - dG y)
            r1 = _dot(d1, V) - (dG11 * y1 + dG12 * y2)
            r2 = _dot(d2, V) - (dG12 * y1 + dG22 * y2)
            dy1, dy2 = solve2(r1, r2)
            dn = -(d1 * y1[:, None] + d2 * y2[:, None]) - (t1 * dy1[:, None] + t2 * dy2[:, None])
            out["n_" + key].append(dn)
    return out


def surface_A(sp, theta, s):
    """W_A and its partials (n, 4): (W, W_theta, W_s)."""
    S = sheet(sp, theta, s, alphas(sp)[0])
    return S["W"], S["Wt"], S["Ws"]


def surface_B(sp, theta, s):
    """W_B and its partials (n, 4): (W, W_theta, W_s)."""
    theta = np.atleast_1d(np.asarray(theta, dtype=np.float64))
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    S = sheet(sp, theta + sp.c0, 1.0 - s, alphas(sp)[1])
    fr = frame(sp, theta, s)
    ph1 = sp.P * (theta - sp.theta0)
    ph2 = sp.Q * math.pi * (s - sp.s0)
    s1, c1 = np.sin(ph1)[:, None], np.cos(ph1)[:, None]
    s2, c2 = np.sin(ph2)[:, None], np.cos(ph2)[:, None]
    n1, n2 = fr["n"]
    H = sp.h_amp * (s1 * n1 + s2 * n2)
    Ht = sp.h_amp * (sp.P * c1 * n1 + s1 * fr["n_t"][0] + s2 * fr["n_t"][1])
    Hs = sp.h_amp * (s1 * fr["n_s"][0] + sp.Q * math.pi * c2 * n2 + s2 * fr["n_s"][1])
    return S["W"] + H, S["Wt"] + Ht, -S["Ws"] + Hs


def residual(sp, x):
    """f(x) (n, 4) of Eq. (tosolve) and Df(x) (n, 4, 4), columns in the order
    (theta_u, s_u, theta_s, s_s)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    WA, WAt, WAs = surface_A(sp, x[:, 0], x[:, 1])
    WB, WBt, WBs = surface_B(sp, x[:, 2], x[:, 3])
    f = WA - WB
    Df = np.stack([WAt, WAs, -WBt, -WBs], axis=2)
    return f, Df


def damped_newton(sp, x0, history: bool = False, **kw):
    """Eq. (dampedNewtonEquation) from seeds x0 (n, 4).  Returns a dict of
    x (n, 4), fnorm (n,) (||f|| at the last evaluation, NaN if none), iters (n,)
    (updates made), status (n,), rho (n,) (det Df / prod of column norms at
    the last evaluation, signed) and, if history, per-seed lists of ||f_k||."""
    opt = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in opt:
            raise KeyError(k)
        opt[k] = v
    x = np.array(np.atleast_2d(np.asarray(x0, dtype=np.float64)), copy=True)
    n = x.shape[0]
    fnorm = np.full(n, np.nan)
    rho = np.full(n, np.nan)
    iters = np.zeros(n, dtype=np.int64)
    status = np.full(n, -1, dtype=np.int64)
    hist = [[] for _ in range(n)]
    active = np.ones(n, dtype=bool)
    k = 0
    while active.any():
        idx = np.nonzero(active)[0]
        xa = x[idx]
        code = np.full(idx.size, -1)
        code[(xa[:, 1] < opt["s_lo"]) | (xa[:, 1] > opt["s_hi"]) |
             (xa[:, 3] < opt["s_lo"]) | (xa[:, 3] > opt["s_hi"])] = ESCAPED
        code[~np.isfinite(xa).all(axis=1)] = NON_FINITE
        ev = code < 0
        ev_idx = idx[ev]
        if ev_idx.size:
            f, Df = residual(sp, x[ev_idx])
            r = np.sqrt(np.sum(f * f, axis=1))
            fin = np.isfinite(f).all(axis=1) & np.isfinite(Df).all(axis=(1, 2))
            Dfs = np.where(fin[:, None, None], Df, np.eye(4))
            rh = np.linalg.det(Dfs) / np.sqrt(np.sum(Dfs * Dfs, axis=1)).prod(axis=1)
            fnorm[ev_idx] = r
            rho[ev_idx] = rh
            if history:
                for i, ri in zip(ev_idx, r):
                    hist[i].append(float(ri))
            sub = np.full(r.size, -1)
            sub[~fin] = NON_FINITE
            sub[(sub < 0) & (r <= opt["tol"])] = CONVERGED
            if k == opt["max_iter"]:
                sub[sub < 0] = MAX_ITER
            sub[(sub < 0) & ~(np.abs(rh) >= opt["rho_min"])] = SINGULAR
            code[ev] = sub
            go = sub < 0
            if go.any():
                # x_{k+1} = x_k - alpha Df^{-1} f
                dx = np.linalg.solve(Dfs[go], f[go][:, :, None])[:, :, 0]
                a = np.where(r[go] > opt["switch_below"], opt["alpha0"], opt["alpha1"])
                x[ev_idx[go]] -= a[:, None] * dx
        done = code >= 0
        status[idx[done]] = code[done]
        iters[idx[done]] = k
        active[idx[done]] = False
        k += 1
    with np.errstate(invalid="ignore"):       # non-finite iterates stay non-finite
        x[:, 0] = np.mod(x[:, 0], TWO_PI)
        x[:, 2] = np.mod(x[:, 2], TWO_PI)
    res = dict(x=x, fnorm=fnorm, iters=iters, status=status, rho=rho)
    if history:
        res["history"] = hist
    return res


def site_roots(sp):
    """The crossings the sheets share by construction: for every lattice site
    (theta, s) of B, x* = (theta + c0 mod 2 pi, 1 - s, theta, s)."""
    st = _np(sp.sites)
    return np.stack([np.mod(st[:, 0] + sp.c0, TWO_PI), 1.0 - st[:, 1], st[:, 0], st[:, 1]], axis=1)


# ---------------------------------------------------------------------------
# continuation of connections through the family parameter (Sec. 8)
# ---------------------------------------------------------------------------

TURNING, JUMPED, STOPPED = 5, 6, 7
CONT_STATUS_NAMES = STATUS_NAMES + ("turning", "jumped", "stopped")


def with_alphas(sp, alpha_u, alpha_s):
    """A shallow copy of the sheet pair at (alpha_u, alpha_s)."""
    out = copy.copy(sp)
    out.alpha_u, out.alpha_s = float(alpha_u), float(alpha_s)
    return out


def continuation(sp, x0, alpha_steps, param: str = "u", rho_turn: float = 1e-8,
                 max_jump: float = 0.25, **kw):
    """Continuation of connections x(alpha) (Sec. 8, Eq. predictor) through the
    values alpha_steps (K,) of alpha_u (param "u") or alpha_s ("s"), the other
    parameter held at the pair's value.  Step 0 corrects the seeds x0 (n, 4) at
    the pair's own parameters; step j >= 1 at alpha_j predicts
        j = 1:  x_0
        j >= 2: x_{j-1} + (alpha_j - alpha_{j-1}) / (alpha_{j-1} - alpha_{j-2}) (x_{j-1} - x_{j-2})
    (theta differences taken on the circle, in [-pi, pi]) and corrects by
    damped_newton(**kw) at alpha_j.  A branch stops at the first step whose
    corrector does not converge (that step keeps the corrector's status), whose
    corrected point lies farther than max_jump from its prediction in some
    coordinate (theta on the circle; JUMPED: the corrector left the branch), or
    whose normalised det Df is below rho_turn in magnitude or has the other sign
    than at the previous step (TURNING); x is kept for those steps.  Later steps
    are STOPPED with NaN outputs.  Returns x (n, K+1, 4), status, iters (n, K+1), rho, fnorm (n, K+1)
    and the parameter values (K+1,)."""
    au, as_ = alphas(sp)
    a0 = au if param == "u" else as_
    avals = np.concatenate([[a0], np.asarray(alpha_steps, dtype=np.float64)])
    x0 = np.atleast_2d(np.asarray(x0, dtype=np.float64))
    n, K1 = x0.shape[0], avals.size
    X = np.full((n, K1, 4), np.nan)
    G = np.full((n, K1, 4), np.nan)
    ST = np.full((n, K1), STOPPED, dtype=np.int64)
    IT = np.zeros((n, K1), dtype=np.int64)
    RH = np.full((n, K1), np.nan)
    FN = np.full((n, K1), np.nan)
    alive = np.ones(n, dtype=bool)
    for j in range(K1):
        idx = np.nonzero(alive)[0]
        if idx.size == 0:
            break
        if j == 0:
            guess = x0[idx]
        elif j == 1:
            guess = X[idx, 0]
        else:
            d = X[idx, j - 1] - X[idx, j - 2]
            d[:, [0, 2]] -= TWO_PI * np.round(d[:, [0, 2]] / TWO_PI)
            guess = X[idx, j - 1] + (avals[j] - avals[j - 1]) / (avals[j - 1] - avals[j - 2]) * d
        G[idx, j] = guess
        spj = with_alphas(sp, avals[j] if param == "u" else au, avals[j] if param == "s" else as_)
        r = damped_newton(spj, guess, **kw)
        X[idx, j] = r["x"]
        IT[idx, j] = r["iters"]
        RH[idx, j] = r["rho"]
        FN[idx, j] = r["fnorm"]
        st = r["status"].copy()
        conv = st == CONVERGED
        dj = np.abs(r["x"] - guess)
        dj[:, [0, 2]] = np.abs(dj[:, [0, 2]] - TWO_PI * np.round(dj[:, [0, 2]] / TWO_PI))
        jump = conv & ~(dj.max(axis=1) <= max_jump)
        turn = conv & ~jump & ~(np.abs(r["rho"]) >= rho_turn)
        if j > 0:
            turn |= conv & ~jump & ((r["rho"] > 0) != (RH[idx, j - 1] > 0))
        st[turn] = TURNING
        st[jump] = JUMPED
        ST[idx, j] = st
        alive[idx[st != CONVERGED]] = False
    stopped = ST == STOPPED
    X[stopped] = np.nan
    return dict(x=X, status=ST, iters=IT, rho=RH, fnorm=FN, alphas=avals, predicted=G)
