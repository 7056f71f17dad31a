"""Pins of the refinement oracle (oracle/refine.py, Sec. 7 Eqs. tosolve and
dampedNewtonEquation) against facts fixed outside it: the generator's own mesh
vertices, finite differences, the sheets' constructed crossings, the
determinant identity at those crossings, Newton's convergence rates and the
Hadamard bound."""
import copy
import math

import numpy as np
import pytest

import synth
from oracle import refine as R


def _pair(stretch="exp", alpha=0.3, seed=4321):
    return synth.build_pair(seed, 48, 20, 40, 24, stretch=stretch,
                            n_folds=0 if stretch == "linear" else 3, sites=(6, 2), n_hits=0,
                            alpha=alpha, with_dalpha=True)


@pytest.mark.parametrize("stretch,alpha", [("linear", 0.0), ("exp", 0.3), ("exp", 0.5)])
def test_sheets_reproduce_mesh_vertices(stretch, alpha):
    # with nothing planted the meshes are exact samples of the two sheets
    p = _pair(stretch, alpha)
    sp = p.surface
    for grid, fn in ((p.A, R.surface_A), (p.B, R.surface_B)):
        X = grid.X.numpy()
        M, N = X.shape[1], X.shape[2]
        th = np.tile(np.arange(N) * (2 * math.pi / N), M)
        s = np.repeat(grid.s.numpy(), N)
        W, _, _ = fn(sp, th, s)
        assert np.abs(W.T.reshape(4, M, N) - X).max() <= 1e-12 * (1.0 + np.abs(X).max())


@pytest.mark.parametrize("stretch", ["linear", "exp"])
def test_partials_match_central_differences(stretch):
    sp = _pair(stretch).surface
    rng = np.random.default_rng(7)
    x = np.stack([rng.uniform(0, 2 * math.pi, 64), rng.uniform(0, 1, 64),
                  rng.uniform(0, 2 * math.pi, 64), rng.uniform(0, 1, 64)], axis=1)
    _, Df = R.residual(sp, x)
    h = 1e-6
    for j in range(4):
        e = np.zeros(4)
        e[j] = h
        fd = (R.residual(sp, x + e)[0] - R.residual(sp, x - e)[0]) / (2 * h)
        assert np.abs(fd - Df[:, :, j]).max() <= 1e-8 * np.abs(Df[:, :, j]).max()


def test_sites_are_roots_with_closed_form_determinant():
    p = _pair("exp", 0.3)
    sp = p.surface
    x = R.site_roots(sp)
    f, Df = R.residual(sp, x)
    scale = np.abs(p.A.X.numpy()).max()
    assert np.abs(f).max() <= 1e-13 * scale
    # at a site Df = [A_t, A_s, -A_t - H_t, A_s - H_s] with H_t = h P cos(.) n1 and
    # H_s = h Q pi cos(.) n2, so det Df = h^2 P Q pi cos cos det[A_t, A_s, n1, n2]
    _, At, As = R.surface_A(sp, x[:, 0], x[:, 1])
    fr = R.frame(sp, x[:, 2], x[:, 3])
    c1 = np.cos(sp.P * (x[:, 2] - sp.theta0))
    c2 = np.cos(sp.Q * math.pi * (x[:, 3] - sp.s0))
    assert np.allclose(np.abs(c1), 1.0) and np.allclose(np.abs(c2), 1.0)
    want = sp.h_amp ** 2 * sp.P * sp.Q * math.pi * c1 * c2 * \
        np.linalg.det(np.stack([At, As, fr["n"][0], fr["n"][1]], axis=2))
    got = np.linalg.det(Df)
    assert np.allclose(got, want, rtol=1e-9, atol=0)
    assert np.all(np.abs(want) > 0)


def test_newton_converges_to_sites_quadratically():
    sp = _pair("exp", 0.3).surface
    roots = R.site_roots(sp)
    rng = np.random.default_rng(11)
    x0 = roots + rng.normal(0.0, 1e-3, roots.shape)
    res = R.damped_newton(sp, x0, history=True, alpha0=1.0, alpha1=1.0, tol=1e-12)
    assert np.all(res["status"] == R.CONVERGED)
    d = np.abs(res["x"] - roots)
    d[:, [0, 2]] = np.minimum(d[:, [0, 2]], 2 * math.pi - d[:, [0, 2]])
    assert d.max() < 1e-10
    for h in res["history"]:
        # r_{k+1} <= C r_k^2 while above the rounding floor
        for r0, r1 in zip(h, h[1:]):
            if r1 > 1e-13:
                assert r1 <= 50.0 * r0 * r0


def test_damping_gives_linear_rate_one_minus_alpha():
    sp = _pair("exp", 0.3).surface
    roots = R.site_roots(sp)
    rng = np.random.default_rng(12)
    x0 = roots + rng.normal(0.0, 1e-4, roots.shape)
    for alpha in (0.5, 0.1):
        res = R.damped_newton(sp, x0, history=True, alpha0=alpha, alpha1=alpha, tol=1e-11,
                              max_iter=400)
        assert np.all(res["status"] == R.CONVERGED)
        for h in res["history"]:
            ratios = [b / a for a, b in zip(h[2:], h[3:]) if b > 1e-10]
            assert ratios and max(abs(q - (1.0 - alpha)) for q in ratios) < 0.02


def test_alpha_switch_goes_quadratic_below_threshold():
    sp = _pair("exp", 0.3).surface
    roots = R.site_roots(sp)
    x0 = roots + np.random.default_rng(13).normal(0.0, 1e-3, roots.shape)
    res = R.damped_newton(sp, x0, history=True, alpha0=0.5, alpha1=1.0, switch_below=1e-5)
    assert np.all(res["status"] == R.CONVERGED)
    for h in res["history"]:
        first_small = next(i for i, r in enumerate(h) if r <= 1e-5)
        # above the threshold the residual halves; below it one full step is quadratic
        assert all(abs(b / a - 0.5) < 0.05 for a, b in zip(h[1:first_small], h[2:first_small + 1]))
        assert len(h) - 1 - first_small <= 3


def test_planted_seeds_from_mesh_records_refine_to_their_sites():
    pair = synth.config1()
    sp = pair.surface
    seeds = pair.planted.params.numpy()
    res = R.damped_newton(sp, seeds)
    roots = R.site_roots(sp)
    assert np.all(res["status"] == R.CONVERGED)
    for x in res["x"]:
        d = np.abs(roots - x)
        d[:, [0, 2]] = np.minimum(d[:, [0, 2]], 2 * math.pi - d[:, [0, 2]])
        assert d.max(axis=1).min() < 1e-9


def test_stop_statuses():
    sp = _pair("exp", 0.3).surface
    roots = R.site_roots(sp)
    x0 = roots[:5].copy()
    x0[0, 1] = 2.0                 # s_u outside [s_lo, s_hi]
    x0[1, 3] = -1.0                # s_s outside
    x0[2, 0] = np.nan
    x0[3] += 0.05                  # not a root: one evaluation, no update
    res = R.damped_newton(sp, x0, max_iter=0)
    assert list(res["status"]) == [R.ESCAPED, R.ESCAPED, R.NON_FINITE, R.MAX_ITER, R.CONVERGED]
    assert np.isnan(res["fnorm"][:3]).all() and np.all(res["iters"] == 0)
    assert np.array_equal(res["x"][3], np.mod(x0[3], 2 * math.pi))
    # Hadamard: |det Df| <= prod of column norms, so rho_min > 1 makes every
    # non-root seed singular at its first evaluation
    res = R.damped_newton(sp, x0[3:4], rho_min=1.0 + 1e-9)
    assert res["status"][0] == R.SINGULAR and 0.0 < abs(res["rho"][0]) <= 1.0


def test_frame_vanishes_only_at_h_zero_keeps_roots():
    # with h_amp = 0 sheet B is sheet A reparameterised: every (theta + c0, 1 - s,
    # theta, s) is a root, and Df there has rank 2 (rho = 0 up to rounding)
    sp = copy.copy(_pair("exp", 0.3).surface)
    sp.h_amp = 0.0
    th = np.linspace(0.1, 6.0, 9)
    s = np.linspace(0.05, 0.95, 9)
    x = np.stack([th + sp.c0, 1.0 - s, th, s], axis=1)
    f, Df = R.residual(sp, x)
    assert np.abs(f).max() <= 1e-12 * (1 + np.abs(R.surface_A(sp, x[:, 0], x[:, 1])[0]).max())
    assert np.allclose(Df[:, :, 2], -Df[:, :, 0], rtol=0, atol=1e-12 * np.abs(Df).max())
    assert np.allclose(Df[:, :, 3], Df[:, :, 1], rtol=0, atol=1e-12 * np.abs(Df).max())


# ---------------------------------------------------------------------------
# continuation (Sec. 8)
# ---------------------------------------------------------------------------

def _dW_dalpha(sp, theta, s):
    """Closed-form d/d alpha of the sheet g(s) T(theta; alpha) + F(s)."""
    k = np.arange(1, 7, dtype=np.float64)
    Ta = (np.cos(np.outer(theta, k)) / k) @ sp.dca.numpy() + \
        (np.sin(np.outer(theta, k)) / k) @ sp.dcb.numpy()
    g = np.exp(math.log(sp.lam) * s) if sp.stretch == "exp" else 1.0 + s
    return g[:, None] * Ta


@pytest.mark.parametrize("param", ["u", "s"])
def test_continued_branches_follow_the_implicit_function_theorem(param):
    # along a branch f(x(alpha); alpha) = 0, so dx/dalpha = -Df^{-1} df/dalpha with
    # df/dalpha_u = dW_A/dalpha and df/dalpha_s = -dW_B/dalpha (closed forms); the
    # central difference of the continued branch converges to it as O(h^2)
    sp = synth.config2().surface
    x0 = R.site_roots(sp)[:16]
    au, as_ = R.alphas(sp)
    errs = {}
    for h in (0.001, 0.0005):
        n_to = int(round(0.01 / h))
        res = R.continuation(sp, x0, h * np.arange(1, n_to + 2), param=param, tol=1e-13)
        a = res["alphas"]
        for b in range(x0.shape[0]):
            # well-conditioned stretches only (away from folds, where the branch bends hard)
            if not (res["status"][b, :n_to + 2] == R.CONVERGED).all() or \
                    np.abs(res["rho"][b, :n_to + 2]).min() < 0.02:
                continue
            x = res["x"][b, n_to]
            spj = R.with_alphas(sp, a[n_to] if param == "u" else au, a[n_to] if param == "s" else as_)
            _, Df = R.residual(spj, x[None])
            if param == "u":
                dfa = _dW_dalpha(sp, x[0:1], x[1:2])[0]
            else:
                dfa = -_dW_dalpha(sp, x[2:3] + sp.c0, 1.0 - x[3:4])[0]
            want = -np.linalg.solve(Df[0], dfa)
            d = res["x"][b, n_to + 1] - res["x"][b, n_to - 1]
            d[[0, 2]] -= 2 * math.pi * np.round(d[[0, 2]] / (2 * math.pi))
            got = d / (a[n_to + 1] - a[n_to - 1])
            errs.setdefault(b, []).append(np.abs(got - want).max() / (1.0 + np.abs(want).max()))
    pairs = [e for e in errs.values() if len(e) == 2]
    assert len(pairs) >= 6
    for e1, e2 in pairs:
        assert e2 <= 1e-3 and (e2 <= 1e-9 or 3.0 < e1 / e2 < 5.0), (e1, e2)


def test_predictor_error_is_second_order():
    # Eq. (predictor) extrapolates linearly: its error shrinks 4x when the step halves
    sp = synth.config2().surface
    x0 = R.site_roots(sp)[:16]
    errs = []
    for h in (0.004, 0.002):
        steps = h * np.arange(1, 6)
        res = R.continuation(sp, x0, steps, param="u", tol=1e-13)
        ok = (res["status"][:, :6] == R.CONVERGED).all(axis=1)
        e = np.abs(res["predicted"][ok, 2:6] - res["x"][ok, 2:6])
        errs.append(np.median(e.max(axis=2)))
    assert 3.0 < errs[0] / errs[1] < 5.5


def test_continuation_statuses():
    sp = synth.config2().surface
    x0 = R.site_roots(sp)[:6]
    steps = np.linspace(0.002, 0.01, 5)
    base = R.continuation(sp, x0, steps)
    # step 0 is the corrector at the pair's own parameters
    ref = R.damped_newton(sp, x0)
    assert np.array_equal(base["x"][:, 0], ref["x"]) and np.array_equal(base["iters"][:, 0], ref["iters"])
    # Hadamard: |rho| <= 1, so rho_turn above 1 turns every branch at step 0
    res = R.continuation(sp, x0, steps, rho_turn=1.0 + 1e-9)
    assert (res["status"][:, 0] == R.TURNING).all() and (res["status"][:, 1:] == R.STOPPED).all()
    assert np.isnan(res["x"][:, 1:]).all() and np.isfinite(res["x"][:, 0]).all()
    # a tiny jump allowance stops every branch whose corrector moved at step 1
    res = R.continuation(sp, x0, steps, max_jump=1e-12)
    moved = res["iters"][:, 1] > 0
    assert moved.all() and (res["status"][:, 1] == R.JUMPED).all()
    # no steps: the start only
    res = R.continuation(sp, x0, [])
    assert res["x"].shape == (6, 1, 4) and (res["status"][:, 0] == R.CONVERGED).all()
