"""Pins of the theta-grid oracle (oracle/theta.py: Eqs. translate, translate2 and
rhoEquationDiscrete) against closed forms: trigonometric polynomials translate
and differentiate exactly, grid shifts are cyclic rolls, shifts compose, and a
rolled copy aligns back to its roll."""
import math

import numpy as np
import pytest

from oracle import theta as T


def _trig(N, K=6, seed=0, rows=3):
    """Rows of a band-limited real signal (degree K < N/2) and closed forms."""
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(rows, K + 1))
    b = rng.normal(size=(rows, K + 1))
    k = np.arange(K + 1)

    def f(th, deriv=False):
        th = np.asarray(th)
        c, s = np.cos(np.multiply.outer(th, k)), np.sin(np.multiply.outer(th, k))
        if deriv:
            return (-s * k) @ a.T + (c * k) @ b.T
        return c @ a.T + s @ b.T
    return f


@pytest.mark.parametrize("N", [16, 64, 1024, 4096])
def test_translation_and_derivative_of_trig_polynomials(N):
    f = _trig(N)
    th = 2 * math.pi * np.arange(N) / N
    x = f(th).T                                   # (rows, N)
    for rho in (0.0, 0.37, -2.5, 13.0, 2 * math.pi / N * 5.5):
        got = T.translate(x, rho)
        assert np.abs(got - f(th + rho).T).max() <= 1e-12 * np.abs(x).max()
        d = T.translate(x, rho, derivative=True)
        assert np.abs(d - f(th + rho, deriv=True).T).max() <= 1e-11 * np.abs(x).max()


@pytest.mark.parametrize("N", [8, 15, 64, 256])
def test_grid_shift_is_a_cyclic_roll_and_shifts_compose(N):
    rng = np.random.default_rng(N)
    x = rng.normal(size=(4, N))                   # not band-limited
    for m in (0, 1, 3, N - 1, -2):
        got = T.translate(x, 2 * math.pi * m / N)
        assert np.abs(got - np.roll(x, -m, axis=-1)).max() <= 1e-12
    # translations compose on data without a Nyquist component (with one, the grid
    # keeps only cos(N rho / 2) of it, so two steps differ from one)
    X = np.fft.fft(x, axis=-1)
    if N % 2 == 0:
        X[:, N // 2] = 0.0
    xb = np.fft.ifft(X, axis=-1).real
    r1, r2 = 0.3, -1.1
    assert np.allclose(T.translate(T.translate(xb, r1), r2), T.translate(xb, r1 + r2), atol=1e-12)
    # per-row shifts broadcast against the leading dimension
    rho = np.array([0.1, 0.2, 0.3, 0.4])
    one = np.stack([T.translate(x[i], rho[i]) for i in range(4)])
    assert np.array_equal(T.translate(x, rho), one)
    # real data stays real and the mean (k = 0) is kept
    assert np.isclose(T.translate(x, 0.77).mean(), x.mean(), atol=1e-13)


def test_phase_alignment_recovers_a_roll():
    rng = np.random.default_rng(5)
    N = 96
    th = 2 * math.pi * np.arange(N) / N
    W = np.stack([np.cos(th) + 0.3 * np.sin(3 * th), np.sin(2 * th), np.cos(5 * th + 1.0),
                  0.1 * rng.normal(size=N)])
    for m0 in (0, 7, 50, N - 1):
        Wr = np.roll(W, m0, axis=1)               # W_r(theta_i) = W(theta_i - alpha_m0)
        m, cost = T.phase_align(Wr, W)
        assert m == m0 and cost[m] == 0.0 and cost.min() == 0.0
        # brute force of the definition at one other shift
        j = (m0 + 3) % N
        want = sum(math.sqrt(sum((Wr[c, (i + j) % N] - W[c, i]) ** 2 for c in range(4)))
                   for i in range(N))
        assert abs(cost[j] - want) <= 1e-12 * want
    # ties go to the smallest shift: a constant circle costs the same at every shift
    m, cost = T.phase_align(np.ones((4, 12)), np.zeros((4, 12)))
    assert m == 0 and np.allclose(cost, 24.0)
