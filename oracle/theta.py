"""CPU oracle of the operations on theta grids -- TEST INFRASTRUCTURE ONLY (the
tests and the benchmark's CPU leg may call it; the CUDA path never does).

Functions of theta are stored at theta_i = 2 pi i / N (Sec. 4 and Sec. 6.1).

Translation, Eq. (translate): with a_hat = FFT(a), the values a(theta_i + rho) are
    (1/N) sum_k a_hat(k) e^{j k rho} e^{j k theta_i};
the derivative, Eq. (translate2), multiplies a_hat(k) by j k instead.  Globalizing
a manifold translates every s column of the four coordinate arrays by
rho = -n omega (Sec. 6.1).

Reading (the paper writes k = 0..N-1, which for real data and a shift off the
grid gives complex values): k runs over the signed frequencies of the grid,
0..N/2-1 and -N/2..-1 (numpy.fft.fftfreq(N) * N); for even N the Nyquist
coefficient k = N/2 is multiplied by cos(N rho / 2) when translating and by 0
when differentiating.  The result is then the trigonometric interpolant of the
samples evaluated at theta_i + rho (or its derivative), real for real data,
and an exact cyclic shift when rho is a multiple of 2 pi / N.

Phase alignment, Eq. (rhoEquationDiscrete): the shift alpha_m = 2 pi m / N,
m in 0..N-1, minimising
    cost(m) = sum_i || W_r(theta_i + alpha_m) - W_prev(theta_i) ||
(Euclidean norm over the coordinates), where W_r(theta_i + alpha_m) is the
stored sample (i + m) mod N.  Ties go to the smallest m.
"""
from __future__ import annotations

import numpy as np


def translate(a, rho, derivative: bool = False):
    """a: (..., N) real samples; rho: scalar or an array broadcasting against
    a's leading dimensions.  Returns the samples of a(theta + rho), or of its
    theta-derivative when `derivative`."""
    a = np.asarray(a, dtype=np.float64)
    N = a.shape[-1]
    rho = np.asarray(rho, dtype=np.float64)
    k = np.fft.fftfreq(N, d=1.0 / N)
    H = np.exp(1j * k * rho[..., None])
    if derivative:
        H = H * (1j * k)
    if N % 2 == 0:
        H[..., N // 2] = 0.0 if derivative else np.cos(0.5 * N * rho)
    return np.fft.ifft(np.fft.fft(a, axis=-1) * H, axis=-1).real


def phase_cost(Wr, Wprev):
    """cost(m), m = 0..N-1, for coordinate arrays Wr, Wprev of shape (C, N)."""
    Wr = np.asarray(Wr, dtype=np.float64)
    Wprev = np.asarray(Wprev, dtype=np.float64)
    N = Wr.shape[-1]
    cost = np.empty(N)
    for m in range(N):
        d = np.roll(Wr, -m, axis=-1) - Wprev          # column i holds W_r[(i + m) mod N]
        cost[m] = np.sqrt((d * d).sum(axis=0)).sum()
    return cost


def phase_align(Wr, Wprev):
    """(m*, cost): the minimising grid shift of Eq. (rhoEquationDiscrete)."""
    cost = phase_cost(Wr, Wprev)
    return int(np.argmin(cost)), cost
