"""GPU parity of the theta-grid operations (tms_theta_translate, Eqs. translate
and translate2; tms_phase_align, Eq. rhoEquationDiscrete) against
oracle/theta.py, on seeded random columns and on closed forms."""
import math

import numpy as np
import pytest
import torch

import paper_2109_14814_gb300 as tms
from oracle import theta as T

pytestmark = pytest.mark.gpu


def _cols(C, M, N, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(C, M, N, generator=g, dtype=torch.float64)


@pytest.mark.parametrize("N", [8, 64, 1024, 4096, 8192])
@pytest.mark.parametrize("C", [1, 3, 4])
def test_translate_matches_oracle(N, C):
    M = 5
    X = _cols(C, M, N, N + C)
    rho = torch.tensor([0.0, 0.37, -2.5, 13.0, 2 * math.pi / N * 5.5], dtype=torch.float64)
    scale = float(X.abs().max())
    for deriv in (False, True):
        want = T.translate(X.numpy(), rho.numpy()[None, :], derivative=deriv)
        got = tms.theta_translate(X.cuda(), rho.cuda(), derivative=deriv).cpu().numpy()
        tol = (1e-13 if not deriv else 1e-13 * N) * math.log2(N) * scale
        assert np.abs(got - want).max() <= tol
        # one shift for every column
        want = T.translate(X.numpy(), 0.81, derivative=deriv)
        got = tms.theta_translate(X.cuda(), 0.81, derivative=deriv).cpu().numpy()
        assert np.abs(got - want).max() <= tol


def test_closed_forms_roll_and_in_place():
    N, M = 1024, 3
    th = 2 * math.pi * torch.arange(N, dtype=torch.float64) / N
    k = torch.arange(1, 7, dtype=torch.float64)
    g = torch.Generator().manual_seed(3)
    a = torch.randn(4, M, 6, generator=g, dtype=torch.float64)
    b = torch.randn(4, M, 6, generator=g, dtype=torch.float64)

    def f(t, d=False):
        kt = k[:, None] * t[None, :]
        if d:
            return torch.einsum("cmk,kn->cmn", -a * k, torch.sin(kt)) + \
                torch.einsum("cmk,kn->cmn", b * k, torch.cos(kt))
        return torch.einsum("cmk,kn->cmn", a, torch.cos(kt)) + torch.einsum("cmk,kn->cmn", b, torch.sin(kt))
    X = f(th).contiguous()
    for rho in (0.3, -4.0):
        assert (tms.theta_translate(X.cuda(), rho).cpu() - f(th + rho)).abs().max() <= 1e-12
        assert (tms.theta_translate(X.cuda(), rho, derivative=True).cpu() - f(th + rho, True)).abs().max() <= 1e-10
    R = torch.randn(4, M, N, generator=g, dtype=torch.float64)
    for m in (1, 17, N - 1):
        got = tms.theta_translate(R.cuda(), 2 * math.pi * m / N).cpu()
        assert (got - torch.roll(R, -m, dims=-1)).abs().max() <= 1e-12
    Rd = R.cuda()
    tms.theta_translate(Rd, 0.5, out=Rd)
    assert (Rd.cpu().numpy() - T.translate(R.numpy(), 0.5)).__abs__().max() <= 1e-12


@pytest.mark.parametrize("N,C,A", [(96, 4, 1), (1000, 4, 5), (4096, 4, 3), (300, 1, 2), (257, 8, 2)])
def test_phase_align_matches_oracle(N, C, A):
    g = torch.Generator().manual_seed(N + C + A)
    Wp = torch.randn(A, C, N, generator=g, dtype=torch.float64)
    rolls = [int(x) for x in torch.randint(0, N, (A,), generator=g)]
    Wr = torch.stack([torch.roll(Wp[a], rolls[a], dims=-1) for a in range(A)])
    Wr = Wr + 1e-3 * torch.randn(A, C, N, generator=g, dtype=torch.float64)
    shift, cost = tms.phase_align(Wr.cuda(), Wp.cuda())
    shift, cost = shift.cpu().numpy(), cost.cpu().numpy()
    for a in range(A):
        m, want = T.phase_align(Wr[a].numpy(), Wp[a].numpy())
        assert shift[a] == m == rolls[a]
        assert np.allclose(cost[a], want, rtol=1e-12, atol=0)
    s1, c1 = tms.phase_align(Wr[0].cuda(), Wp[0].cuda())
    assert int(s1) == shift[0] and np.array_equal(c1.cpu().numpy(), cost[0])
