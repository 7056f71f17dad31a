"""Adjoint of the hit outputs: GPU (tms_backward / HitPoint) against the CPU
oracle's reverse-mode derivative, central finite differences in the vertices
and in the family parameter alpha, and the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
import paper_2109_14814_gb300 as tms
import synth

pytestmark = pytest.mark.gpu


def _setup(pair):
    XA = pair.A.X.cuda().contiguous()
    XB = pair.B.X.cuda().contiguous()
    A = tms.Mesh(XA, pair.A.s)
    B = tms.Mesh(XB, pair.B.s)
    hits = tms.search(A, B)
    return XA, XB, A, B, hits


def test_backward_matches_oracle_gradient_config5():
    pair = synth.config5()
    XA, XB, A, B, hits = _setup(pair)
    n = len(hits)
    assert n >= 512
    g = torch.Generator().manual_seed(7)
    gP = torch.randn(n, 4, generator=g, dtype=torch.float64)
    gZ = torch.randn(n, 4, generator=g, dtype=torch.float64)
    gA = torch.zeros_like(XA)
    gB = torch.zeros_like(XB)
    galpha = torch.zeros(n, dtype=torch.float64, device="cuda")
    dA = pair.A.dXdalpha.cuda().contiguous()
    dB = pair.B.dXdalpha.cuda().contiguous()
    tms.backward(A, B, hits, gP=gP.cuda(), gZ=gZ.cuda(), gradA=gA, gradB=gB,
                 dA_dalpha=dA, dB_dalpha=dB, galpha=galpha)
    torch.cuda.synchronize()
    OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
    rA, rB, ralpha = oracle.hit_grads(OA, OB, hits.triA.cpu().numpy(), hits.triB.cpu().numpy(),
                                      gP.numpy(), gZ.numpy(), pair.A.dXdalpha.numpy(),
                                      pair.B.dXdalpha.numpy())
    scale = max(np.abs(rA).max(), np.abs(rB).max())
    assert np.abs(gA.cpu().numpy() - rA).max() <= 1e-9 * scale
    assert np.abs(gB.cpu().numpy() - rB).max() <= 1e-9 * scale
    ga = galpha.cpu().numpy()
    assert np.abs(ga - ralpha).max() <= 1e-9 * max(1.0, np.abs(ralpha).max())


def test_backward_central_differences_vertices():
    """d(gP . P + gZ . z)/d(vertex coordinate) by central differences (h = 1e-7)
    of the oracle's narrow-phase solve, for well-conditioned hits."""
    pair = synth.config1()
    XA, XB, A, B, hits = _setup(pair)
    n = len(hits)
    g = torch.Generator().manual_seed(3)
    gP = torch.randn(n, 4, generator=g, dtype=torch.float64)
    gZ = torch.randn(n, 4, generator=g, dtype=torch.float64)
    OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
    rho = hits.rho.cpu().numpy()
    checked = 0
    for h in range(n):
        if rho[h] < 1e-3:
            continue
        gA = torch.zeros_like(XA)
        gB = torch.zeros_like(XB)
        one = tms.Hits(hits.raw[h:h + 1])
        tms.backward(A, B, one, gP=gP[h:h + 1].cuda().contiguous(), gZ=gZ[h:h + 1].cuda().contiguous(),
                     gradA=gA, gradB=gB)
        ta, tb = int(hits.triA[h]), int(hits.triB[h])
        x = oracle.tri_coords(OA, [ta])[0]
        y = oracle.tri_coords(OB, [tb])[0]
        va = oracle.tri_vertex_ids(OA, ta)
        vb = oracle.tri_vertex_ids(OB, tb)

        def f(xx, yy):
            r = oracle.tri_pair(xx, yy)
            return float(np.dot(gP[h].numpy(), r["P"]) + np.dot(gZ[h].numpy(), r["z"]))

        step = 1e-7
        ga, gb = gA.cpu().numpy(), gB.cpu().numpy()
        fd_x = np.zeros((3, 4))
        fd_y = np.zeros((3, 4))
        for j in range(3):
            for c in range(4):
                e = np.zeros((3, 4))
                e[j, c] = step
                fd_x[j, c] = (f(x + e, y) - f(x - e, y)) / (2 * step)
                fd_y[j, c] = (f(x, y + e) - f(x, y - e)) / (2 * step)
        got_x = np.stack([ga[:, v // OA.N, v % OA.N] for v in va])
        got_y = np.stack([gb[:, v // OB.N, v % OB.N] for v in vb])
        scale = max(np.abs(fd_x).max(), np.abs(fd_y).max())
        assert np.abs(got_x - fd_x).max() <= 1e-6 * scale
        assert np.abs(got_y - fd_y).max() <= 1e-6 * scale
        checked += 1
    assert checked >= 4


def test_alpha_derivative_central_differences():
    """d/d alpha of a hit's loss along the alpha family (both meshes move) by
    central differences of the oracle solve on regenerated meshes."""
    seed, alpha, step = 4242, 0.5, 1e-6
    pair = synth.family_pair(seed, alpha)
    XA, XB, A, B, hits = _setup(pair)
    n = len(hits)
    assert n >= 4
    gP = torch.ones(n, 4, dtype=torch.float64)
    gZ = torch.zeros(n, 4, dtype=torch.float64)
    galpha = torch.zeros(n, dtype=torch.float64, device="cuda")
    tms.backward(A, B, hits, gP=gP.cuda(), gZ=gZ.cuda(),
                 dA_dalpha=pair.A.dXdalpha.cuda().contiguous(),
                 dB_dalpha=pair.B.dXdalpha.cuda().contiguous(), galpha=galpha)
    plus = synth.family_pair(seed, alpha + step)
    minus = synth.family_pair(seed, alpha - step)
    ta, tb = hits.triA.cpu().numpy(), hits.triB.cpu().numpy()

    def loss(p):
        OA, OB = oracle.OMesh.from_grid(p.A), oracle.OMesh.from_grid(p.B)
        r = oracle.eval_pairs(OA, OB, ta, tb)
        return r["P"].sum(axis=1)

    fd = (loss(plus) - loss(minus)) / (2 * step)
    got = galpha.cpu().numpy()
    rho = hits.rho.cpu().numpy()
    ok = rho >= 1e-3
    assert ok.sum() >= 4
    assert np.abs(got[ok] - fd[ok]).max() <= 1e-6 * max(1.0, np.abs(fd[ok]).max())


def test_hitpoint_autograd_matches_backward():
    pair = synth.config1()
    XA = pair.A.X.cuda().contiguous().requires_grad_(True)
    XB = pair.B.X.cuda().contiguous().requires_grad_(True)
    A = tms.Mesh(XA.detach(), pair.A.s)
    B = tms.Mesh(XB.detach(), pair.B.s)
    hits = tms.search(A, B)
    P, z = tms.HitPoint.apply(XA, XB, A, B, hits)
    g = torch.Generator().manual_seed(11)
    wP = torch.randn(P.shape, generator=g, dtype=torch.float64).cuda()
    wZ = torch.randn(z.shape, generator=g, dtype=torch.float64).cuda()
    ((P * wP).sum() + (z * wZ).sum()).backward()
    gA = torch.zeros_like(XA.detach())
    gB = torch.zeros_like(XB.detach())
    tms.backward(A, B, hits, gP=wP.contiguous(), gZ=wZ.contiguous(), gradA=gA, gradB=gB)
    assert torch.allclose(XA.grad, gA, rtol=0, atol=1e-12 * float(gA.abs().max()))
    assert torch.allclose(XB.grad, gB, rtol=0, atol=1e-12 * float(gB.abs().max()))
    # translation invariance: the vertex gradients of P alone sum to gP
    gA.zero_()
    gB.zero_()
    tms.backward(A, B, hits, gP=wP.contiguous(), gradA=gA, gradB=gB)
    tot = gA.sum(dim=(1, 2)) + gB.sum(dim=(1, 2))
    assert torch.allclose(tot, wP.sum(dim=0), rtol=1e-10, atol=1e-10)


def test_hitpoint_alpha_gradient_central_differences():
    """d/d alpha through the autograd wrapper: HitPoint with alpha and the
    meshes' dX/d alpha gives alpha's gradient of sum(wP . P + wZ . z) over the
    well-conditioned hits, equal to central differences (h = 1e-7) of the
    oracle's solve on the family members at alpha +- h, to 1e-6 relative."""
    seed, a0, step = 4242, 0.5, 1e-7
    pair = synth.family_pair(seed, a0)
    XA = pair.A.X.cuda().contiguous().requires_grad_(True)
    XB = pair.B.X.cuda().contiguous().requires_grad_(True)
    A = tms.Mesh(XA.detach(), pair.A.s)
    B = tms.Mesh(XB.detach(), pair.B.s)
    hits = tms.search(A, B)
    n = len(hits)
    rho = hits.rho.cpu().numpy()
    ok = rho >= 1e-3
    assert ok.sum() >= 4
    g = torch.Generator().manual_seed(19)
    wP = torch.randn(n, 4, generator=g, dtype=torch.float64)
    wZ = torch.randn(n, 4, generator=g, dtype=torch.float64)
    wP[~torch.as_tensor(ok)] = 0.0
    wZ[~torch.as_tensor(ok)] = 0.0
    alpha = torch.tensor(a0, dtype=torch.float64, device="cuda", requires_grad=True)
    dA = pair.A.dXdalpha.cuda().contiguous()
    dB = pair.B.dXdalpha.cuda().contiguous()
    P, z = tms.HitPoint.apply(XA, XB, A, B, hits, alpha, dA, dB)
    ((P * wP.cuda()).sum() + (z * wZ.cuda()).sum()).backward()
    got = float(alpha.grad)
    ta, tb = hits.triA.cpu().numpy(), hits.triB.cpu().numpy()

    def loss(p):
        OA, OB = oracle.OMesh.from_grid(p.A), oracle.OMesh.from_grid(p.B)
        r = oracle.eval_pairs(OA, OB, ta, tb)
        return float((r["P"] * wP.numpy()).sum() + (r["z"] * wZ.numpy()).sum())

    fd = (loss(synth.family_pair(seed, a0 + step)) - loss(synth.family_pair(seed, a0 - step))) / (2 * step)
    assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (got, fd)
    # the same number as the raw adjoint's per-hit alpha derivatives, summed
    galpha = torch.zeros(n, dtype=torch.float64, device="cuda")
    tms.backward(A, B, hits, gP=wP.cuda(), gZ=wZ.cuda(), dA_dalpha=dA, dB_dalpha=dB, galpha=galpha)
    assert abs(float(galpha.sum()) - got) <= 1e-12 * max(1.0, abs(got))
    # vertex gradients unchanged by the alpha input
    gA = torch.zeros_like(XA.detach())
    tms.backward(A, B, hits, gP=wP.cuda(), gZ=wZ.cuda(), gradA=gA)
    assert torch.allclose(XA.grad, gA, rtol=0, atol=1e-12 * float(gA.abs().max()))
