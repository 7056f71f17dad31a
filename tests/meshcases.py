"""Hand-built mesh pairs with intersections known in closed form (test inputs).

These constructors only place vertices; the expected results are derived by
hand in each docstring.  They feed both the CPU oracle tests and the GPU
parity tests.

Planar cases: A lies in the (x, y) plane, B in the plane (x0, y0) + span(px, py),
both as open strips with spacing 1/4, so the only common point of the two planes
is (x0, y0, 0, 0) and every weight is an exact dyadic number.
"""
from __future__ import annotations

import math

import torch

from synth import MeshGrid

H = 0.25


def _planar_A(N=5, M=5):
    X = torch.zeros(4, M, N, dtype=torch.float64)
    i = torch.arange(N, dtype=torch.float64)
    k = torch.arange(M, dtype=torch.float64)
    X[0] = (i * H)[None, :].expand(M, N)
    X[1] = (k * H)[:, None].expand(M, N)
    s = k * H
    return MeshGrid(X, s, periodic=False)


def _planar_B(x0, y0, ox, oy, N=5, M=5):
    X = torch.zeros(4, M, N, dtype=torch.float64)
    j = torch.arange(N, dtype=torch.float64)
    l = torch.arange(M, dtype=torch.float64)
    X[0] = x0
    X[1] = y0
    X[2] = (j * H - ox)[None, :].expand(M, N)
    X[3] = (l * H - oy)[:, None].expand(M, N)
    s = l * H
    return MeshGrid(X, s, periodic=False)


def tri_id(N, i, k, tau):
    return 2 * (k * N + i) + tau


def interior_case():
    """A point (5/16, 9/32): quad (1, 1) of A, cell fractions (1/4, 1/8) -> T1 with
    (a, b) = (1/4, 1/8).  B point (px, py) = 0 at j = 3/2, l = 5/4: quad (1, 1),
    fractions (1/2, 1/4) -> T1 with (c, d) = (1/2, 1/4).  One hit, point
    (5/16, 9/32, 0, 0); theta_u = 2 pi (1 + 1/4) / 5, s_u = 9/32,
    theta_s = 2 pi (1 + 1/2) / 5, s_s = 5/16."""
    A = _planar_A()
    B = _planar_B(5 / 16, 9 / 32, 3 / 8, 5 / 16)
    exp = [dict(triA=tri_id(5, 1, 1, 0), triB=tri_id(5, 1, 1, 0),
                z=(0.25, 0.125, 0.5, 0.25), P=(5 / 16, 9 / 32, 0.0, 0.0),
                params=(2 * math.pi * 1.25 / 5, 9 / 32, 2 * math.pi * 1.5 / 5, 5 / 16))]
    return A, B, exp, 1


def diagonal_case():
    """A point (7/16, 5/16): quad (1, 1), fractions (3/4, 1/4), on the T1/T2
    diagonal.  T1 gives (a, b) = (3/4, 1/4), T2 gives (1/4, 3/4); both margins
    are exactly 0, so two raw hits, merged into one (the smaller triA, T1)."""
    A = _planar_A()
    B = _planar_B(7 / 16, 5 / 16, 3 / 8, 5 / 16)
    exp = [dict(triA=tri_id(5, 1, 1, 0), triB=tri_id(5, 1, 1, 0),
                z=(0.75, 0.25, 0.5, 0.25), P=(7 / 16, 5 / 16, 0.0, 0.0))]
    return A, B, exp, 2


def vertex_case():
    """A point (1/2, 1/2) is grid vertex (2, 2) of A, shared by six triangles:
    T1(2,2), T1(1,2), T1(2,1), T2(2,1), T2(1,1), T2(1,2).  Six raw hits, merged
    into one: the smallest id, T2(1,1) = 13, where the vertex is x2 (a = b = 0)."""
    A = _planar_A()
    B = _planar_B(0.5, 0.5, 3 / 8, 5 / 16)
    exp = [dict(triA=tri_id(5, 1, 1, 1), triB=tri_id(5, 1, 1, 0),
                z=(0.0, 0.0, 0.5, 0.25), P=(0.5, 0.5, 0.0, 0.0))]
    return A, B, exp, 6


def coplanar_case():
    """B lies in A's plane and overlaps it: every system is singular -> no hit."""
    A = _planar_A()
    X = torch.zeros(4, 5, 5, dtype=torch.float64)
    j = torch.arange(5, dtype=torch.float64)
    X[0] = (j * H - 3 / 16)[None, :]
    X[1] = (j * H - 5 / 32)[:, None]
    B = MeshGrid(X, j * H, periodic=False)
    return A, B, [], 0


def parallel_case():
    """B is A shifted by 1/4 along px: parallel planes, singular -> no hit."""
    A = _planar_A()
    X = A.X.clone()
    X[2] += 0.25
    return A, MeshGrid(X, A.s.clone(), periodic=False), [], 0


def near_miss_case(sign: int):
    """B's strip starts at j = 0 with px = -ox; the common point has
    c = 4 ox = sign * 2**-30 in T1(0, 1) of B.  sign = -1: the point is 2**-30
    outside B (no B triangle contains it) -> no hit; sign = +1: one hit with
    c = 2**-30."""
    A = _planar_A()
    c = sign * 2.0 ** -30
    B = _planar_B(5 / 16, 9 / 32, c / 4.0, 5 / 16)
    if sign < 0:
        return A, B, [], 0
    exp = [dict(triA=tri_id(5, 1, 1, 0), triB=tri_id(5, 0, 1, 0),
                z=(0.25, 0.125, c, 0.25), P=(5 / 16, 9 / 32, 0.0, 0.0))]
    return A, B, exp, 1


def seam_case(N=16, M=4):
    """A periodic cylinder A(theta, s) = (cos theta, sin theta, s, 0) and a small
    planar patch B through a point of the seam quad (i = N-1, k = 1), which
    joins vertex N-1 to vertex 0.  The point is placed at weights (a, b) =
    (3/8, 1/4) of T1 of that quad; B spans py and the chord normal and holds the
    point at (c, d) = (1/4, 1/2) of its T1(1, 1)."""
    th = torch.arange(N, dtype=torch.float64) * (2 * math.pi / N)
    s = torch.arange(M, dtype=torch.float64) * H
    XA = torch.zeros(4, M, N, dtype=torch.float64)
    XA[0] = torch.cos(th)[None, :]
    XA[1] = torch.sin(th)[None, :]
    XA[2] = s[:, None]
    A = MeshGrid(XA, s, periodic=True)
    i, k = N - 1, 1
    x2 = XA[:, k, i]
    x1 = XA[:, k, 0]
    x3 = XA[:, k + 1, i]
    a, b = 0.375, 0.25
    P = (1 - a - b) * x2 + a * x1 + b * x3
    chord = x1 - x2
    n = torch.tensor([chord[1].item(), -chord[0].item(), 0.0, 0.0], dtype=torch.float64)
    n = n / n.norm()
    e_py = torch.tensor([0, 0, 0, 1.0], dtype=torch.float64)
    hb = 0.125
    c, d = 0.25, 0.5
    XB = torch.zeros(4, 4, 4, dtype=torch.float64)
    for l in range(4):
        for j in range(4):
            XB[:, l, j] = P + ((j - 1) - c) * hb * e_py + ((l - 1) - d) * hb * n
    B = MeshGrid(XB, torch.arange(4, dtype=torch.float64) * hb, periodic=False)
    exp = [dict(triA=tri_id(N, i, k, 0), triB=tri_id(4, 1, 1, 0), z=(a, b, c, d),
                P=tuple(P.tolist()))]
    return A, B, exp, 1


ALL_CASES = {
    "interior": interior_case,
    "diagonal": diagonal_case,
    "vertex": vertex_case,
    "coplanar": coplanar_case,
    "parallel": parallel_case,
    "near_miss_out": lambda: near_miss_case(-1),
    "near_miss_in": lambda: near_miss_case(+1),
    "seam": seam_case,
}
