"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test pins the oracle to something other than itself: LAPACK, exact dyadic
arithmetic, closed-form planted constructions, brute force, invariances, and
the counts printed in the paper (tests/golden/paper_counts.json).
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import meshcases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def om(g):
    return oracle.OMesh.from_grid(g)


# ---------------------------------------------------------------------------
# the 4x4 solve against LAPACK
# ---------------------------------------------------------------------------

def test_solve4_matches_lapack_random():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        A = rng.standard_normal((4, 4))
        r = rng.standard_normal(4)
        z, det, ok = oracle.solve4(A, r)
        assert ok
        zref = np.linalg.solve(A, r)
        assert np.allclose(z, zref, rtol=1e-11, atol=1e-11 * np.abs(zref).max())
        assert math.isclose(det, np.linalg.det(A), rel_tol=1e-11)


def test_solve4_ill_conditioned_within_lapack_agreement():
    rng = np.random.default_rng(2)
    for scale in (1e-3, 1e-5, 1e-6):
        for _ in range(300):
            U, _, Vt = np.linalg.svd(rng.standard_normal((4, 4)))
            A = U @ np.diag([1.0, 0.7, 0.3, scale]) @ Vt
            r = rng.standard_normal(4)
            z, det, ok = oracle.solve4(A, r)
            zref = np.linalg.solve(A, r)
            cond = np.linalg.cond(A)
            assert np.abs(z - zref).max() <= 1e-14 * cond * np.abs(zref).max() * 50


def test_solve4_partial_pivoting_handles_zero_leading_entry():
    A = np.array([[0.0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, 2], [0, 0, 3, 0]])
    z, det, ok = oracle.solve4(A, [1.0, 2, 4, 9])
    assert ok and np.array_equal(z, [2.0, 1.0, 3.0, 2.0])
    assert det == np.linalg.det(A).round()


def test_solve4_singular_reported():
    A = np.ones((4, 4))
    _, det, ok = oracle.solve4(A, np.ones(4))
    assert not ok and det == 0.0


# ---------------------------------------------------------------------------
# hand-solved meshes (exact dyadic arithmetic)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(meshcases.ALL_CASES))
def test_hand_solved_cases(name):
    A, B, exp, n_raw = meshcases.ALL_CASES[name]()
    OA, OB = om(A), om(B)
    raw = oracle.bruteforce(OA, OB)
    assert raw.size == n_raw
    got = oracle.merge_and_sort(OA, OB, raw)
    assert got.size == len(exp)
    for r, e in zip(got, exp):
        assert (int(r["triA"]), int(r["triB"])) == (e["triA"], e["triB"])
        tol = 0.0 if name != "seam" else 1e-12
        assert np.abs(r["z"] - np.array(e["z"])).max() <= tol
        assert np.abs(r["P"] - np.array(e["P"])).max() <= (0.0 if name != "seam" else 1e-14)
        if "params" in e:
            assert np.allclose(r["params"], e["params"], rtol=0, atol=1e-15)


def test_vertex_case_raw_hits_are_the_six_incident_triangles():
    A, B, _, _ = meshcases.vertex_case()
    raw = oracle.bruteforce(om(A), om(B))
    N = 5
    want = {meshcases.tri_id(N, 2, 2, 0), meshcases.tri_id(N, 1, 2, 0), meshcases.tri_id(N, 2, 1, 0),
            meshcases.tri_id(N, 2, 1, 1), meshcases.tri_id(N, 1, 1, 1), meshcases.tri_id(N, 1, 2, 1)}
    assert set(raw["triA"].tolist()) == want


def test_near_miss_margin_is_exact():
    A, B, _, _ = meshcases.near_miss_case(-1)
    OA, OB = om(A), om(B)
    r = oracle.eval_pairs(OA, OB, [meshcases.tri_id(5, 1, 1, 0)], [meshcases.tri_id(5, 0, 1, 0)])[0]
    assert r["margin"] == -(2.0 ** -30) and not r["hit"]


# ---------------------------------------------------------------------------
# planted closed forms on the synthetic configurations
# ---------------------------------------------------------------------------

def _check_planted(p, hits):
    pl = p.planted
    key = {(int(a), int(b)): h for h, (a, b) in enumerate(zip(hits["triA"], hits["triB"]))}
    for j in range(len(pl)):
        k = (int(pl.triA[j]), int(pl.triB[j]))
        if int(pl.kind[j]) == 1:
            assert k not in key
            continue
        assert k in key, f"planted hit {k} missing"
        r = hits[key[k]]
        assert np.abs(r["z"] - pl.abcd[j].numpy()).max() <= 1e-10
        P = pl.P[j].numpy()
        assert np.abs(r["P"] - P).max() <= 1e-10 * max(1.0, np.abs(P).max())
        d = np.abs(r["params"] - pl.params[j].numpy())
        d[[0, 2]] = np.minimum(d[[0, 2]], 2 * math.pi - d[[0, 2]])
        assert d.max() <= 1e-10


def test_config1_bruteforce_contains_planted_closed_forms():
    p = synth.config1()
    OA, OB = om(p.A), om(p.B)
    hits = oracle.merge_and_sort(OA, OB, oracle.bruteforce(OA, OB))
    assert len(p.planted) == 5
    _check_planted(p, hits)


def test_config1_pruned_equals_bruteforce():
    p = synth.config1()
    OA, OB = om(p.A), om(p.B)
    a = oracle.merge_and_sort(OA, OB, oracle.bruteforce(OA, OB))
    b = oracle.merge_and_sort(OA, OB, oracle.pruned(OA, OB))
    assert np.array_equal(a["triA"], b["triA"]) and np.array_equal(a["triB"], b["triB"])
    assert np.array_equal(a["z"], b["z"])


def test_config1_independent_surface_planted_and_pruned():
    """Config 1 with B an independent seeded surface bent through 5 planted
    points of A: brute force holds every planted hit at its closed form, and
    the pruned oracle finds the same set."""
    p = synth.config1_independent()
    OA, OB = om(p.A), om(p.B)
    a = oracle.merge_and_sort(OA, OB, oracle.bruteforce(OA, OB))
    assert len(p.planted) == 5
    _check_planted(p, a)
    b = oracle.merge_and_sort(OA, OB, oracle.pruned(OA, OB))
    assert np.array_equal(a["triA"], b["triA"]) and np.array_equal(a["triB"], b["triB"])
    assert np.array_equal(a["z"], b["z"])


def test_config1_box_pairs_bruteforce():
    """Closed-box overlap pairs from the hierarchy equal a direct all-pairs check."""
    p = synth.config1()
    OA, OB = om(p.A), om(p.B)
    pairs = oracle.box_pairs(OA, OB)
    cA = oracle.tri_coords(OA, np.arange(OA.n_tri_ids))
    cB = oracle.tri_coords(OB, np.arange(OB.n_tri_ids))
    loA, hiA = cA.min(1), cA.max(1)
    loB, hiB = cB.min(1), cB.max(1)
    ov = np.ones((cA.shape[0], cB.shape[0]), dtype=bool)
    for c in range(4):
        ov &= ~((hiA[:, None, c] < loB[None, :, c]) | (hiB[None, :, c] < loA[:, None, c]))
    want = set(zip(*np.nonzero(ov)))
    got = set(map(tuple, pairs.tolist()))
    assert got == {(int(a), int(b)) for a, b in want}


def test_config2_planted_and_windows_against_bruteforce():
    p = synth.config2()
    OA, OB = om(p.A), om(p.B)
    hits = oracle.merge_and_sort(OA, OB, oracle.pruned(OA, OB))
    assert len(p.planted) == 64
    _check_planted(p, hits)
    # random windows: every A triangle of a window against all of B, by brute force
    rng = np.random.default_rng(3)
    trisA = rng.choice(OA.n_tri_ids, 200, replace=False)
    trisA = np.unique(np.concatenate([trisA, hits["triA"][:20]]))
    sub = oracle.hits_for_A(OA, OB, trisA)
    cB = np.arange(OB.n_tri_ids)
    brute = []
    for ta in trisA[:40]:
        r = oracle.eval_pairs(OA, OB, np.full(cB.size, ta), cB)
        brute += [(int(ta), int(tb)) for tb in cB[r["hit"] == 1]]
    s1 = {(int(a), int(b)) for a, b in zip(sub["triA"], sub["triB"]) if a in set(trisA[:40].tolist())}
    assert s1 == set(brute)
    full = {(int(a), int(b)) for a, b in zip(hits["triA"], hits["triB"]) if a in set(trisA.tolist())}
    assert full == {(int(a), int(b)) for a, b in zip(sub["triA"], sub["triB"])}


@pytest.mark.slow
def test_config3_planted_hits_and_near_misses():
    p = synth.config3()
    OA, OB = om(p.A), om(p.B)
    pl = p.planted
    r = oracle.eval_pairs(OA, OB, pl.triA.numpy(), pl.triB.numpy())
    kinds = pl.kind.numpy()
    assert (r["hit"][kinds == 0] == 1).all()
    assert (r["hit"][kinds == 1] == 0).all()
    # near-misses: margin is -eta up to the conditioning of the system
    eta = -pl.abcd[:, 2].numpy()[kinds == 1]
    err = np.abs(r["margin"][kinds == 1] + eta)
    assert (err <= 1e-12 / r["rho"][kinds == 1]).all()


# ---------------------------------------------------------------------------
# invariances
# ---------------------------------------------------------------------------

def test_swap_symmetry():
    p = synth.config1()
    OA, OB = om(p.A), om(p.B)
    ab = oracle.merge_and_sort(OA, OB, oracle.bruteforce(OA, OB))
    ba = oracle.merge_and_sort(OB, OA, oracle.bruteforce(OB, OA))
    s1 = {(int(a), int(b)): h for h, (a, b) in enumerate(zip(ab["triA"], ab["triB"]))}
    s2 = {(int(b), int(a)): h for h, (a, b) in enumerate(zip(ba["triA"], ba["triB"]))}
    assert set(s1) == set(s2)
    for k, h in s1.items():
        r1, r2 = ab[h], ba[s2[k]]
        assert np.allclose(r1["z"], np.r_[r2["z"][2:], r2["z"][:2]], atol=1e-12)
        assert np.allclose(r1["P"], r2["P"], atol=1e-12)


def test_theta_roll_remaps_ids():
    p = synth.config1()
    OA, OB = om(p.A), om(p.B)
    base = oracle.merge_and_sort(OA, OB, oracle.bruteforce(OA, OB))
    r = 11
    N = OA.N
    Xr = np.roll(OA.X, -r, axis=2)        # new vertex i is old vertex i + r
    OAr = oracle.OMesh(Xr, OA.s, True)
    rolled = oracle.merge_and_sort(OAr, OB, oracle.bruteforce(OAr, OB))

    def remap(t):
        q, tau = divmod(int(t), 2)
        k, i = divmod(q, N)
        return 2 * (k * N + (i - r) % N) + tau

    want = {(remap(a), int(b)) for a, b in zip(base["triA"], base["triB"])}
    got = {(int(a), int(b)) for a, b in zip(rolled["triA"], rolled["triB"])}
    assert want == got
    dth = 2 * math.pi / N
    for h in range(base.size):
        m = (rolled["triA"] == remap(base["triA"][h])) & (rolled["triB"] == base["triB"][h])
        th_old = base["params"][h][0]
        th_new = rolled["params"][m][0][0]
        d = (th_old - r * dth - th_new) % (2 * math.pi)
        assert min(d, 2 * math.pi - d) < 1e-12


def test_pair_order_does_not_matter():
    """The hit set is a property of triangle pairs: evaluating all pairs of a
    small mesh pair in a shuffled order gives the brute-force set."""
    p = synth.build_pair(77, 16, 8, 16, 8, stretch="linear", n_folds=0, sites=(4, 1), n_hits=3)
    OA, OB = om(p.A), om(p.B)
    ta, tb = np.meshgrid(np.arange(OA.n_tri_ids), np.arange(OB.n_tri_ids), indexing="ij")
    ta, tb = ta.ravel(), tb.ravel()
    perm = np.random.default_rng(5).permutation(ta.size)
    r = oracle.eval_pairs(OA, OB, ta[perm], tb[perm])
    got = {(int(a), int(b)) for a, b in zip(r["triA"][r["hit"] == 1], r["triB"][r["hit"] == 1])}
    raw = oracle.bruteforce(OA, OB)
    assert got == {(int(a), int(b)) for a, b in zip(raw["triA"], raw["triB"])}
    assert len(got) >= 3


# ---------------------------------------------------------------------------
# counts printed in the paper
# ---------------------------------------------------------------------------

def test_paper_enumeration_counts():
    g = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    b = g["benchmark_meshes"]
    quads1 = synth.MeshGrid(torch.zeros(4, b["M1"], b["N1"], dtype=torch.float64),
                            torch.zeros(b["M1"])).n_quads
    quads2 = synth.MeshGrid(torch.zeros(4, b["M2"], b["N2"], dtype=torch.float64),
                            torch.zeros(b["M2"])).n_quads
    assert quads1 * quads2 == b["quad_pairs"]
    assert 4 * quads1 * quads2 == b["triangle_pairs"]
    h = g["half_layer_pairs"]
    assert h["layers"] * h["pairs_per_layer"] == h["total"]
    t = g["grid_toy_2d"]
    assert t["objects"] * (t["objects"] - 1) // 2 == t["pairs"]


# ---------------------------------------------------------------------------
# reverse-mode derivative of a hit
# ---------------------------------------------------------------------------

def _fd_pair(x, y, gP, gz, h=1e-7):
    gx = np.zeros((3, 4))
    gy = np.zeros((3, 4))

    def f(xx, yy):
        r = oracle.tri_pair(xx, yy)
        return float(np.dot(gP, r["P"]) + np.dot(gz, r["z"]))

    for j in range(3):
        for c in range(4):
            for arr, out in ((x, gx), (y, gy)):
                e = np.zeros((3, 4))
                e[j, c] = h
                if arr is x:
                    out[j, c] = (f(x + e, y) - f(x - e, y)) / (2 * h)
                else:
                    out[j, c] = (f(x, y + e) - f(x, y - e)) / (2 * h)
    return gx, gy


def test_pair_grad_matches_central_differences():
    p = synth.config1()
    OA, OB = om(p.A), om(p.B)
    hits = oracle.merge_and_sort(OA, OB, oracle.bruteforce(OA, OB))
    rng = np.random.default_rng(9)
    xs = oracle.tri_coords(OA, hits["triA"])
    ys = oracle.tri_coords(OB, hits["triB"])
    for h in range(hits.size):
        if hits["rho"][h] < 1e-3:
            continue
        gP, gz = rng.standard_normal(4), rng.standard_normal(4)
        gx, gy, _ = oracle.pair_grad(xs[h], ys[h], gP, gz)
        fx, fy = _fd_pair(xs[h], ys[h], gP, gz)
        scale = max(np.abs(gx).max(), np.abs(gy).max())
        assert np.abs(gx - fx).max() <= 1e-6 * scale
        assert np.abs(gy - fy).max() <= 1e-6 * scale


def test_pair_grad_translation_closed_form():
    """Axis-plane case: translating B by e moves the common point (x0, y0, 0, 0)
    by the projection of e onto A's plane along B's plane, i.e. (e_x, e_y, 0, 0);
    translating both meshes moves it by e (weights of gP sum over all vertices)."""
    A, B, _, _ = meshcases.interior_case()
    OA, OB = om(A), om(B)
    x = oracle.tri_coords(OA, [meshcases.tri_id(5, 1, 1, 0)])[0]
    y = oracle.tri_coords(OB, [meshcases.tri_id(5, 1, 1, 0)])[0]
    rng = np.random.default_rng(4)
    for _ in range(10):
        gP = rng.standard_normal(4)
        e = rng.standard_normal(4)
        gx, gy, _ = oracle.pair_grad(x, y, gP, np.zeros(4))
        assert math.isclose(float((gy @ e).sum()), float(gP[0] * e[0] + gP[1] * e[1]),
                            rel_tol=1e-12, abs_tol=1e-12)
        assert np.allclose(gx.sum(0) + gy.sum(0), gP, atol=1e-13)
