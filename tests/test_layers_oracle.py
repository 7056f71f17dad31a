"""Pins of the method-of-layers oracle (oracle/layers.py, Sec. 5 Eq.
layerintersection and Sec. 6.2): the orbit-shift arithmetic, the half-layer
column ranges against their closed-form boundaries, the paper's printed pair
counts, and the two formulations of a sweep against each other."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import layers as L

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_counts.json")


def test_orbit_shift_lands_in_a_searched_pair():
    # F^k(x) in U_(n1+k) cap S_(n2-k), and the chosen k gives (U_n, S_n) or (U_n, S_(n-1))
    for n1 in range(1, 31):
        for n2 in range(1, 31):
            k, n, m = L.layer_shift(n1, n2)
            assert n1 + k == n and n2 - k == m
            assert m in (n, n - 1) and n >= 1
            assert (m == n) == ((n1 - n2) % 2 == 0)
            # time of flight n1 + n2 maps is kept by the shift
            assert n + m == n1 + n2


def _small():
    return synth.layered_pair(NA=96, NB=128, n_max=3, per_layer=8, sites=(8, 6), n_hits=12)


def _pairs(p):
    lay = p.meta["layers"]
    return L.layer_pairs(p.A.s.numpy(), lay["D_u"], lay["lam_u"], p.B.s.numpy(), lay["D_s"],
                         lay["lam_s"], lay["n_max"])


def test_half_layer_ranges_match_their_boundaries():
    p = _small()
    lay = p.meta["layers"]
    pairs = _pairs(p)
    assert len(pairs) == 8 * lay["n_max"]
    sA, sB = p.A.s.numpy(), p.B.s.numpy()
    for pr in pairs:
        n, m, su, ss = pr["n"], pr["m"], pr["sign_u"], pr["sign_s"]
        (a0, a1), (b0, b1) = pr["a"], pr["b"]
        ua = sorted([su * lay["D_u"] * lay["lam_u"] ** (n - 1), su * lay["D_u"] * lay["lam_u"] ** n])
        sb = sorted([ss * lay["D_s"] / lay["lam_s"] ** (m - 1), ss * lay["D_s"] / lay["lam_s"] ** m])
        assert np.allclose([sA[a0], sA[a1 - 1]], ua, rtol=1e-12)
        assert np.allclose([sB[b0], sB[b1 - 1]], sb, rtol=1e-12)
        assert a1 - a0 == lay["per_layer"] + 1 and b1 - b0 == lay["per_layer"] + 1
    # mirror symmetry of the two signs, and consecutive half-layers share one column
    by = {(pr["n"], pr["sign_u"]): pr["a"] for pr in pairs}
    MA = sA.size
    for n in range(1, lay["n_max"] + 1):
        (p0, p1), (q0, q1) = by[(n, 1)], by[(n, -1)]
        assert (q0, q1) == (MA - p1, MA - p0)
        if n > 1:
            assert by[(n - 1, 1)][1] - 1 == p0
    with pytest.raises(ValueError):
        L.half_layer(sA, 0.3 * lay["D_u"], lay["D_u"])        # 0.3 D_u is not a stored value


def test_paper_benchmark_pair_counts():
    g = json.load(open(GOLDEN))
    bm, hl = g["benchmark_meshes"], g["half_layer_pairs"]
    p = synth.layered_pair()          # the paper's shapes
    pairs = _pairs(p)
    assert len(pairs) == hl["total"] == hl["layers"] * hl["pairs_per_layer"]
    for pr in pairs:
        (a0, a1), (b0, b1) = pr["a"], pr["b"]
        assert (a1 - a0, b1 - b0) == (bm["M1"], bm["M2"])
        quads = (p.A.N * (a1 - a0 - 1)) * (p.B.N * (b1 - b0 - 1))
        assert quads == bm["quad_pairs"] and 4 * quads == bm["triangle_pairs"]


def test_sweep_filter_equals_per_pair_searches():
    p = _small()
    A, B = oracle.OMesh.from_grid(p.A), oracle.OMesh.from_grid(p.B)
    pairs = _pairs(p)
    r1, p1 = L.sweep(A, B, pairs)
    r2, p2 = L.sweep_by_pairs(A, B, pairs)
    assert len(r1) > 20 and len(set(p1.tolist())) > 5
    assert np.array_equal(p1, p2)
    assert np.array_equal(r1["triA"], r2["triA"]) and np.array_equal(r1["triB"], r2["triB"])
    assert np.abs(r1["P"] - r2["P"]).max() <= 1e-12 * max(1.0, np.abs(r1["P"]).max())
    assert np.abs(r1["params"] - r2["params"]).max() <= 1e-12 * max(1.0, np.abs(r1["params"]).max())
