"""CPU oracle of the method of layers -- TEST INFRASTRUCTURE ONLY (the tests and
the benchmark's CPU leg may call it; the CUDA path never does).

Sec. 5 defines half-layers of the globalized manifolds by intervals of s:
    U_n^+ = W^u(T x [D_u lam_u^(n-1), D_u lam_u^n]),   U_n^- = the same with -D_u,
    S_n^+ = W^s(T x [D_s / lam_s^(n-1), D_s / lam_s^n]), S_n^- likewise,
and Eq. (layerintersection) moves any heteroclinic point along its orbit into
some U_n cap S_n or U_n cap S_(n-1), n >= 1.  Sec. 6.2 notes that the
boundaries +-D lam^n are among the stored s values, so a half-layer is the
contiguous set of vertex columns whose s lies in its interval, and searches the
eight half-layer pairs (U_n^+-, S_n^+-), (U_n^+-, S_(n-1)^+-) of each layer
n = 1..n_max.

The expected output of a layer sweep is written two ways here: the hits of the
full-mesh search (oracle.search) kept when the A triangle's quad lies in some
U half-layer and the B triangle's quad in an S half-layer forming one of the
pairs (`sweep`), and the concatenated searches of the column-range submeshes
(`sweep_by_pairs`).  Pair order: n ascending, then U sign (+ before -), then
m = n before m = n - 1, then S sign (+ before -).  Triangle ids in the output
are those of the full meshes.
"""
from __future__ import annotations

import numpy as np

import oracle


def layer_shift(n1: int, n2: int):
    """Eq. (layerintersection): a point of U_n1 cap S_n2 maps under F^k into
    U_(n1+k) cap S_(n2-k).  Returns (k, n, m) with (U_n, S_m) one of the
    searched forms: m = n for n1, n2 of equal parity, m = n - 1 otherwise."""
    if (n1 - n2) % 2 == 0:
        k = (n2 - n1) // 2
        n = (n1 + n2) // 2
        return k, n, n
    k = (n2 - n1 + 1) // 2
    n = (n1 + n2 + 1) // 2
    return k, n, n - 1


def half_layer(s, lo: float, hi: float, rel_tol: float = 1e-9):
    """Vertex columns [k0, k1) whose s lies in the closed interval [lo, hi]; the
    interval's ends must be stored s values (within rel_tol)."""
    s = np.asarray(s, dtype=np.float64)
    lo, hi = min(lo, hi), max(lo, hi)
    inside = (s >= lo - rel_tol * abs(lo)) & (s <= hi + rel_tol * abs(hi))
    cols = np.nonzero(inside)[0]
    if cols.size < 2:
        raise ValueError(f"half-layer [{lo}, {hi}] holds fewer than two columns")
    k0, k1 = int(cols[0]), int(cols[-1]) + 1
    if cols.size != k1 - k0:
        raise ValueError("half-layer columns are not contiguous")
    if abs(s[k0] - lo) > rel_tol * abs(lo) or abs(s[k1 - 1] - hi) > rel_tol * abs(hi):
        raise ValueError(f"boundary of [{lo}, {hi}] is not a stored s value")
    return k0, k1


def layer_pairs(sA, D_u: float, lam_u: float, sB, D_s: float, lam_s: float, n_max: int,
                rel_tol: float = 1e-9):
    """The 8 n_max half-layer pairs of Sec. 6.2 as dicts with n, m, sign_u,
    sign_s and the column ranges a = (k0, k1) in A, b = (k0, k1) in B."""
    out = []
    for n in range(1, n_max + 1):
        for su in (1, -1):
            a = half_layer(sA, su * D_u * lam_u ** (n - 1), su * D_u * lam_u ** n, rel_tol)
            for m in (n, n - 1):
                for ss in (1, -1):
                    b = half_layer(sB, ss * D_s / lam_s ** (m - 1), ss * D_s / lam_s ** m, rel_tol)
                    out.append(dict(n=n, m=m, sign_u=su, sign_s=ss, a=a, b=b))
    return out


def _quad_col(tri, N: int):
    return (np.asarray(tri, dtype=np.int64) // 2) // N


def sweep(A: "oracle.OMesh", B: "oracle.OMesh", pairs, full=None):
    """Expected sweep output from the full-mesh search: (records, pair index),
    sorted by (pair, triA, triB).  A hit belongs to pair p when its A quad's
    two columns lie in p's A range and its B quad's in p's B range."""
    recs = oracle.search(A, B) if full is None else full
    ka, kb = _quad_col(recs["triA"], A.N), _quad_col(recs["triB"], B.N)
    pid = np.full(len(recs), -1, dtype=np.int64)
    for p, pr in enumerate(pairs):
        (a0, a1), (b0, b1) = pr["a"], pr["b"]
        sel = (ka >= a0) & (ka + 1 < a1) & (kb >= b0) & (kb + 1 < b1)
        assert not (pid[sel] >= 0).any(), "a hit in two half-layer pairs"
        pid[sel] = p
    keep = pid >= 0
    recs, pid = recs[keep], pid[keep]
    order = np.lexsort((recs["triB"], recs["triA"], pid))
    return recs[order], pid[order]


def sweep_by_pairs(A: "oracle.OMesh", B: "oracle.OMesh", pairs):
    """The same output from one search per half-layer pair on the column-range
    submeshes, triangle ids shifted to the full meshes."""
    all_recs, all_pid = [], []
    for p, pr in enumerate(pairs):
        (a0, a1), (b0, b1) = pr["a"], pr["b"]
        SA = oracle.OMesh(A.X[:, a0:a1], A.s[a0:a1], A.periodic)
        SB = oracle.OMesh(B.X[:, b0:b1], B.s[b0:b1], B.periodic)
        r = oracle.search(SA, SB)
        r["triA"] += 2 * A.N * a0
        r["triB"] += 2 * B.N * b0
        all_recs.append(r)
        all_pid.append(np.full(len(r), p, dtype=np.int64))
    recs = np.concatenate(all_recs) if all_recs else np.zeros(0, dtype=oracle.REC_DTYPE)
    pid = np.concatenate(all_pid) if all_pid else np.zeros(0, dtype=np.int64)
    order = np.lexsort((recs["triB"], recs["triA"], pid))
    return recs[order], pid[order]
