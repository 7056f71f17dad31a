"""Parity rule between the CUDA search and the CPU oracle (test helper).

Outside the near-degeneracy band (rho < 1e-12 or |margin| < 1e-12, evaluated by
the oracle) the hit pair sets must be identical; for pairs found by both, the
weights (a, b, c, d), the point P and the (theta, s) estimates must agree to
1e-10 relative (theta compared on the circle).
"""
from __future__ import annotations

import math

import numpy as np

import oracle

BAND = 1e-12
TOL = 1e-10


def gpu_records(hits):
    d = hits.to_dict()
    return {k: v.cpu().numpy() for k, v in d.items()}


def compare(OA, OB, gpu, ref, tau=oracle.TAU, restrict_A=None):
    """Check the parity rule; returns a summary dict.  `gpu` from gpu_records,
    `ref` a merged oracle record array.  restrict_A limits both sides to a set
    of A triangles (sampled parity)."""
    g_keys = list(zip(gpu["triA"].tolist(), gpu["triB"].tolist()))
    o_keys = list(zip(ref["triA"].tolist(), ref["triB"].tolist()))
    if restrict_A is not None:
        ra = set(int(t) for t in restrict_A)
        gi = [h for h, k in enumerate(g_keys) if k[0] in ra]
        oi = [h for h, k in enumerate(o_keys) if k[0] in ra]
    else:
        gi = list(range(len(g_keys)))
        oi = list(range(len(o_keys)))
    gset = {g_keys[h]: h for h in gi}
    oset = {o_keys[h]: h for h in oi}
    only_g = [k for k in gset if k not in oset]
    only_o = [k for k in oset if k not in gset]
    band_g = 0
    if only_g:
        r = oracle.eval_pairs(OA, OB, [k[0] for k in only_g], [k[1] for k in only_g], tau)
        inb = oracle.in_band(r, BAND)
        bad = [only_g[i] for i in np.nonzero(~inb)[0]]
        assert not bad, f"GPU-only hits outside the band: {bad[:5]} (of {len(bad)})"
        band_g = len(only_g)
    if only_o:
        r = ref[[oset[k] for k in only_o]]
        inb = oracle.in_band(r, BAND)
        bad = [only_o[i] for i in np.nonzero(~inb)[0]]
        assert not bad, f"oracle hits missed by the GPU outside the band: {bad[:5]} (of {len(bad)})"
    common = [k for k in gset if k in oset]
    max_z = max_p = max_t = 0.0
    for k in common:
        g, o = gset[k], oset[k]
        zg, zo = gpu["z"][g], ref["z"][o]
        if oracle.in_band(ref[o:o + 1], BAND)[0]:
            continue
        dz = np.abs(zg - zo).max() / max(1.0, np.abs(zo).max())
        dp = np.abs(gpu["P"][g] - ref["P"][o]).max() / max(1.0, np.abs(ref["P"][o]).max())
        d = np.abs(gpu["params"][g] - ref["params"][o])
        d[[0, 2]] = np.minimum(d[[0, 2]], 2 * math.pi - d[[0, 2]])
        dt = d.max() / max(1.0, np.abs(ref["params"][o]).max())
        max_z, max_p, max_t = max(max_z, dz), max(max_p, dp), max(max_t, dt)
    assert max_z <= TOL, f"weights differ by {max_z}"
    assert max_p <= TOL, f"points differ by {max_p}"
    assert max_t <= TOL, f"(theta, s) estimates differ by {max_t}"
    return dict(common=len(common), only_gpu=len(only_g), only_oracle=len(only_o),
                band=band_g + len(only_o), max_z=max_z, max_p=max_p, max_t=max_t)


def check_sorted_unique(gpu):
    keys = list(zip(gpu["pair"].tolist(), gpu["triA"].tolist(), gpu["triB"].tolist()))
    assert keys == sorted(keys), "hits not sorted by (pair, triA, triB)"
    assert len(set(keys)) == len(keys), "duplicate hit records"
