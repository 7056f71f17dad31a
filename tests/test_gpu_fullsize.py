"""Full-size parity: the benchmark's 4096 x 512 search and the 256-pair batched
sweep, compared with the CPU oracle on every hit.

The oracle's pruned search (exact: a triangle lies inside its box, so pruning by
closed box overlap drops no intersecting pair) gives the complete hit set of
each workload; the GPU answer must equal it outside the near-degeneracy band,
with weights, points and (theta, s) estimates to 1e-10 relative (Sec. 6.2.4,
Eq. (precise)).  The plain form (FP64 boxes and keys, every candidate to the
FP64 solve) must find the identical hit set, and the batched form of the
sweep (one launch sequence over all pairs, Sec. 6.4's loop over half-layer
pairs made one batch) must equal both the oracle and a loop of plain searches,
pair by pair.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2109_14814_gb300 as tms
import synth
from tests.parity import check_sorted_unique, compare, gpu_records

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

PLAIN = dict(precision=0, narrow_filter=0)


def _keys(rec):
    return list(zip(rec["triA"].tolist(), rec["triB"].tolist()))


def test_config3_full_parity_and_plain_form():
    """4096 x 512 meshes in the benchmark's launch configuration: the complete
    hit set against the oracle, planted hits at their closed forms, no planted
    near-miss reported, and the plain FP64 form at the identical hit set."""
    p = synth.config3()
    A = tms.Mesh.from_grid(p.A)
    B = tms.Mesh.from_grid(p.B)
    g = gpu_records(tms.search(A, B))
    torch.cuda.synchronize()
    check_sorted_unique(g)
    OA, OB = oracle.OMesh.from_grid(p.A), oracle.OMesh.from_grid(p.B)
    ref = oracle.search(OA, OB)
    s = compare(OA, OB, g, ref)
    assert s["common"] >= 12000, s
    keys = {k: h for h, k in enumerate(_keys(g))}
    pl = p.planted
    for j in range(len(pl)):
        k = (int(pl.triA[j]), int(pl.triB[j]))
        if int(pl.kind[j]) == 1:
            assert k not in keys
            continue
        h = keys[k]
        assert np.abs(g["z"][h] - pl.abcd[j].numpy()).max() <= 1e-10
        assert np.abs(g["P"][h] - pl.P[j].numpy()).max() <= 1e-10 * max(1, np.abs(pl.P[j].numpy()).max())
    plain = gpu_records(tms.search(A, B, **PLAIN))
    assert _keys(plain) == _keys(g)
    compare(OA, OB, plain, ref)


def test_config4_batched_sweep_parity():
    """The 256 uneven pairs of the alpha sweep in one batched search: each
    pair's slice equals the oracle's search of that pair, and equals a loop of
    plain FP64 searches (precision 0, no FP32 filter) at the identical hit set."""
    n = 256
    sizes = synth.config4_sizes(n_pairs=n)
    pairs = [synth.config4_pair(q, n_pairs=n, sizes=sizes) for q in range(n)]
    As = [tms.Mesh.from_grid(q.A) for q in pairs]
    Bs = [tms.Mesh.from_grid(q.B) for q in pairs]
    out = torch.empty((1 << 17, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    offs_t = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    h = tms.search_batched(As, Bs, out=out, offsets=offs_t)
    rec = gpu_records(h)
    offs = offs_t.cpu().numpy()
    assert offs[0] == 0 and (np.diff(offs) >= 0).all() and offs[-1] == len(h)
    check_sorted_unique(rec)
    total_common = 0
    for q, pair in enumerate(pairs):
        got = {k: v[offs[q]:offs[q + 1]] for k, v in rec.items()}
        assert (got["pair"] == q).all()
        plain = gpu_records(tms.search(As[q], Bs[q], **PLAIN))
        assert _keys(plain) == _keys(got), f"pair {q}: batched and plain hit sets differ"
        OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
        s = compare(OA, OB, got, oracle.search(OA, OB))
        total_common += s["common"]
    assert total_common >= 4 * n
