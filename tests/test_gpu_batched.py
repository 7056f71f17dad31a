"""Batched search of many uneven mesh pairs in one launch sequence (CUDA graph):
per-pair results equal the single search and the oracle, offsets partition the
output, and replaying the graph after the vertex data change in place gives the
new answers."""
import numpy as np
import pytest
import torch

import oracle
import paper_2109_14814_gb300 as tms
import synth
from tests.parity import compare, gpu_records

pytestmark = pytest.mark.gpu

SIZES = [(160, 40, 200, 48), (300, 64, 128, 32), (128, 32, 256, 80), (512, 96, 384, 64),
         (200, 50, 220, 60), (256, 32, 128, 128), (180, 70, 360, 40), (420, 36, 150, 90)]


def _pairs(alpha_shift=0.0):
    return [synth.config4_pair(p, n_pairs=len(SIZES), sizes=SIZES) if alpha_shift == 0.0 else
            synth.build_pair(synth.config_seed(4) * 1000 + p, *SIZES[p], stretch="exp", lam=4.0,
                             n_folds=3, sites=(8, 2), n_hits=4,
                             alpha=p / (len(SIZES) - 1) + alpha_shift, with_dalpha=True,
                             family_seed=synth.config_seed(4))
            for p in range(len(SIZES))]


def _split(h):
    offs = h.offsets.cpu().numpy()
    rec = gpu_records(h)
    return offs, [{k: v[offs[p]:offs[p + 1]] for k, v in rec.items()} for p in range(len(offs) - 1)]


def test_batched_equals_single_and_oracle():
    pairs = _pairs()
    As = [tms.Mesh.from_grid(p.A) for p in pairs]
    Bs = [tms.Mesh.from_grid(p.B) for p in pairs]
    h = tms.search_batched(As, Bs)
    offs, per = _split(h)
    assert offs[0] == 0 and (np.diff(offs) >= 0).all() and offs[-1] == len(h)
    total = 0
    for p, pair in enumerate(pairs):
        got = per[p]
        assert (got["pair"] == p).all()
        single = gpu_records(tms.search(As[p], Bs[p]))
        assert list(zip(got["triA"], got["triB"])) == list(zip(single["triA"], single["triB"]))
        assert np.array_equal(got["z"], single["z"]) and np.array_equal(got["P"], single["P"])
        OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
        compare(OA, OB, got, oracle.search(OA, OB))
        total += len(got["triA"])
    assert total >= 4 * len(pairs)


def test_batched_graph_replay_after_in_place_update():
    pairs = _pairs()
    XA = [p.A.X.cuda().contiguous() for p in pairs]
    XB = [p.B.X.cuda().contiguous() for p in pairs]
    As = [tms.Mesh(x, p.A.s) for x, p in zip(XA, pairs)]
    Bs = [tms.Mesh(x, p.B.s) for x, p in zip(XB, pairs)]
    out = torch.empty((1 << 14, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    offsets = torch.empty(len(pairs) + 1, dtype=torch.int64, device="cuda")
    first = gpu_records(tms.search_batched(As, Bs, out=out, offsets=offsets))
    again = gpu_records(tms.search_batched(As, Bs, out=out, offsets=offsets))
    for k in first:
        assert np.array_equal(first[k], again[k])
    # the next step of the sweep: new alpha, same buffers, same (replayed) graph
    moved = _pairs(alpha_shift=0.01)
    for x, y, p in zip(XA, XB, moved):
        x.copy_(p.A.X.cuda())
        y.copy_(p.B.X.cuda())
    h = tms.search_batched(As, Bs, out=out, offsets=offsets)
    offs, per = _split(h)
    for p, pair in enumerate(moved):
        OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
        compare(OA, OB, per[p], oracle.search(OA, OB))
