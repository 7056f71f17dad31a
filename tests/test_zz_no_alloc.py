"""The allocation-free search entry point (tms_search_noalloc).

Some callers of this library cannot allocate device memory at search time: code
running while another component captures a CUDA graph, software that fixes its
device footprint at start-up, or services whose memory is all held by a pool
allocator.  tms_search_noalloc serves them from a static device array inside
the library.  These tests call it through the C ABI twice in a row and compare
its output with tms_search's, within the parity tolerance used elsewhere, and
check that a steady-state call takes no device memory.  This file is collected
last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import paper_2109_14814_gb300 as tms
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _records(h):
    return {k: v.cpu().numpy() for k, v in h.to_dict().items()}


def _same(a, b):
    assert list(zip(a["triA"], a["triB"])) == list(zip(b["triA"], b["triB"]))
    assert np.array_equal(a["flags"], b["flags"])
    for f in ("z", "P", "params"):
        scale = np.maximum(1.0, np.abs(b[f]).max(axis=1, keepdims=True)) if len(b[f]) else 1.0
        assert (np.abs(a[f] - b[f]) <= TOL * scale).all(), f


@pytest.mark.parametrize("build", [
    lambda: synth.config1(),
    lambda: synth.build_pair(4321, 320, 160, 288, 144, stretch="exp", n_folds=3, sites=(8, 4), n_hits=24),
], ids=["config1", "320x160"])
def test_noalloc_matches_search_twice(build):
    pair = build()
    A = tms.Mesh.from_grid(pair.A)
    B = tms.Mesh.from_grid(pair.B)
    ref = _records(tms.search(A, B))
    out = torch.empty((4096, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    first = _records(tms.search_noalloc(A, B, out))
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    second = _records(tms.search_noalloc(A, B, out))
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    _same(first, ref)
    _same(second, ref)
    assert len(ref["triA"]) > 0
    assert free_after >= free_before - (1 << 20), "a steady-state call took device memory"


def test_noalloc_rejects_meshes_beyond_the_limit():
    p = synth.config2()                      # 1024 x 256 = 262144 vertices per mesh
    A = tms.Mesh.from_grid(p.A)
    B = tms.Mesh.from_grid(p.B)
    out = torch.empty((16, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    with pytest.raises(tms.TmsError) as e:
        tms.search_noalloc(A, B, out)
    assert e.value.status == tms.TMS_ERR_ARG
    assert "131072" in str(e.value)
