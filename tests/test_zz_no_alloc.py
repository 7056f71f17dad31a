"""The allocation-free search entry point (tms_search_noalloc).

Some callers of this library cannot allocate device memory at search time:
software that fixes its device footprint at start-up and forbids allocation
afterwards, or services whose device memory is all held by a pool allocator.
tms_search_noalloc serves them from a static device array inside the library.
These tests call it through the C ABI several times in a row and check each
result against the CPU oracle (the parity rule of the other search tests) and,
bit for bit, against tms_search, which runs the same kernels on allocated
scratch.  They also check that a call after a larger call, and a call after one
that overflowed the static limits, are still exact, and that a steady-state
call takes no device memory.  This file is collected last so that a failure
here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2109_14814_gb300 as tms
import synth
from tests.parity import compare

pytestmark = pytest.mark.gpu


def _records(h):
    return {k: v.cpu().numpy() for k, v in h.to_dict().items()}


def _identical(a, b):
    """Bit-exact equality of two hit record sets (same kernels, same inputs)."""
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def _check(pair, got):
    """got against tms_search (bit for bit) and the oracle (parity rule)."""
    A = tms.Mesh.from_grid(pair.A)
    B = tms.Mesh.from_grid(pair.B)
    _identical(got, _records(tms.search(A, B)))
    OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
    compare(OA, OB, got, oracle.search(OA, OB))


def _noalloc(pair, out):
    A = tms.Mesh.from_grid(pair.A)
    B = tms.Mesh.from_grid(pair.B)
    return _records(tms.search_noalloc(A, B, out))


def _pair_320x160():
    return synth.build_pair(4321, 320, 160, 288, 144, stretch="exp", n_folds=3, sites=(8, 4), n_hits=24)


def _dense_pair():
    """Two 40 x 20 vertex meshes inside one small ball: nearly every one of the
    760 x 760 quad pairs has overlapping boxes, far more than the static
    candidate limit (262144) allows."""
    g0 = torch.Generator().manual_seed(23)
    XA = 0.01 * torch.randn(4, 20, 40, generator=g0, dtype=torch.float64)
    XB = 0.01 * torch.randn(4, 20, 40, generator=g0, dtype=torch.float64)
    s = torch.linspace(0.0, 1.0, 20, dtype=torch.float64)
    return synth.MeshPair(synth.MeshGrid(XA, s), synth.MeshGrid(XB, s), None)


@pytest.mark.parametrize("build", [synth.config1, _pair_320x160], ids=["config1", "320x160"])
def test_noalloc_matches_oracle_twice(build):
    pair = build()
    out = torch.empty((4096, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    first = _noalloc(pair, out)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    second = _noalloc(pair, out)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert len(first["triA"]) > 0
    _check(pair, first)
    _check(pair, second)
    assert free_after >= free_before - (1 << 20), "a steady-state call took device memory"


def test_noalloc_smaller_call_after_larger_call():
    """State a larger call leaves in the shared array (cell table, counters,
    bitmaps) must not leak into a smaller call, nor a tms_search in between."""
    out = torch.empty((4096, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    big, small = _pair_320x160(), synth.config1()
    _check(big, _noalloc(big, out))
    _check(small, _noalloc(small, out))
    _check(big, _noalloc(big, out))
    _check(small, _noalloc(small, out))


def test_noalloc_overflow_then_exact():
    """A call whose candidates exceed the static limit returns TMS_ERR_CAPACITY
    with *nHits = -1 and grows nothing; the next call is still exact, so the
    overflowing call left the cell table free."""
    dense = _dense_pair()
    out = torch.empty((4096, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    A = tms.Mesh.from_grid(dense.A)
    B = tms.Mesh.from_grid(dense.B)
    for _ in range(2):
        with pytest.raises(tms.TmsError) as e:
            tms.search_noalloc(A, B, out)
        assert e.value.status == tms.TMS_ERR_CAPACITY
        assert "static scratch limits" in str(e.value)
        small = synth.config1()
        _check(small, _noalloc(small, out))


def test_noalloc_rejects_meshes_beyond_the_limit():
    p = synth.config2()                      # 1024 x 256 = 262144 vertices per mesh
    A = tms.Mesh.from_grid(p.A)
    B = tms.Mesh.from_grid(p.B)
    out = torch.empty((16, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    with pytest.raises(tms.TmsError) as e:
        tms.search_noalloc(A, B, out)
    assert e.value.status == tms.TMS_ERR_ARG
    assert "131072" in str(e.value)
