"""GPU parity tests: the CUDA search through the C ABI against the CPU oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2109_14814_gb300 as tms
import synth
from tests import meshcases
from tests.parity import check_sorted_unique, compare, gpu_records

pytestmark = pytest.mark.gpu

_cache = {}


def cached(name, fn):
    if name not in _cache:
        _cache[name] = fn()
    return _cache[name]


def oracle_hits(name, pair):
    def run():
        OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
        return OA, OB, oracle.search(OA, OB)
    return cached("oracle:" + name, run)


def gpu_search(pair, **kw):
    A = tms.Mesh.from_grid(pair.A)
    B = tms.Mesh.from_grid(pair.B)
    h = tms.search(A, B, **kw)
    torch.cuda.synchronize()
    return gpu_records(h)


# ---------------------------------------------------------------------------
# hand-solved meshes: exact results
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(meshcases.ALL_CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_hand_solved_cases_exact(name, precision):
    A, B, exp, _ = meshcases.ALL_CASES[name]()
    g = gpu_search(synth.MeshPair(A, B, None), precision=precision)
    assert len(g["triA"]) == len(exp)
    for h, e in enumerate(exp):
        assert (int(g["triA"][h]), int(g["triB"][h])) == (e["triA"], e["triB"])
        tol = 0.0 if name != "seam" else 1e-12
        assert np.abs(g["z"][h] - np.array(e["z"])).max() <= tol
        assert np.abs(g["P"][h] - np.array(e["P"])).max() <= (0.0 if name != "seam" else 1e-14)
        if "params" in e:
            assert np.allclose(g["params"][h], e["params"], rtol=0, atol=1e-15)
    if name in ("diagonal", "vertex"):
        assert int(g["flags"][0]) & 2


# ---------------------------------------------------------------------------
# synthetic configurations against the oracle
# ---------------------------------------------------------------------------

def test_config1_parity_and_planted():
    p = cached("c1", synth.config1)
    OA, OB, ref = oracle_hits("c1", p)
    g = gpu_search(p)
    check_sorted_unique(g)
    s = compare(OA, OB, g, ref)
    assert s["common"] >= 5
    keys = set(zip(g["triA"].tolist(), g["triB"].tolist()))
    for a, b in zip(p.planted.triA.tolist(), p.planted.triB.tolist()):
        assert (a, b) in keys


@pytest.mark.parametrize("patch", [0, 1])
def test_config1_independent_surface_parity(patch):
    """B an independent seeded surface (not A reparameterised) bent through 5
    planted points of A: the GPU hits equal brute force, planted ones included."""
    p = cached("c1i", synth.config1_independent)
    OA, OB = oracle.OMesh.from_grid(p.A), oracle.OMesh.from_grid(p.B)
    ref = cached("oracle:c1i", lambda: oracle.search(OA, OB, method="brute"))
    g = gpu_search(p, patch=patch)
    check_sorted_unique(g)
    s = compare(OA, OB, g, ref)
    assert s["common"] >= 5
    keys = set(zip(g["triA"].tolist(), g["triB"].tolist()))
    for a, b in zip(p.planted.triA.tolist(), p.planted.triB.tolist()):
        assert (a, b) in keys


def test_config2_parity():
    p = cached("c2", synth.config2)
    OA, OB, ref = oracle_hits("c2", p)
    g = gpu_search(p)
    check_sorted_unique(g)
    s = compare(OA, OB, g, ref)
    assert s["common"] >= 64


def test_config5_parity():
    p = cached("c5", synth.config5)
    OA, OB, ref = oracle_hits("c5", p)
    g = gpu_search(p)
    s = compare(OA, OB, g, ref)
    assert s["common"] >= 512


VARIANTS = [
    dict(precision=0),
    dict(face_level=0),
    dict(precision=0, face_level=0),
    dict(moller=1),
    dict(moller=1, face_level=0),
    dict(cell_filter=0),
    dict(narrow_filter=0),
    dict(cell_mult=2.0),
    dict(cell_mult=5.0),
    dict(block_faces=64),
    dict(block_faces=256),
    dict(tile_rows=4),
    dict(use_graph=0),
    dict(patch=0),
    dict(patch=0, precision=0),
    dict(patch=0, moller=1),
    dict(patch=0, cell_filter=0),
    dict(patch=0, cell_mult=2.0),
    dict(block_faces=64, tile_rows=8),
    dict(block_faces=256, tile_rows=8, precision=0),
]


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: ",".join(f"{k}={x}" for k, x in v.items()))
def test_variants_same_hit_set(variant):
    """The hit set does not depend on precision mode, face level, broad-phase
    level (faces or patches in the grid), Moller test, occupancy filter, FP32
    pre-solve, cell size, tiling or graph use."""
    p = cached("c2", synth.config2)
    OA, OB, ref = oracle_hits("c2", p)
    base = gpu_search(p)
    g = gpu_search(p, **variant)
    assert list(zip(g["triA"], g["triB"])) == list(zip(base["triA"], base["triB"]))
    compare(OA, OB, g, ref)


def test_ragged_tiles_and_open_strip_against_bruteforce():
    """Sizes that leave ragged tiles in both directions, an open strip (no
    theta wrap), and a half-layer view of columns [k0, k1)."""
    p = synth.build_pair(91, 131, 27, 75, 19, stretch="exp", n_folds=2, sites=(4, 2), n_hits=6)
    OA, OB = oracle.OMesh.from_grid(p.A), oracle.OMesh.from_grid(p.B)
    ref = oracle.search(OA, OB, method="brute")
    g = gpu_search(p, block_faces=64, tile_rows=8)
    compare(OA, OB, g, ref)
    for kw in (dict(patch=0), dict(patch=1, tile_rows=4), dict(patch=1, precision=0)):
        compare(OA, OB, gpu_search(p, **kw), ref)
    # open strip version of A
    Ao = synth.MeshGrid(p.A.X, p.A.s, periodic=False)
    OAo = oracle.OMesh.from_grid(Ao)
    refo = oracle.search(OAo, OB, method="brute")
    go = gpu_search(synth.MeshPair(Ao, p.B, None))
    compare(OAo, OB, go, refo)
    # half-layer view: columns [5, 21) of A
    XA = p.A.X.cuda()
    A = tms.Mesh(XA, p.A.s, True, k0=5, k1=21)
    B = tms.Mesh.from_grid(p.B)
    h = gpu_records(tms.search(A, B))
    OAv = oracle.OMesh(p.A.X[:, 5:21].numpy(), p.A.s[5:21].numpy(), True)
    refv = oracle.search(OAv, OB, method="brute")
    compare(OAv, OB, h, refv)


def test_minimal_meshes():
    """N = 3 periodic, M = 2 (one quad row) against brute force."""
    g0 = torch.Generator().manual_seed(5)
    XA = torch.randn(4, 2, 3, generator=g0, dtype=torch.float64)
    XB = XA.mean(dim=(1, 2), keepdim=True) + 0.7 * torch.randn(4, 2, 3, generator=g0, dtype=torch.float64)
    for seed in range(20):
        g0.manual_seed(seed)
        XB = XA.mean(dim=(1, 2), keepdim=True) + 0.8 * torch.randn(4, 2, 3, generator=g0, dtype=torch.float64)
        A = synth.MeshGrid(XA, torch.tensor([0.0, 1.0], dtype=torch.float64))
        B = synth.MeshGrid(XB, torch.tensor([0.0, 1.0], dtype=torch.float64))
        OA, OB = oracle.OMesh.from_grid(A), oracle.OMesh.from_grid(B)
        ref = oracle.search(OA, OB, method="brute")
        for patch in (0, 1):
            g = gpu_search(synth.MeshPair(A, B, None), patch=patch)
            compare(OA, OB, g, ref)


@pytest.mark.parametrize("patch", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_dense_cells_every_overlap_emitted_once(precision, patch):
    """Both meshes inside one small ball: 89% of all quad pairs have overlapping
    boxes, the grid has 1 x 2 x 2 x 1 cells and every face lies in several of
    them, and one 32 x 32 tile keeps about 980 pairs (more than the emission's
    per-warp stage holds, so its dense-tile path writes them).  Every
    box-overlapping pair must be a candidate exactly once (the nearest
    non-overlapping pair is 1.6e-6 apart, far above FP32 rounding), and the hits
    must match brute force.  The same holds at the patch level: a quad pair
    lies in exactly one patch pair, which the patch-level grid finds once."""
    g0 = torch.Generator().manual_seed(11)
    XA = 0.01 * torch.randn(4, 13, 12, generator=g0, dtype=torch.float64)
    XB = 0.01 * torch.randn(4, 13, 12, generator=g0, dtype=torch.float64)
    s = torch.linspace(0.0, 1.0, 13, dtype=torch.float64)
    A, B = synth.MeshGrid(XA, s), synth.MeshGrid(XB, s)
    OA, OB = oracle.OMesh.from_grid(A), oracle.OMesh.from_grid(B)
    ref = oracle.search(OA, OB, method="brute")
    g = gpu_search(synth.MeshPair(A, B, None), precision=precision, patch=patch)
    compare(OA, OB, g, ref)

    def quad_boxes(X):
        X = X.numpy()
        Xn = np.roll(X, -1, axis=2)
        v = [X[:, :-1, :], Xn[:, :-1, :], X[:, 1:, :], Xn[:, 1:, :]]
        lo = np.minimum(np.minimum(v[0], v[1]), np.minimum(v[2], v[3])).reshape(4, -1).T
        hi = np.maximum(np.maximum(v[0], v[1]), np.maximum(v[2], v[3])).reshape(4, -1).T
        return lo, hi

    la, ha = quad_boxes(XA)
    lb, hb = quad_boxes(XB)
    overlapping = int(((la[:, None, :] <= hb[None, :, :]) & (lb[None, :, :] <= ha[:, None, :])).all(-1).sum())
    assert overlapping == 18556
    assert tms.last_stats()["candidates"] == overlapping


def test_disjoint_meshes_empty_world():
    p = cached("c1", synth.config1)
    XB = p.B.X + 1000.0
    g = gpu_search(synth.MeshPair(p.A, synth.MeshGrid(XB, p.B.s), None))
    assert len(g["triA"]) == 0
    assert tms.last_stats()["empty"] == 1


# ---------------------------------------------------------------------------
# errors and fault injection (host side; no GPU fault)
# ---------------------------------------------------------------------------

def test_nonfinite_vertex_rejected():
    p = cached("c1", synth.config1)
    X = p.A.X.clone()
    X[2, 5, 7] = float("nan")
    A = tms.Mesh(X.cuda(), p.A.s)
    B = tms.Mesh.from_grid(p.B)
    with pytest.raises(tms.TmsError) as e:
        tms.search(A, B)
    assert e.value.status == tms.TMS_ERR_ARG


def test_capacity_retry_and_injected_errors():
    p = cached("c2", synth.config2)
    base = gpu_search(p)
    A = tms.Mesh.from_grid(p.A)
    B = tms.Mesh.from_grid(p.B)
    # forced tiny entry capacity: the library grows its scratch and retries
    h = gpu_records(tms.search(A, B, inject=1))
    assert list(zip(h["triA"], h["triB"])) == list(zip(base["triA"], base["triB"]))
    assert tms.last_stats()["retries"] >= 1
    # a cell table started at 1024 slots: grown (x4 per retry) until under half full
    h = gpu_records(tms.search(A, B, inject=8))
    assert list(zip(h["triA"], h["triB"])) == list(zip(base["triA"], base["triB"]))
    assert np.array_equal(h["z"], base["z"])
    assert tms.last_stats()["retries"] >= 1
    # patch-pair, candidate, survivor and raw-hit buffers started at one record:
    # each overflows in turn and is grown; the final search matches bit for bit
    for kw in (dict(), dict(patch=0)):
        ref = gpu_records(tms.search(A, B, **kw))
        h = gpu_records(tms.search(A, B, inject=32, **kw))
        for k in ref:
            assert np.array_equal(h[k], ref[k], equal_nan=ref[k].dtype.kind == "f"), k
        assert tms.last_stats()["retries"] >= (4 if not kw else 3)
    # too-small output buffer: TMS_ERR_CAPACITY with the required count
    out = torch.empty((3, tms.HIT_BYTES), dtype=torch.uint8, device="cuda")
    with pytest.raises(tms.TmsError) as e:
        tms.search(A, B, out=out)
    assert e.value.status == tms.TMS_ERR_CAPACITY
    with pytest.raises(tms.TmsError) as e:
        tms.search(A, B, inject=2)
    assert e.value.status == tms.TMS_ERR_CAPACITY
    with pytest.raises(tms.TmsError) as e:
        tms.search(A, B, inject=4)
    assert e.value.status == tms.TMS_ERR_TIMEOUT
    # the context is still usable
    h = gpu_records(tms.search(A, B))
    assert len(h["triA"]) == len(base["triA"])


def test_device_wait_runs_out_then_exact():
    """The hit sort's look-back is the search's one device-side wait.  With
    inject bit 4 every earlier tile reads as unpublished, so each wait gives up
    after spin_limit polls: the kernel records the timeout, writes nothing out
    of bounds and returns (no fault), the merge keeps nothing, and the call
    reports TMS_ERR_TIMEOUT with the output buffer untouched.  The next call is
    exact.  2582 raw hits make two sort tiles, so a wait exists."""
    p = synth.build_pair(777, 384, 128, 384, 128, stretch="exp", n_folds=3, sites=(96, 24), n_hits=0)
    OA, OB = oracle.OMesh.from_grid(p.A), oracle.OMesh.from_grid(p.B)
    ref = oracle.search(OA, OB)
    A = tms.Mesh.from_grid(p.A)
    B = tms.Mesh.from_grid(p.B)
    base = gpu_records(tms.search(A, B))
    assert tms.last_stats()["raw_hits"] > 2048
    compare(OA, OB, base, ref)
    out = torch.full((4096, tms.HIT_BYTES), 0xA5, dtype=torch.uint8, device="cuda")
    for limit in (1, 16):
        with pytest.raises(tms.TmsError) as e:
            tms.search(A, B, out=out, inject=16, spin_limit=limit)
        assert e.value.status == tms.TMS_ERR_TIMEOUT
        assert "look-back" in str(e.value)
        torch.cuda.synchronize()
        assert bool((out == 0xA5).all()), "a timed-out search wrote hit records"
        again = gpu_records(tms.search(A, B, out=out))
        for k in base:
            assert np.array_equal(again[k], base[k]), k
        out.fill_(0xA5)
    # the same parameters without the switch: the bounded wait never runs out
    h = gpu_records(tms.search(A, B, spin_limit=1 << 20))
    assert list(zip(h["triA"], h["triB"])) == list(zip(base["triA"], base["triB"]))


def test_bad_arguments():
    p = cached("c1", synth.config1)
    X = p.A.X.cuda()
    with pytest.raises(tms.TmsError):
        tms.Mesh(X, p.A.s.flip(0))                 # s not increasing
    with pytest.raises(tms.TmsError):
        tms.Mesh(X, p.A.s, k0=3, k1=4)             # fewer than 2 columns
    with pytest.raises(KeyError):
        tms.params(no_such_field=1)
    A = tms.Mesh(X, p.A.s)
    with pytest.raises(tms.TmsError):
        tms.search(A, A, cell_mult=0.5)            # cells narrower than faces
    with pytest.raises(tms.TmsError):
        tms.search(A, A, spin_limit=-1)
    with pytest.raises(tms.TmsError):
        tms.search(A, A, patch=2)


def test_search_host_matches_device_search():
    """tms_search_host: host coordinates copied into the meshes' device arrays,
    the search, the hits copied back -- bit for bit the device search, for
    pinned and pageable host memory and for a half-layer view."""
    p = cached("c2", synth.config2)
    XA = torch.empty_like(p.A.X, device="cuda")
    XB = torch.empty_like(p.B.X, device="cuda")
    A = tms.Mesh(XA, p.A.s, True)
    B = tms.Mesh(XB, p.B.s, True)
    ref = gpu_search(p)
    for pin in (False, True):
        hA = p.A.X.contiguous().pin_memory() if pin else p.A.X.contiguous()
        hB = p.B.X.contiguous().pin_memory() if pin else p.B.X.contiguous()
        XA.zero_()
        XB.zero_()
        out = torch.empty((1 << 12, tms.HIT_BYTES), dtype=torch.uint8)
        h = tms.search_host(A, B, hA, hB, out=out.pin_memory() if pin else out)
        assert h.raw.device.type == "cpu"
        g = gpu_records(h)
        for k in ref:
            assert np.array_equal(g[k], ref[k], equal_nan=ref[k].dtype.kind == "f"), k
        assert torch.equal(XA.cpu(), p.A.X) and torch.equal(XB.cpu(), p.B.X)
    # a view: only its columns are copied
    XA.zero_()
    Av = tms.Mesh(XA, p.A.s, True, k0=40, k1=200)
    Bf = tms.Mesh.from_grid(p.B)
    hv = gpu_records(tms.search_host(Av, Bf, p.A.X.contiguous(), p.B.X.contiguous()))
    Xv = p.A.X.cuda()
    rv = gpu_records(tms.search(tms.Mesh(Xv, p.A.s, True, k0=40, k1=200), Bf))
    assert list(zip(hv["triA"], hv["triB"])) == list(zip(rv["triA"], rv["triB"]))
    assert float(XA[:, :40].abs().sum()) == 0.0
    # a host output too small: TMS_ERR_CAPACITY (pageable and pinned)
    for pin in (False, True):
        out = torch.empty((3, tms.HIT_BYTES), dtype=torch.uint8)
        with pytest.raises(tms.TmsError) as e:
            tms.search_host(A, B, p.A.X.contiguous(), p.B.X.contiguous(), out=out.pin_memory() if pin else out)
        assert e.value.status == tms.TMS_ERR_CAPACITY


@pytest.mark.parametrize("seed", range(12))
def test_random_small_pairs_against_bruteforce(seed):
    """Seeded random small pairs -- sizes that leave ragged strips, patches and
    tiles, periodic or open A, a half-layer view -- in every precision mode and
    broad-phase level, each against the oracle's brute force."""
    rng = np.random.default_rng(1000 + seed)
    NA, MA = int(rng.integers(3, 70)), int(rng.integers(2, 30))
    NB, MB = int(rng.integers(3, 70)), int(rng.integers(2, 30))
    p = synth.build_pair(5000 + seed, NA, MA, NB, MB, stretch="exp", n_folds=int(rng.integers(0, 3)),
                         sites=(2 * int(rng.integers(1, 4)), int(rng.integers(1, 3))),
                         n_hits=int(rng.integers(0, 6)))
    A = p.A
    if seed % 3 == 1:
        A = synth.MeshGrid(p.A.X, p.A.s, periodic=False)
    OA, OB = oracle.OMesh.from_grid(A), oracle.OMesh.from_grid(p.B)
    ref = oracle.search(OA, OB, method="brute")
    for kw in (dict(), dict(patch=0), dict(precision=0), dict(face_level=0), dict(precision=0, patch=0)):
        g = gpu_search(synth.MeshPair(A, p.B, None), **kw)
        check_sorted_unique(g)
        compare(OA, OB, g, ref)
    if MA >= 6:
        k0, k1 = 1, MA - 2
        XA = A.X.cuda()
        h = gpu_records(tms.search(tms.Mesh(XA, A.s, A.periodic, k0=k0, k1=k1), tms.Mesh.from_grid(p.B)))
        OAv = oracle.OMesh(A.X[:, k0:k1].numpy(), A.s[k0:k1].numpy(), A.periodic)
        compare(OAv, OB, h, oracle.search(OAv, OB, method="brute"))


def test_patch_frames_cull_without_changing_hits():
    """The patch-frame test drops patch pairs (fewer listed than with the FP32
    filters off) and the hit set stays the same."""
    p = cached("c2", synth.config2)
    base = gpu_search(p)
    kept_on = tms.last_stats()["patch_kept"]
    off = gpu_search(p, narrow_filter=0)
    kept_off = tms.last_stats()["patch_kept"]
    assert kept_on < kept_off
    assert list(zip(base["triA"], base["triB"])) == list(zip(off["triA"], off["triB"]))


@pytest.mark.parametrize("delta", [1e-5, 1e-9, 0.0])
@pytest.mark.parametrize("tau", [1e-12, 1e-6, 0.05])
def test_patch_frames_near_contact(delta, tau):
    """B is A moved by delta along a fixed direction: every patch pair along
    the diagonal is a near miss (or, at delta = 0, coincident), the case where
    a frame test without its error terms would drop a pair with hits.  The
    hit set equals the one with the FP32 filters and frames off, and, for the
    small tolerances the hit test is meant for, the oracle's brute force.  A
    large tau (0.05) widens the hit test but not the broad phase (the boxes are
    the triangles' own), so there the oracle, which tries every pair, finds
    more; the filters must still drop no FP64 hit."""
    pr = synth.build_pair(77, 40, 14, 40, 14, stretch="exp", n_folds=1, sites=(2, 1), n_hits=3)
    v = torch.tensor([0.5, -0.5, 0.5, 0.5], dtype=torch.float64)
    XB = (pr.A.X + delta * v[:, None, None]).contiguous()
    B = synth.MeshGrid(XB, pr.A.s.clone(), True)
    pair = synth.MeshPair(pr.A, B, None)
    OA, OB = oracle.OMesh.from_grid(pr.A), oracle.OMesh.from_grid(B)
    ref = oracle.search(OA, OB, tau=tau, method="brute") if tau < 1e-3 else None
    base = gpu_search(pair, tau=tau, narrow_filter=0)
    keys = list(zip(base["triA"], base["triB"]))
    for kw in (dict(), dict(tile_rows=8), dict(block_faces=64)):
        g = gpu_search(pair, tau=tau, **kw)
        assert list(zip(g["triA"], g["triB"])) == keys
    if tau < 1e-3:
        compare(OA, OB, base, ref, tau=tau)


def _check_frames(F, grid):
    """Every FP64 vertex of every patch within the bounds of its frame (the
    record of tms_last_patch_frames), evaluated in FP64 with a margin far below
    the frame's own rounding terms; returns the share of patches with a frame."""
    X = grid.X.numpy()
    M, N = X.shape[1], X.shape[2]
    nqk, nqi = M - 1, (N if grid.periodic else N - 1)
    npk, npi = F.shape[0], F.shape[1]
    assert npk == (nqk + 3) // 4 and npi == (nqi + 7) // 8
    usable = 0
    for pk in range(npk):
        rows = np.arange(4 * pk, min(4 * pk + 4, nqk) + 1)
        for pi in range(npi):
            cols = np.arange(8 * pi, min(8 * pi + 8, nqi) + 1) % N
            V = X[:, rows][:, :, cols].reshape(4, -1).T
            f = F[pk, pi].astype(np.float64)
            c, E, h, rho, L, n2, n3 = f[0:4], f[4:20].reshape(4, 4), f[20:24], f[24], f[25], f[26], f[27]
            assert np.abs(V).max() <= L
            if not np.isfinite(h).all():
                continue
            usable += 1
            d = V - c
            a = d @ E.T
            tol = 1e-13 * max(1.0, np.abs(V).max())
            assert (np.abs(a).max(0) <= h + tol).all(), (pk, pi, np.abs(a).max(0), h)
            r = d - a @ E
            assert np.abs(r).max() <= rho + tol, (pk, pi, np.abs(r).max(), rho)
            assert n2 >= np.abs(E[2]).sum() and n3 >= np.abs(E[3]).sum()
    return usable / (npk * npi)


@pytest.mark.parametrize("case", ["config2", "ragged_open_tile8", "block64"])
def test_patch_frames_bound_every_vertex(case):
    """The frames the bounds pass writes hold every vertex of their patch, and
    nearly every patch gets one (with normal extents below its tangent ones)."""
    if case == "config2":
        p, kw = cached("c2", synth.config2), {}
    else:
        q = synth.build_pair(91, 131, 27, 75, 19, stretch="exp", n_folds=2, sites=(4, 2), n_hits=6)
        if case == "ragged_open_tile8":
            p = synth.MeshPair(synth.MeshGrid(q.A.X, q.A.s, periodic=False), q.B, None)
            kw = dict(tile_rows=8)
        else:
            p, kw = q, dict(block_faces=64)
    A, B = tms.Mesh.from_grid(p.A), tms.Mesh.from_grid(p.B)
    tms.search(A, B, **kw)
    torch.cuda.synchronize()
    for side, grid in ((0, p.A), (1, p.B)):
        F = tms.last_patch_frames(side)
        assert _check_frames(F, grid) >= 0.9
        h = F[..., 20:24].reshape(-1, 4)
        h = h[np.isfinite(h).all(1)]
        assert np.median(h[:, 2:].max(1)) < np.median(h[:, :2].max(1))
