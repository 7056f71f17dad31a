"""GPU parity of tms_refine (Sec. 7, damped Newton on the true surfaces) against
oracle/refine.py.  Seeds never come from the CUDA path: they are the oracle
search's hit estimates, the generator's planted records, or points placed near
the sheets' constructed crossings."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2109_14814_gb300 as tms
import synth
from oracle import refine as R

pytestmark = pytest.mark.gpu

_cache = {}


def cached(name, fn):
    if name not in _cache:
        _cache[name] = fn()
    return _cache[name]


def _oracle_hits(name, pair):
    def run():
        OA, OB = oracle.OMesh.from_grid(pair.A), oracle.OMesh.from_grid(pair.B)
        return oracle.search(OA, OB)
    return cached("hits:" + name, run)


def _gpu_refine(surface, seeds_np, **kw):
    seeds = torch.as_tensor(np.ascontiguousarray(seeds_np), dtype=torch.float64, device="cuda")
    out = tms.refine(surface, seeds, **kw)
    torch.cuda.synchronize()
    return {k: getattr(out, k).cpu().numpy() for k in ("x", "fnorm", "rho", "iters", "status")}


def _xdiff(a, b):
    d = np.abs(a - b)
    d[:, [0, 2]] = np.minimum(d[:, [0, 2]], 2 * math.pi - d[:, [0, 2]])
    return d.max(axis=1)


def compare(g, o, tol):
    """Statuses equal; iteration counts equal except where the stop was within
    rounding of the tolerance (then off by one, both converged); iterates,
    residual norms and normalised determinants agree."""
    assert np.array_equal(g["status"], o["status"]), (g["status"], o["status"])
    di = g["iters"].astype(np.int64) - o["iters"]
    assert np.all(np.abs(di) <= 1)
    off = di != 0
    assert off.mean() <= 0.01
    assert np.all(o["status"][off] == R.CONVERGED)
    fin = np.isfinite(o["x"]).all(axis=1)
    same = fin & ~off
    dx = _xdiff(g["x"][same], o["x"][same])
    assert dx.max(initial=0.0) <= 1e-9, dx.max()
    if off.any():
        assert _xdiff(g["x"][off], o["x"][off]).max() <= 1e-6
    conv = o["status"] == R.CONVERGED
    assert np.all(g["fnorm"][conv] <= tol)
    ev = same & np.isfinite(o["fnorm"])
    assert np.allclose(g["fnorm"][ev], o["fnorm"][ev], rtol=1e-3, atol=1e-12)
    assert np.array_equal(np.isnan(g["fnorm"]), np.isnan(o["fnorm"]))
    assert np.allclose(g["rho"][ev], o["rho"][ev], rtol=1e-7, atol=1e-15)
    th = g["x"][fin][:, [0, 2]]
    assert np.all((th >= 0.0) & (th < 2 * math.pi))


def _on_sites(x, surface, tol=1e-8):
    roots = R.site_roots(surface)
    d = np.abs(x[:, None, :] - roots[None, :, :])
    d[..., [0, 2]] = np.minimum(d[..., [0, 2]], 2 * math.pi - d[..., [0, 2]])
    return d.max(axis=2).min(axis=1) < tol


@pytest.mark.parametrize("name,fn", [("c1", synth.config1), ("c2", synth.config2),
                                     ("c5", synth.config5)])
def test_oracle_search_hits_refine_alike(name, fn):
    pair = cached(name, fn)
    seeds = _oracle_hits(name, pair)["params"]
    g = _gpu_refine(pair.surface, seeds)
    o = R.damped_newton(pair.surface, seeds)
    compare(g, o, 1e-10)
    assert np.all(g["status"] == R.CONVERGED)
    # the planted hits sit at lattice sites: their refinements land on sites
    assert _on_sites(g["x"], pair.surface).sum() >= len(pair.planted) * 0.9


def test_hit_records_read_in_place():
    # seeds read straight from the tms_hit records of the CUDA search match the
    # oracle search's estimates, so the refinements agree pair by pair
    pair = cached("c2", synth.config2)
    ref = _oracle_hits("c2", pair)
    A, B = tms.Mesh.from_grid(pair.A), tms.Mesh.from_grid(pair.B)
    hits = tms.search(A, B)
    out = tms.refine(pair.surface, hits)
    torch.cuda.synchronize()
    keys = list(zip(hits.triA.cpu().tolist(), hits.triB.cpu().tolist()))
    okeys = {k: j for j, k in enumerate(zip(ref["triA"].tolist(), ref["triB"].tolist()))}
    idx = [okeys[k] for k in keys]
    o = R.damped_newton(pair.surface, ref["params"][idx])
    assert np.array_equal(out.status.cpu().numpy(), o["status"])
    assert _xdiff(out.x.cpu().numpy(), o["x"]).max() <= 1e-7


def _near_site_seeds(surface, n, scale, seed):
    roots = R.site_roots(surface)
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, len(roots), n)
    return roots[pick] + rng.normal(0.0, scale, (n, 4))


@pytest.mark.parametrize("kw", [dict(), dict(alpha0=1.0, alpha1=1.0),
                                dict(alpha0=0.5, alpha1=1.0, switch_below=1e-5),
                                dict(alpha0=0.05, alpha1=0.05, max_iter=40),
                                dict(tol=0.0, max_iter=12)])
def test_schedules_ragged_counts(kw):
    pair = cached("small", lambda: synth.build_pair(777, 48, 20, 40, 24, sites=(6, 2), n_hits=0,
                                                    alpha=0.3, with_dalpha=True))
    for n in (1, 7, 37, 300):
        seeds = _near_site_seeds(pair.surface, n, 2e-3, n)
        compare(_gpu_refine(pair.surface, seeds, **kw), R.damped_newton(pair.surface, seeds, **kw),
                kw.get("tol", 1e-10))


def test_stop_statuses_and_edge_seeds():
    pair = cached("small", lambda: synth.build_pair(777, 48, 20, 40, 24, sites=(6, 2), n_hits=0,
                                                    alpha=0.3, with_dalpha=True))
    sp = pair.surface
    roots = R.site_roots(sp)
    x0 = np.repeat(roots[:1], 9, axis=0)
    x0[0, 1] = 2.0                  # escaped
    x0[1, 3] = -0.9                 # escaped
    x0[2, 0] = np.nan               # non-finite
    x0[3, 2] = np.inf               # non-finite
    x0[4] += 0.03                   # ordinary
    x0[5, 0] += 40 * math.pi        # unwrapped angle
    x0[6, 1] = 1.49                 # drifts out through the box
    x0[7] = roots[1] + 1e-14        # already converged
    x0[8, 2] -= 2 * math.pi
    for kw in (dict(), dict(max_iter=0), dict(rho_min=1.0 + 1e-9), dict(s_lo=0.0, s_hi=1.0)):
        g = _gpu_refine(sp, x0, **kw)
        o = R.damped_newton(sp, x0, **kw)
        compare(g, o, 1e-10)
    o = R.damped_newton(sp, x0, rho_min=1.0 + 1e-9)
    assert o["status"][4] == R.SINGULAR
    o = R.damped_newton(sp, x0)
    assert list(o["status"][:4]) == [R.ESCAPED, R.ESCAPED, R.NON_FINITE, R.NON_FINITE]


def test_strided_seeds_in_place_and_empty():
    pair = cached("small", lambda: synth.build_pair(777, 48, 20, 40, 24, sites=(6, 2), n_hits=0,
                                                    alpha=0.3, with_dalpha=True))
    sp = pair.surface
    seeds = _near_site_seeds(sp, 50, 1e-3, 5)
    o = R.damped_newton(sp, seeds)
    wide = torch.zeros((50, 7), dtype=torch.float64, device="cuda")
    wide[:, 2:6] = torch.as_tensor(seeds, device="cuda")
    out = tms.refine(sp, wide[:, 2:6])
    assert np.array_equal(out.status.cpu().numpy(), o["status"])
    assert _xdiff(out.x.cpu().numpy(), o["x"]).max() <= 1e-9
    assert float(wide[:, 0].abs().sum()) == 0.0 and float(wide[:, 6].abs().sum()) == 0.0
    buf = torch.as_tensor(seeds, device="cuda").contiguous()
    res = tms.Refined(buf, torch.empty(50, dtype=torch.float64, device="cuda"),
                      torch.empty(50, dtype=torch.float64, device="cuda"),
                      torch.empty(50, dtype=torch.int32, device="cuda"),
                      torch.empty(50, dtype=torch.int32, device="cuda"))
    tms.refine(sp, buf, out=res)
    assert _xdiff(buf.cpu().numpy(), o["x"]).max() <= 1e-9
    empty = tms.refine(sp, torch.empty((0, 4), dtype=torch.float64, device="cuda"))
    assert empty.x.shape == (0, 4) and empty.status.numel() == 0


def test_full_size_planted_seeds_and_search_hits():
    """4096 x 512 (the benchmark's meshes): every planted record's estimate as a
    seed, GPU against the oracle on all of them; then the CUDA search's own hits
    refined in place, each converged root confirmed by the oracle's f."""
    pair = cached("c3", synth.config3)
    sp = pair.surface
    seeds = pair.planted.params.numpy()
    g = _gpu_refine(sp, seeds)
    o = R.damped_newton(sp, seeds)
    compare(g, o, 1e-10)
    hits_kind = pair.planted.kind.numpy() == 0
    assert np.all(g["status"][hits_kind] == R.CONVERGED)
    assert _on_sites(g["x"][hits_kind], sp).all()
    A, B = tms.Mesh.from_grid(pair.A), tms.Mesh.from_grid(pair.B)
    hits = tms.search(A, B)
    out = tms.refine(sp, hits)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()
    assert (st == R.CONVERGED).mean() > 0.99
    x = out.x.cpu().numpy()[st == R.CONVERGED]
    rng = np.random.default_rng(3)
    pick = rng.choice(len(x), min(3000, len(x)), replace=False)
    f, _ = R.residual(sp, x[pick])
    assert np.sqrt((f * f).sum(axis=1)).max() <= 1.5e-10


# ---------------------------------------------------------------------------
# continuation (Sec. 8)
# ---------------------------------------------------------------------------

def _gpu_continue(surface, seeds_np, alphas, param="u", **kw):
    seeds = torch.as_tensor(np.ascontiguousarray(seeds_np), dtype=torch.float64, device="cuda")
    out = tms.continue_branches(surface, seeds, alphas, param=param, **kw)
    torch.cuda.synchronize()
    return {k: getattr(out, k).cpu().numpy() for k in ("x", "status", "iters", "rho", "fnorm")}


def compare_continuation(g, o, max_iter=200, rho_turn=1e-8):
    """Branch by branch: identical up to the first step where either side did not
    converge; there both sides stop, or the side that went on had wandered
    (a corrector of at least max_iter/2 updates) or sat on the turning threshold.
    At least 75% of the branches must agree at every step."""
    n, K1 = o["status"].shape
    identical = 0
    for b in range(n):
        gs, os_ = g["status"][b], o["status"][b]
        bad = np.nonzero((gs != R.CONVERGED) | (os_ != R.CONVERGED))[0]
        js = int(bad[0]) if bad.size else K1
        upto = slice(0, js + 1) if js < K1 and gs[js] == os_[js] == R.TURNING else slice(0, js)
        ok = np.isfinite(o["x"][b, upto]).all(axis=1)
        d = _xdiff(g["x"][b, upto][ok], o["x"][b, upto][ok])
        assert d.max(initial=0.0) <= 1e-8, (b, d.max())
        assert np.all(np.abs(g["iters"][b, :js].astype(np.int64) - o["iters"][b, :js]) <= 1)
        if js == K1 or (gs[js] == os_[js] and np.array_equal(gs, os_)):
            identical += 1
            continue
        if gs[js] != os_[js]:
            wandered = max(g["iters"][b, js], o["iters"][b, js]) >= max_iter // 2
            on_edge = abs(abs(o["rho"][b, js]) - rho_turn) <= 1e-6 * rho_turn
            both_fail = gs[js] not in (R.CONVERGED, R.TURNING) and os_[js] not in (R.CONVERGED, R.TURNING)
            assert wandered or on_edge or both_fail, (b, js, gs[js], os_[js])
    assert identical >= 0.75 * n, (identical, n)


@pytest.mark.parametrize("param,steps", [
    ("u", np.linspace(0.002, 0.2, 100)),
    ("s", np.linspace(0.002, 0.2, 100)),
    ("u", -0.1 * (np.geomspace(1e-3, 1.0, 40))),          # backwards, uneven steps
])
def test_continuation_parity(param, steps):
    pair = cached("c2", synth.config2)
    sp = pair.surface
    x0 = R.site_roots(sp)[:64]
    g = _gpu_continue(sp, x0, steps, param=param, max_jump=0.05)
    o = R.continuation(sp, x0, steps, param=param, max_jump=0.05)
    compare_continuation(g, o)
    assert (g["status"][:, -1] == R.CONVERGED).mean() >= 0.5


def test_continuation_edges():
    pair = cached("c2", synth.config2)
    sp = pair.surface
    x0 = R.site_roots(sp)[:7]
    steps = np.linspace(0.002, 0.01, 5)
    # no steps: exactly the refinement of the seeds
    g = _gpu_continue(sp, x0, [])
    r = _gpu_refine(sp, x0)
    assert g["x"].shape == (7, 1, 4)
    assert np.array_equal(g["x"][:, 0], r["x"]) and np.array_equal(g["status"][:, 0], r["status"])
    # turning at step 0 (rho_turn above the Hadamard bound), jumps at step 1
    for kw in (dict(rho_turn=1.0 + 1e-9), dict(max_jump=1e-12), dict(alpha0=1.0, alpha1=1.0)):
        g = _gpu_continue(sp, x0, steps, **kw)
        o = R.continuation(sp, x0, steps, **kw)
        compare_continuation(g, o)
        assert np.array_equal(g["status"], o["status"])
    empty = tms.continue_branches(sp, torch.empty((0, 4), dtype=torch.float64, device="cuda"), steps)
    assert empty.x.shape == (0, 6, 4)
