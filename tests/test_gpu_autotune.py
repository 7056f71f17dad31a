"""tms_autotune: the chosen setting is one of the swept ones, finds the same hits
as the defaults, a second call is answered from the cache file, and a search
given the cache file (tms_params.autotune_cache) runs the tuned settings --
per size class cell multipliers included -- with identical results."""
import numpy as np
import pytest

import paper_2109_14814_gb300 as tms
import synth
from tests.parity import gpu_records

pytestmark = pytest.mark.gpu


def _same(a, b):
    ra, rb = gpu_records(a), gpu_records(b)
    assert list(zip(ra["triA"], ra["triB"])) == list(zip(rb["triA"], rb["triB"]))
    assert np.array_equal(ra["z"], rb["z"])


def test_autotune_single_pair_and_cache(tmp_path):
    pair = synth.config2()
    A, B = tms.Mesh.from_grid(pair.A), tms.Mesh.from_grid(pair.B)
    cache = str(tmp_path / "tune.txt")
    best, ms = tms.autotune([A], [B], cache_path=cache)
    assert best["face_level"] in (0, 1) and best["block_faces"] in (64, 128, 256)
    assert any(abs(best["cell_mult"] - m) < 1e-6 for m in (1.0625, 1.5, 2.5))
    assert best["precision"] == 1 and best["narrow_filter"] == 1 and ms > 0.0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    again, ms2 = tms.autotune([A], [B], cache_path=cache)
    assert again == best and abs(ms2 - ms) <= 1e-5 * ms
    assert len(open(cache).read().splitlines()) == 1
    tuned = {k: best[k] for k in ("face_level", "cell_mult", "block_faces", "tile_rows", "patch")}
    _same(tms.search(A, B, **tuned), tms.search(A, B))
    _same(tms.search(A, B, autotune_cache=cache), tms.search(A, B))


def test_autotune_batched_keeps_results():
    sizes = [(160, 40, 200, 48), (300, 64, 128, 32), (128, 32, 256, 80), (512, 96, 384, 64)]
    pairs = [synth.config4_pair(p, n_pairs=len(sizes), sizes=sizes) for p in range(len(sizes))]
    As = [tms.Mesh.from_grid(p.A) for p in pairs]
    Bs = [tms.Mesh.from_grid(p.B) for p in pairs]
    best, ms = tms.autotune(As, Bs, precision=0)
    assert best["precision"] == 0 and ms > 0.0
    tuned = {k: best[k] for k in ("face_level", "cell_mult", "block_faces", "tile_rows")}
    a = tms.search_batched(As, Bs, precision=0, **tuned)
    b = tms.search_batched(As, Bs, precision=0)
    _same(a, b)
    assert np.array_equal(a.offsets.cpu().numpy(), b.offsets.cpu().numpy())


def test_autotune_size_classes_through_the_cache(tmp_path):
    """A batch of uneven pairs: the cache gets the batch's line and one line per
    size class (a cell multiplier each); a batched search reading the cache
    finds exactly the default hits, pair by pair."""
    sizes = [(160, 40, 200, 48), (300, 64, 128, 32), (128, 32, 256, 80), (512, 96, 384, 64),
             (640, 128, 512, 160), (96, 24, 128, 16)]
    pairs = [synth.config4_pair(p, n_pairs=len(sizes), sizes=sizes) for p in range(len(sizes))]
    As = [tms.Mesh.from_grid(p.A) for p in pairs]
    Bs = [tms.Mesh.from_grid(p.B) for p in pairs]
    cache = str(tmp_path / "tune.txt")
    best, ms = tms.autotune(As, Bs, cache_path=cache)
    lines = open(cache).read().splitlines()
    assert sum(1 for l in lines if l.startswith("G|")) == 1
    classes = [l for l in lines if l.startswith("C|")]
    assert len(classes) >= 2
    for l in classes:
        assert float(l.split()[-1]) in (1.0625, 1.5, 2.5, 4.0)
    a = tms.search_batched(As, Bs, autotune_cache=cache)
    b = tms.search_batched(As, Bs)
    _same(a, b)
    assert np.array_equal(a.offsets.cpu().numpy(), b.offsets.cpu().numpy())
    again, ms2 = tms.autotune(As, Bs, cache_path=cache)
    assert again == best and len(open(cache).read().splitlines()) == len(lines)
