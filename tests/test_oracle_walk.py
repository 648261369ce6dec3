"""Pins of the oracle's tet walk (Sec. 3, "Path Tracing within Tetrahedral Grids"):
optical depth against brute-force clipping of the ray with every cell, the
visited sequence, at most three faces tested per cell, and Beer-Lambert in a
homogeneous medium, including axis-aligned and lattice-line rays."""
import numpy as np
import pytest

import oracle as O
from tests import _checks as CK
from tests.conftest import paper_count


def random_grid(seed, n=8, theta=0.1, max_depth=9, value=None):
    rng = np.random.default_rng(seed)
    if value is None:
        vol = rng.uniform(0, 1, (n, n, n)).astype(np.float32)
        vol[rng.uniform(0, 1, vol.shape) < 0.3] = 0
    else:
        vol = np.full((n, n, n), value, np.float32)
    g = O.Grid(vol, (0, 0, 0), 1.0 / n, theta=theta, max_depth=max_depth)
    return g, vol


def random_rays(rng, m):
    target = rng.uniform(0.05, 0.95, (m, 3))
    dirs = rng.normal(size=(m, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    origins = target - 3.0 * dirs
    return origins, dirs


@pytest.mark.parametrize("seed", [0, 1])
def test_optical_depth_matches_brute_force_clipping(seed):
    g, _ = random_grid(seed)
    a = g.export()
    rng = np.random.default_rng(10 + seed)
    o, d = random_rays(rng, 200)
    sigma = 3.0
    res = g.optical_depth(o, d, sigma, seq_cap=4096)
    assert np.all(res["max_faces_tested"] <= paper_count("max_faces_tested"))   # Sec. 3
    nondeg = 0
    for r in range(len(o)):
        se = CK.slab(o[r], d[r], (1, 1, 1))
        t0, t1 = CK.clip_all_tets(a.verts, a.K, o[r], d[r])
        lo, hi = np.maximum(t0, se[0]), np.minimum(t1, se[1])
        chord = np.maximum(hi - lo, 0)
        tau = sigma * float(np.sum(a.density.astype(np.float64) * chord))
        assert res["tau"][r] == pytest.approx(tau, rel=1e-9, abs=1e-12)
        if res["flags"][r] & 1:
            continue
        nondeg += 1
        vis = np.nonzero(chord > 1e-9)[0]
        vis = vis[np.argsort(lo[vis])]
        got = res["seq"][r, :res["seq_len"][r]]
        assert list(got) == list(vis)
    assert nondeg > 150


def test_homogeneous_beer_lambert_and_degenerate_rays():
    g, _ = random_grid(3, value=0.5, theta=-1.0, max_depth=7)
    rng = np.random.default_rng(4)
    o, d = random_rays(rng, 100)
    # axis-aligned rays, and rays running along lattice lines and through vertices
    extra_o = np.array([[-1, 0.3, 0.7], [0.25, -1, 0.5], [0.5, 0.5, -2], [-1, -1, -1], [-1, 0.5, 0.5],
                        [0.125, 0.375, -1]])
    extra_d = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [1, 0, 0], [0, 0, 1]], np.float64)
    extra_d /= np.linalg.norm(extra_d, axis=1, keepdims=True)
    o = np.concatenate([o, extra_o]); d = np.concatenate([d, extra_d])
    res = g.optical_depth(o, d, 2.0)
    for r in range(len(o)):
        se = CK.slab(o[r], d[r], (1, 1, 1))
        L = se[1] - se[0]
        assert res["tau"][r] == pytest.approx(2.0 * 0.5 * L, rel=1e-12)
        assert res["flags"][r] & ~1 == 0


def test_rays_that_miss_have_zero_depth():
    g, _ = random_grid(5)
    o = np.array([[-1, 2, 0.5], [2, 2, 2], [0.5, 0.5, 3]], np.float64)
    d = np.array([[1, 0, 0], [1, 0, 0], [0, 0, 1]], np.float64)
    res = g.optical_depth(o, d, 1.0)
    assert np.all(res["tau"] == 0) and np.all(res["flags"] & 4)
