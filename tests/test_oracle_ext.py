"""Pins of the oracle's extra channels (Sec. 3: "extra channels for, e.g.,
temperature, albedo, phase function parameters") and of its voxel-medium mode
tracked against the tet majorants: channel means and majorants by brute force,
the emission-absorption closed form, reduction to the plain estimator when the
channels equal the medium's constants, the white furnace, and delta tracking
on the tet grid against the regular-grid comparator's estimate of the same
voxel medium."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests import _checks as CK
from tests.conftest import scene_volume
from tests.test_oracle_leb import _brute_stats
from tests.test_oracle_render import all_paths, camera_rays

EMISSION, ALBEDO, GCHAN, VOXEL = 1, 2, 4, 8


def _q(v):
    return np.clip(np.rint(v.astype(np.float64) * 2 ** 24), 0, 2 ** 24).astype(np.int64)


@pytest.fixture(scope="module")
def small():
    s = W.scene("adaptive_small")
    vol = scene_volume("adaptive_small")
    t, a, g = (c.numpy() for c in W.make_channels(s))
    G = O.Grid.for_scene(s, vol)
    G.channels(vol, t, a, g)
    return s, vol, (t, a, g), G


def test_channel_means_and_majorants_by_brute_force(small):
    s, vol, (t, a, g), G = small
    arr = G.export()
    chan, vmaj = G.export_channels()
    K, n = arr.K, arr.voxels_per_cube
    qt, qa, qg, qd = _q(t), _q(a), _q(g), _q(vol)
    nz, ny, nx = vol.shape
    w = 1 << (K - int(np.log2(n)))
    rng = np.random.default_rng(4)
    depth = O.code_depth(arr.codes)
    picks = list(rng.choice(len(arr.codes), 50, replace=False)) + list(np.nonzero(depth == depth.min())[0][:3])
    for i in picks:
        for c, q in enumerate((qt, qa, qg)):
            cnt, sm, _, _ = _brute_stats(q, arr.verts[i], K, n)
            m = np.float32(np.float64(sm) / (np.float64(cnt) * 2.0 ** 24))
            if c == 2:
                m = np.float32(min(0.99, max(-0.99, 2.0 * float(m) - 1.0)))
            assert chan[i, c] == m
        v = arr.verts[i].astype(np.int64)
        lo = np.maximum(v.min(0) // w, 0)
        hi = np.minimum(v.max(0) // w, [nx - 1, ny - 1, nz - 1])
        box = qd[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        assert vmaj[i] == np.float32((box.max() + 1) / 2.0 ** 24)


def test_majorant_bounds_the_voxel_density_inside_every_tet(small):
    s, vol, _, G = small
    arr = G.export()
    _, vmaj = G.export_channels()
    K, n = arr.K, arr.voxels_per_cube
    rng = np.random.default_rng(5)
    idx = rng.choice(len(arr.codes), 3000)
    bary = rng.dirichlet(np.ones(4), size=len(idx))
    # points in the closed tets, including vertices
    bary[:100] = np.eye(4)[rng.integers(0, 4, 100)]
    p = np.einsum("ij,ijk->ik", bary, arr.verts[idx].astype(np.float64)) / 2.0 ** K     # grid space
    vi = np.clip(np.floor(p * n).astype(np.int64), 0, np.array(vol.shape[::-1]) - 1)
    rho = vol[vi[:, 2], vi[:, 1], vi[:, 0]]
    assert np.all(rho <= vmaj[idx])


def _homog_grid(value, channels):
    vol = np.full((16, 16, 16), value, np.float32)
    G = O.Grid(vol, (0, 0, 0), 1 / 16, theta=-1, max_depth=6)
    G.channels(vol, *channels)
    return vol, G


def test_emission_absorption_closed_form():
    """Pure absorber (albedo channel 0) at uniform temperature T, no lights: the
    collision estimator of emission gives E[L | ray] = Le (1 - exp(-sigma rho chord)),
    Le = scale * T; with the voxel medium (delta tracking) too."""
    rho, sig, T, scale = 0.5, 3.0, 0.75, 2.0
    one = lambda v: np.full((16, 16, 16), v, np.float32)
    vol, G = _homog_grid(rho, (one(T), one(0.0), one(0.5)))
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 40, 32)
    med = W.Medium(0.9, 0.0, sig, 4, (0, -1, 0), 0.0, 0.0)
    px, py, sm = all_paths(cam, 16)
    o, D = camera_rays(cam, 7, px, py, sm)
    p = np.empty(len(px))
    for i in range(len(px)):
        se = CK.slab(o, D[i], (1, 1, 1))
        p[i] = 0.0 if se is None else 1 - math.exp(-sig * rho * (se[1] - se[0]))
    for flags in (EMISSION | ALBEDO, EMISSION | ALBEDO | VOXEL):
        r = G.render_ext_paths(cam, med, 7, px, py, sm, flags, emission_scale=scale, density=vol)
        L = r["L"]
        assert set(np.unique(L)) <= {0.0, scale * T}
        hits = L / (scale * T)
        sd = math.sqrt(np.sum(p * (1 - p)))
        assert abs(hits.sum() - p.sum()) < 4 * sd, flags


def test_constant_channels_reduce_to_the_plain_estimator(small):
    """Channels equal to the medium's albedo and g: the extended estimator (without
    the voxel medium) draws the same random numbers and gives the plain path."""
    s, vol, _, _ = small
    G = O.Grid.for_scene(s, vol)
    alb, g = 0.75, 0.5
    one = lambda v: np.full(vol.shape, v, np.float32)
    G.channels(vol, one(0.0), one(alb), one((1 + g) / 2))
    med = W.Medium(alb, g, s.medium.sigma_scale, s.medium.max_bounces, s.medium.sun_dir,
                   s.medium.sun_irradiance, s.medium.env_radiance)
    px, py, sm = all_paths(s.camera, 1)
    plain = G.render_paths(s.camera, med, 5, px, py, sm)
    ext = G.render_ext_paths(s.camera, med, 5, px, py, sm, ALBEDO | GCHAN | EMISSION, emission_scale=3.0)
    assert np.array_equal(ext["L"], plain["L"])
    assert np.array_equal(ext["collisions"], plain["collisions"])


def test_furnace_with_unit_albedo_channel_and_voxel_medium(small):
    s, vol, (t, _, g), _ = small
    G = O.Grid.for_scene(s, vol)
    G.channels(vol, t, np.ones_like(vol), g)
    med = W.Medium(0.3, 0.0, s.medium.sigma_scale, 100000, s.medium.sun_dir, 0.0, 1.0)
    px, py, sm = all_paths(s.camera, 1)
    for flags in (ALBEDO | GCHAN, ALBEDO | GCHAN | VOXEL):
        r = G.render_ext_paths(s.camera, med, 3, px, py, sm, flags, density=vol)
        ok = (r["flags"] & 2) == 0
        assert ok.mean() > 0.999 and np.all(r["L"][ok] == 1.0), flags
        assert r["collisions"].max() > 10


def test_delta_tracking_escape_probability():
    """Uniform voxel medium, one bounce, environment 1, no sun: the path escapes
    uncollided with probability exp(-sigma rho chord); the tet majorant is above
    rho, so null collisions occur and must not change it."""
    rho, sig = 0.5, 3.0
    vol, G = _homog_grid(rho, (None, None, None))
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 40, 32)
    med = W.Medium(0.7, 0.0, sig, 1, (0, -1, 0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 16)
    r = G.render_ext_paths(cam, med, 9, px, py, sm, VOXEL, density=vol)
    o, D = camera_rays(cam, 9, px, py, sm)
    p = np.empty(len(px))
    for i in range(len(px)):
        se = CK.slab(o, D[i], (1, 1, 1))
        p[i] = 1.0 if se is None else math.exp(-sig * rho * (se[1] - se[0]))
    L = r["L"]
    assert set(np.unique(L)) <= {0.0, 1.0}
    sd = math.sqrt(np.sum(p * (1 - p)))
    assert abs(L.sum() - p.sum()) < 4 * sd


def test_delta_tracking_on_tets_estimates_the_voxel_medium():
    """The voxel medium tracked against the tet majorants and the regular-grid
    comparator (DDA through the same voxels) estimate the same image: their
    per-pixel means agree within 4 sigma (two independent unbiased estimators)."""
    s = W.scene("adaptive_small")
    vol = scene_volume("adaptive_small")
    G = O.Grid.for_scene(s, vol)
    G.channels(vol)
    cam = W.with_camera(s, width=24, height=20).camera
    med = W.Medium(0.9, 0.5, 48.0, 16, s.medium.sun_dir, 2.0, 0.25)
    px, py, sm = all_paths(cam, 64)
    a = G.render_ext_paths(cam, med, 21, px, py, sm, VOXEL, density=vol)["L"]
    b = O.dda_render_paths(vol, s.box_min, s.voxel_size, cam, med, 22, px, py, sm)["L"]
    npx = cam.width * cam.height
    A, B = a.reshape(npx, 64), b.reshape(npx, 64)
    diff = A.mean(1) - B.mean(1)
    se = np.sqrt(A.var(1, ddof=1) / 64 + B.var(1, ddof=1) / 64)
    z = diff.sum() / math.sqrt((se ** 2).sum())
    assert abs(z) < 4, z
    assert np.mean(np.abs(diff) <= 4 * se + 1e-12) > 0.99
