"""Parity at the benchmark sizes, in the launch configuration bench.py times.

adaptive (256^3 cloud, 512^2 at 32 spp, ~4.2 M tets): the whole GPU grid is
compared bit for bit with the oracle's; a seeded subset of paths is compared
one by one; and the full-frame render's accumulations at sampled pixels are
compared with the oracle's sums over the same paths.

production (1024x1024x512 cloud, 1024^2 at 32 spp, ~50 M tets, BF16): the
oracle cannot build this grid in test time, so the GPU grid is checked by
properties that hold at any size (exact volumes tiling the domain, symmetric
links joining identical faces, orientation ids, planes, longest-edge
refinement), and at sampled points against the oracle's own descent of the
LEB hierarchy (the leaf holding a point is a node of the oracle's descent, the
criterion does not split it, and its statistics and stored density are the
oracle's).  The full-frame render is checked by its counters, the white
furnace on sampled paths, and Beer-Lambert optical depths along sampled rays
against brute-force clipping with every cell of the grid.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests import _checks_torch as CT
from tests.test_gpu_render import FRAC, REL, compare_paths

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def adaptive():
    import paper_2506_11510_gb300 as tv
    s = W.scene("adaptive")
    vol = W.make_volume(s, device="cuda")
    grid = tv.build_scene_grid(s, vol)
    vnp = vol.cpu().numpy()
    ref = O.Grid.for_scene(s, vnp, nthreads=NTHREADS)
    return s, vol, vnp, grid, ref


def test_adaptive_volume_generation_is_device_independent(adaptive):
    s, vol, vnp, _, _ = adaptive
    cpu = W.make_volume(s, z_range=(100, 104)).numpy()
    assert np.array_equal(cpu, vnp[100:104])


def test_adaptive_grid_bit_exact(adaptive):
    from tests.test_gpu_build import assert_same_grid, gpu_arrays
    s, _, _, grid, ref = adaptive
    a = ref.export()
    assert 2_000_000 <= len(a.codes) <= 5_000_000
    assert_same_grid(gpu_arrays(grid), a)


def test_adaptive_sampled_paths_match_oracle(adaptive):
    import paper_2506_11510_gb300 as tv
    s, _, _, grid, ref = adaptive
    px, py, sm = W.random_path_ids(s, 4096, seed=21)
    got = tv.tet_trace_paths(grid, s.camera, s.medium, s.render_seed, px, py, sm, seq_cap=512)
    want = ref.render_paths(s.camera, s.medium, s.render_seed, px.numpy(), py.numpy(), sm.numpy(), seq_cap=512,
                            nthreads=NTHREADS)
    compare_paths(got, want)


def test_adaptive_full_frame_sampled_pixels(adaptive):
    """The full 512^2 x 32 spp frame as bench.py renders it, at 256 random pixels
    (8192 paths):
    * each pixel's accumulated sum is the sum of its 32 paths traced one by one
      (tet_trace_paths), up to the float additions' rounding: 32 terms added in
      any order differ by at most 32 * 2^-24 of the sum of their magnitudes;
    * those paths match the fp64 oracle's (1e-4 relative for >= 99.9%, flags,
      collision counts, mean difference inside 3 sd / sqrt(n));
    * so the pixel sums match the oracle's to 1e-4 (floor 1e-6 spp) except where
      one of their paths is among the <= 0.1% outliers: at least
      1 - 32 * 0.001 of the pixels, and in practice all."""
    import paper_2506_11510_gb300 as tv
    s, _, _, grid, ref = adaptive
    stats = tv.new_stats()
    img, img2 = tv.tet_render(grid, s.camera, s.medium, s.spp, s.render_seed, stats=stats)
    st = tv.stats_dict(stats)
    assert st["paths"] == s.paths_per_frame and st["step_limit"] == 0
    rng = np.random.default_rng(8)
    pix = rng.choice(s.camera.width * s.camera.height, 256, replace=False)
    px = np.repeat(pix % s.camera.width, s.spp).astype(np.int32)
    py = np.repeat(pix // s.camera.width, s.spp).astype(np.int32)
    sm = np.tile(np.arange(s.spp), len(pix)).astype(np.int32)
    got = tv.tet_trace_paths(grid, s.camera, s.medium, s.render_seed, px, py, sm)
    want = ref.render_paths(s.camera, s.medium, s.render_seed, px, py, sm, nthreads=NTHREADS)
    compare_paths(got, want, seq=False)
    Lg = got["L"].cpu().numpy().astype(np.float64).reshape(len(pix), s.spp)
    g = img.cpu().numpy().reshape(-1)[pix].astype(np.float64)
    g2 = img2.cpu().numpy().reshape(-1)[pix].astype(np.float64)
    bound = s.spp * 2.0 ** -24
    assert np.all(np.abs(g - Lg.sum(1)) <= bound * np.abs(Lg).sum(1) + 1e-12)
    assert np.all(np.abs(g2 - (Lg ** 2).sum(1)) <= 2 * bound * (Lg ** 2).sum(1) + 1e-12)
    osum = want["L"].reshape(len(pix), s.spp).sum(1)
    close = np.abs(g - osum) <= REL * np.maximum(np.abs(osum), 1e-6 * s.spp)
    assert close.mean() >= 1 - s.spp * (1 - FRAC)


# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def production():
    import paper_2506_11510_gb300 as tv
    s = W.scene("production")
    vol = W.make_volume(s, device="cuda")
    grid = tv.build_scene_grid(s, vol)
    return s, vol, grid


def test_production_grid_properties(production):
    s, _, grid = production
    ex = grid.export(("codes", "verts", "tag", "nbr", "nid", "plane"))
    n = ex["codes"].shape[0]
    assert 20_000_000 <= n <= 80_000_000, n
    CT.check_grid_torch(ex, grid.info.K, (2, 2, 1))
    assert len(torch.unique(ex["nid"])) == 18


def test_production_sampled_leaves_follow_the_oracle(production):
    s, vol, grid = production
    vnp = vol.cpu().numpy()
    ex = grid.export(("codes", "density", "count", "sum", "qmin", "qmax"))
    codes = ex["codes"].cpu().numpy().view(np.uint64)
    rng = np.random.default_rng(31)
    pts = rng.uniform([0, 0, 0], [2, 2, 1], (24, 3))
    pr = O.path_profile(vnp, s.box_min, s.voxel_size, s.camera, s.footprint_px, s.variation_threshold, s.max_depth,
                        s.density_format, pts, nthreads=NTHREADS)
    pos = {int(c): i for i, c in enumerate(codes)}
    for p in range(len(pts)):
        hits = [d for d in range(s.max_depth + 1) if int(pr["codes"][p, d]) in pos]
        assert len(hits) == 1, "the point's leaf is not a node of the oracle's descent"
        d = hits[0]
        i = pos[int(pr["codes"][p, d])]
        assert pr["split"][p, d] == 0, "the criterion would split this leaf"
        assert int(ex["count"][i]) == int(pr["count"][p, d]) and int(ex["sum"][i]) == int(pr["sum"][p, d])
        assert int(ex["qmin"][i]) == int(pr["qmin"][p, d]) and int(ex["qmax"][i]) == int(pr["qmax"][p, d])
        assert float(ex["density"][i]) == float(pr["density"][p, d])


def test_production_full_frame_and_furnace(production):
    import paper_2506_11510_gb300 as tv
    s, _, grid = production
    stats = tv.new_stats()
    img, _ = tv.tet_render(grid, s.camera, s.medium, s.spp, s.render_seed, stats=stats)
    st = tv.stats_dict(stats)
    assert st["paths"] == s.paths_per_frame and st["step_limit"] == 0
    assert bool(torch.isfinite(img).all()) and float(img.min()) >= 0
    med = W.Medium(1.0, s.medium.g, s.medium.sigma_scale, 100000, s.medium.sun_dir, 0.0, 1.0)
    px, py, sm = W.random_path_ids(s, 20000, seed=4)
    out = tv.tet_trace_paths(grid, s.camera, med, 3, px, py, sm)
    ok = (out["flags"].cpu().numpy() & 2) == 0
    assert ok.mean() > 0.99 and np.all(out["L"].cpu().numpy()[ok] == 1.0)


def test_production_optical_depth_by_brute_force(production):
    import paper_2506_11510_gb300 as tv
    s, _, grid = production
    ex = grid.export(("verts", "density"))
    K = grid.info.K
    v = ex["verts"].to(torch.float64) * 2.0 ** (-K)
    rho = ex["density"].to(torch.float64)
    FACE = CT.FACE
    rng = np.random.default_rng(12)
    target = rng.uniform([0.1, 0.1, 0.1], [1.9, 1.9, 0.9], (16, 3))
    d = rng.normal(size=(16, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = target - 3.0 * d
    got = tv.tet_optical_depth(grid, torch.tensor(o, dtype=torch.float32, device="cuda"),
                               torch.tensor(d, dtype=torch.float32, device="cuda"), 1.0)["tau"].cpu().numpy()
    for r in range(len(o)):
        oo = torch.tensor(o[r].astype(np.float32).astype(np.float64), device="cuda")
        dd = torch.tensor(d[r].astype(np.float32).astype(np.float64), device="cuda")
        dd = dd / dd.norm()
        t0 = torch.full((v.shape[0],), -math.inf, dtype=torch.float64, device="cuda")
        t1 = torch.full_like(t0, math.inf)
        for f in range(4):
            fv = v[:, FACE[f], :]
            n = torch.cross(fv[:, 1] - fv[:, 0], fv[:, 2] - fv[:, 0], dim=1)
            out = (n * (v[:, f] - fv[:, 0])).sum(1) > 0
            n = torch.where(out[:, None], -n, n)
            c = (n * fv[:, 0]).sum(1)
            nd = n @ dd
            t = (c - n @ oo) / nd
            t1 = torch.where(nd > 0, torch.minimum(t1, t), t1)
            t0 = torch.where(nd < 0, torch.maximum(t0, t), t0)
        tau = float((rho * torch.clamp(t1 - t0, min=0)).sum())
        assert got[r] == pytest.approx(tau, rel=1e-4, abs=1e-5)


def test_production_cached_furnace_is_exact(production):
    """Radiance cache at full size: in the white furnace a cache returning 1 makes
    every path exactly 1, so every pixel of the cached frame sums to spp."""
    from oracle import mlp as M
    from paper_2506_11510_gb300 import cache as RC
    s, _, grid = production
    med = W.Medium(1.0, s.medium.g, s.medium.sigma_scale, 100000, s.medium.sun_dir, 0.0, 1.0)
    p = torch.zeros(M.NUM_PARAMS, dtype=torch.float32, device="cuda")
    p[M.O_B4] = 1.0
    for depth in (1, 2):
        img, _ = RC.render_cached(grid, s.camera, med, 2, 5, depth, p)
        assert torch.all(img == 2.0)
    assert RC.timeouts() == 0


def test_production_channels_majorants_and_voxel_medium(production):
    """Extra channels at full size: the voxel majorant bounds the voxel density at
    points inside sampled cells, channel means lie in their ranges, and the
    voxel-medium furnace (unit albedo channel) returns exactly 1 per path."""
    import paper_2506_11510_gb300 as tv
    s, vol, grid = production
    t, a, g = W.make_channels(s, device="cuda")
    grid.channels(vol, t, torch.ones_like(a), g)
    chan, vmaj = grid.export_channels()
    ex = grid.export(("verts",))
    K = grid.info.K
    n = s.dims[0] // 2                                    # voxels per cube edge (2 x 2 x 1 cubes)
    gen = torch.Generator(device="cuda").manual_seed(3)
    idx = torch.randint(0, vmaj.numel(), (200000,), device="cuda", generator=gen)
    w = torch.distributions.Dirichlet(torch.ones(4, device="cuda")).sample((idx.numel(),))
    w = 0.99 * w + 0.0025          # strictly inside: a point on a face may round to the far side of it
    pts = (w[:, :, None] * ex["verts"][idx].double()).sum(1) * 2.0 ** (-K)
    vi = torch.floor(pts * n).long()
    vi[:, 0].clamp_(0, s.dims[0] - 1); vi[:, 1].clamp_(0, s.dims[1] - 1); vi[:, 2].clamp_(0, s.dims[2] - 1)
    rho = vol[vi[:, 2], vi[:, 1], vi[:, 0]]
    assert bool((rho <= vmaj[idx]).all())
    assert float(chan[:, 0].min()) >= 0 and float(chan[:, 0].max()) <= 1
    assert bool((chan[:, 1] == 1.0).all())
    assert float(chan[:, 2].min()) >= -0.99 and float(chan[:, 2].max()) <= 0.99
    med = W.Medium(0.3, s.medium.g, s.medium.sigma_scale, 100000, s.medium.sun_dir, 0.0, 1.0)
    px, py, sm = W.random_path_ids(s, 20000, seed=6)
    out = tv.tet_trace_ext_paths(grid, s.camera, med, 8 | 2 | 4, 3, px, py, sm, density=vol)
    ok = (out["flags"].cpu().numpy() & 2) == 0
    assert ok.mean() > 0.99 and np.all(out["L"].cpu().numpy()[ok] == 1.0)


def test_production_rebuild_for_a_closer_camera(production):
    """A camera moved close enough to change the grid: the rebuild equals the fresh build."""
    import paper_2506_11510_gb300 as tv
    s, vol, grid = production
    s1 = W.with_camera(s, pos=(1.0, 1.0, -0.6))
    g1 = tv.rebuild_scene_grid(grid, s1, vol)
    g2 = tv.build_scene_grid(s1, vol)
    assert g1.info.num_tets == g2.info.num_tets
    e1, e2 = g1.export(("codes", "nbr", "density")), g2.export(("codes", "nbr", "density"))
    for k in e1:
        assert torch.equal(e1[k], e2[k]), k
