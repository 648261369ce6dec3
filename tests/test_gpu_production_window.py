"""Parity on the benchmark's production volume (1024x1024x512 fBm x Worley
cloud, 20% occupancy) with the benchmark's medium (albedo 0.95, HG g 0.7, up to
128 bounces, sun and environment), through a window camera: the benchmark
camera with its field of view narrowed to the central 64x64 pixels of the
1024^2 frame.  Those pixels subtend the same angle as in the full frame, so the
camera criterion refines the window's sub-frustum to the same 1-pixel
footprint; outside it the grid stays coarse, which keeps the oracle's build and
walks within test time.

* the GPU LEB build of that grid is bit-exact with the oracle's (codes,
  vertices, links, orientation ids, planes, statistics, stored densities), for
  BF16 (the benchmark's storage), FP16 and FP32 densities;
* 4096 window paths (pixels and samples of the benchmark's 32 spp) traced by
  the GPU match the fp64 oracle per path (1e-4 relative for >= 99.9%, flags,
  collision counts, visited cells of non-degenerate paths, mean difference
  inside 3 sd / sqrt(n)), for each density format;
* the storage error of BF16 and FP16 densities against FP32 densities is
  measured on the oracle alone (fp64 arithmetic, the same paths): it is a
  property of the storage format, not of the GPU.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests.test_gpu_build import assert_same_grid, gpu_arrays
from tests.test_gpu_render import compare_paths

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 8
SIDE = 64


def window_scene(s, side=SIDE, density_format=None):
    """The scene with the camera narrowed to the central side x side pixels."""
    cam = s.camera
    frac = side / cam.height
    fov = 2 * math.degrees(math.atan(math.tan(math.radians(cam.fov_y_deg) / 2) * frac))
    w = W.with_camera(s, fov_y_deg=fov, width=side, height=side)
    if density_format is not None:
        w = W.scene(s.name, camera=w.camera, density_format=density_format)
    return w


@pytest.fixture(scope="module")
def production_window():
    s = W.scene("production")
    vol = W.make_volume(s, device="cuda")
    vnp = vol.cpu().numpy()
    return s, vol, vnp, {}


def grids(fx, fmt):
    """GPU and oracle grids of the window for one density format (cached per module)."""
    import paper_2506_11510_gb300 as tv
    s, vol, vnp, cache = fx
    if fmt not in cache:
        w = window_scene(s, density_format=fmt)
        cache[fmt] = (w, tv.build_scene_grid(w, vol), O.Grid.for_scene(w, vnp, nthreads=NTHREADS))
    return cache[fmt]


def window_paths(n, seed, spp=32):
    rng = np.random.default_rng(seed)
    px = rng.integers(0, SIDE, n).astype(np.int32)
    py = rng.integers(0, SIDE, n).astype(np.int32)
    sm = rng.integers(0, spp, n).astype(np.int32)
    return px, py, sm


@pytest.mark.parametrize("fmt", [1, 2, 0])
def test_window_grid_bit_exact(production_window, fmt):
    w, grid, ref = grids(production_window, fmt)
    a = ref.export()
    assert a.max_depth >= 20, "the window grid should reach the production depths (%d)" % a.max_depth
    assert grid.info.max_depth == a.max_depth and grid.info.rounds == a.rounds
    assert_same_grid(gpu_arrays(grid), a)


@pytest.mark.parametrize("fmt", [1, 2, 0])
def test_window_paths_match_oracle(production_window, fmt):
    import paper_2506_11510_gb300 as tv
    w, grid, ref = grids(production_window, fmt)
    px, py, sm = window_paths(4096, 77)
    got = tv.tet_trace_paths(grid, w.camera, w.medium, w.render_seed, px, py, sm, seq_cap=512)
    want = ref.render_paths(w.camera, w.medium, w.render_seed, px, py, sm, seq_cap=512, nthreads=NTHREADS)
    assert want["collisions"].mean() > 1.0                 # multiple scattering, not a transmittance test
    compare_paths(got, want)


def test_window_storage_error_against_fp32_density(production_window):
    """BF16 and FP16 density storage against FP32 storage, both rendered by the
    fp64 oracle on the same paths: the per-pixel means of the 64x64 window at
    32 spp differ by a small fraction of the image's RMS radiance, and the image
    means agree within the Monte Carlo error of the difference."""
    w32, _, r32 = grids(production_window, 0)
    py, px, sm = np.meshgrid(np.arange(SIDE), np.arange(SIDE), np.arange(32), indexing="ij")
    px, py, sm = px.ravel().astype(np.int32), py.ravel().astype(np.int32), sm.ravel().astype(np.int32)
    L32 = r32.render_paths(w32.camera, w32.medium, w32.render_seed, px, py, sm, nthreads=NTHREADS)["L"]
    img32 = L32.reshape(SIDE * SIDE, 32).mean(1)
    rms = float(np.sqrt(np.mean(img32 ** 2)))
    for fmt, bound in ((1, 0.02), (2, 0.01)):
        w, _, r = grids(production_window, fmt)
        L = r.render_paths(w.camera, w.medium, w.render_seed, px, py, sm, nthreads=NTHREADS)["L"]
        img = L.reshape(SIDE * SIDE, 32).mean(1)
        d = img - img32
        assert float(np.sqrt(np.mean(d ** 2))) <= bound * rms
        dp = L - L32
        assert abs(dp.mean()) <= 3 * dp.std() / math.sqrt(len(dp)) + 1e-9
