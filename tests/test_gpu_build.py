"""GPU LEB build (Sec. 2) against the CPU oracle: bit-exact codes, vertices,
tags, neighbour links, orientation ids, plane offsets, statistics, stored
densities and majorants."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests import _checks as CK
from tests.conftest import scene_volume

pytestmark = pytest.mark.gpu

FIELDS = ("codes", "verts", "tag", "nbr", "nid", "plane", "density", "majorant", "count", "sum", "qmin", "qmax")


def gpu_arrays(grid):
    ex = grid.export()
    out = {k: v.cpu().numpy() for k, v in ex.items()}
    out["codes"] = out["codes"].view(np.uint64)
    out["sum"] = out["sum"].view(np.uint64)
    for k in ("count", "qmin", "qmax"):
        out[k] = out[k].view(np.uint32)
    return out


def assert_same_grid(gpu, ref):
    assert len(gpu["codes"]) == len(ref.codes), "tet counts differ: %d vs %d" % (len(gpu["codes"]), len(ref.codes))
    for k in FIELDS:
        g, r = gpu[k], getattr(ref, k)
        assert np.array_equal(g, r), "field %s differs at %d cells" % (k, int(np.sum(g != r)))


def build_both(s, vol):
    import paper_2506_11510_gb300 as tv
    grid = tv.build_scene_grid(s, torch.from_numpy(vol).cuda())
    ref = O.Grid.for_scene(s, vol).export()
    return grid, ref


@pytest.mark.parametrize("name", ["tiny", "adaptive_small", "production_small"])
def test_build_matches_oracle(name):
    s = W.scene(name)
    grid, ref = build_both(s, scene_volume(name))
    assert_same_grid(gpu_arrays(grid), ref)
    assert grid.info.K == ref.K and grid.info.max_depth == ref.max_depth and grid.info.rounds == ref.rounds


@pytest.mark.parametrize("fmt", [1, 2])
def test_build_density_formats(fmt):
    s = W.scene("adaptive_small", density_format=fmt)
    grid, ref = build_both(s, scene_volume("adaptive_small"))
    assert_same_grid(gpu_arrays(grid), ref)


@pytest.mark.parametrize("case", ["empty", "ragged_cubes", "uniform_d0", "uniform_d7", "no_camera", "camera_inside"])
def test_build_edge_cases(case):
    import paper_2506_11510_gb300 as tv
    base = W.scene("adaptive_small")
    rng = np.random.default_rng(5)
    if case == "empty":
        vol = np.zeros((16, 16, 16), np.float32)
        s = W.scene("adaptive_small", dims=(16, 16, 16), voxel_size=1 / 16, max_depth=12)
    elif case == "ragged_cubes":
        # 24 x 16 x 8 voxels: 3 x 2 x 1 cubes of 8^3, 36 roots
        vol = rng.uniform(0, 1, (8, 16, 24)).astype(np.float32)
        vol[vol < 0.4] = 0
        s = W.scene("adaptive_small", dims=(24, 16, 8), voxel_size=1 / 8, max_depth=12,
                    camera=W.Camera((1.5, 1.0, -2.5), (1.5, 1.0, 0.5), (0, 1, 0), 50.0, 40, 30))
    elif case == "uniform_d0":
        vol = scene_volume("tiny")
        s = W.scene("tiny", max_depth=0)
    elif case == "uniform_d7":
        vol = scene_volume("tiny")
        s = W.scene("tiny", max_depth=7)
    elif case == "no_camera":
        vol = scene_volume("adaptive_small")
        s = W.scene("adaptive_small", footprint_px=0.0, max_depth=12)
    else:
        vol = scene_volume("adaptive_small")
        s = W.with_camera(W.scene("adaptive_small", max_depth=15), pos=(0.4, 0.45, 0.5), target=(0.9, 0.5, 0.6))
    grid = tv.build_scene_grid(s, torch.from_numpy(np.ascontiguousarray(vol)).cuda())
    ref = O.Grid.for_scene(s, vol).export()
    assert_same_grid(gpu_arrays(grid), ref)
    CK.check_grid(ref)


@pytest.mark.parametrize("k", range(4))
def test_build_camera_criterion_random_views(k):
    """Criterion 2 alone (the density criterion off) for seeded random views -- eyes
    inside and outside the box, frustum edges and the near plane across it: the
    kernel's float decisions, and its fp64 evaluation where a comparison is too
    close to call in float, give the oracle's grid."""
    import paper_2506_11510_gb300 as tv
    rng = np.random.default_rng(300 + k)
    vol = scene_volume("adaptive_small")
    eye = tuple(float(v) for v in rng.uniform(-0.5, 1.5, 3))
    target = tuple(float(v) for v in rng.uniform(0.2, 0.8, 3))
    s = W.with_camera(W.scene("adaptive_small", variation_threshold=-1.0, footprint_px=float(rng.uniform(0.5, 3.0)),
                              max_depth=18),
                      pos=eye, target=target, fov_y_deg=float(rng.uniform(20.0, 80.0)))
    grid = tv.build_scene_grid(s, torch.from_numpy(vol).cuda())
    ref = O.Grid.for_scene(s, vol).export()
    assert len(ref.codes) > 24
    assert_same_grid(gpu_arrays(grid), ref)


def test_build_rejects_bad_arguments():
    import paper_2506_11510_gb300 as tv
    vol = torch.zeros((16, 16, 16), device="cuda")
    with pytest.raises(tv.TetvolError):
        tv.leb_build(vol, (0, 0, 0), 1 / 16, max_depth=51)
    with pytest.raises(tv.TetvolError):
        # 9 x 8 x 8 cubes of 2^3 voxels -> 3456 roots, more than the code's 8 root bits
        tv.leb_build(torch.zeros((16, 16, 18), device="cuda"), (0, 0, 0), 1 / 16, max_depth=3)


@pytest.mark.parametrize("name", ["adaptive_small", "production_small"])
def test_build_from_pinned_host_volume(name):
    """leb_build reads a pinned host volume in place (each value once, in the
    quantisation kernel): the grid equals the build from the same volume in
    device memory, bit for bit, and a rebuild from it equals one from device memory."""
    import paper_2506_11510_gb300 as tv
    s = W.scene(name)
    host = torch.from_numpy(scene_volume(name)).pin_memory()
    dev = host.cuda()
    a = gpu_arrays(tv.build_scene_grid(s, dev))
    g = tv.build_scene_grid(s, host)
    b = gpu_arrays(g)
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    s1 = W.with_camera(s, pos=(s.camera.pos[0] + 0.2, s.camera.pos[1], s.camera.pos[2]))
    r1 = gpu_arrays(tv.rebuild_scene_grid(g, s1, host))
    r2 = gpu_arrays(tv.build_scene_grid(s1, dev))
    for k in ("codes", "nbr", "density"):
        assert np.array_equal(r1[k], r2[k]), k


def test_build_refuses_pageable_host_memory():
    """A pageable host volume is refused before any kernel runs (the device could not read it)."""
    import ctypes as C
    from paper_2506_11510_gb300 import _native as N
    from paper_2506_11510_gb300 import api
    s = W.scene("tiny")
    vol = np.ascontiguousarray(scene_volume("tiny"))          # ordinary (pageable) host memory
    desc = api.volume_desc(torch.from_numpy(vol), s.box_min, s.voxel_size)
    out = C.c_void_p()
    st = N.lib().leb_build(C.c_void_p(vol.ctypes.data), C.byref(desc), None, 0.0, -1.0, 6, 0, None, C.byref(out))
    assert st == N.TG_EINVAL and not out.value
    with pytest.raises(TypeError):
        api.leb_build(torch.from_numpy(vol), s.box_min, s.voxel_size)


def test_builds_reuse_their_memory_and_release_it():
    """Builds take their buffers from the library's memory pool: a second build of
    the same scene equals the first and takes (almost) no new device memory -- the
    pool's memory is reused, not grown -- and tg_release_build_memory hands the
    unused part back to the driver."""
    import paper_2506_11510_gb300 as tv
    s = W.scene("production_small")
    vol = torch.from_numpy(scene_volume("production_small")).cuda()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    a = gpu_arrays(tv.build_scene_grid(s, vol))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    b = gpu_arrays(tv.build_scene_grid(s, vol))
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    assert free1 - free2 <= 0.1 * max(free0 - free1, 0) + (8 << 20)
    tv.release_build_memory()
    assert torch.cuda.mem_get_info()[0] >= free2
