"""The GPU walk alone (Sec. 3): optical depth and visited cells along rays
against the oracle, Beer-Lambert in a homogeneous medium, axis-aligned and
lattice-line rays, grid import/export round trip, and the step limit on a
corrupted neighbour table (a bounded walk, never a hang)."""
import numpy as np
import pytest
import torch

import oracle as O
from tests import _checks as CK

pytestmark = pytest.mark.gpu


def random_grid(seed, n=16, theta=0.1, max_depth=11, value=None):
    rng = np.random.default_rng(seed)
    if value is None:
        vol = rng.uniform(0, 1, (n, n, n)).astype(np.float32)
        vol[rng.uniform(0, 1, vol.shape) < 0.3] = 0
    else:
        vol = np.full((n, n, n), value, np.float32)
    return vol, dict(box_min=(0, 0, 0), voxel_size=1.0 / n, theta=theta, max_depth=max_depth)


def gpu_grid(vol, kw):
    import paper_2506_11510_gb300 as tv
    return tv.leb_build(torch.from_numpy(vol).cuda(), kw["box_min"], kw["voxel_size"], None, 0.0, kw["theta"],
                        kw["max_depth"], 0)


def rays(rng, m):
    target = rng.uniform(0.02, 0.98, (m, 3))
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return target - 2.5 * d, d


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_optical_depth_and_sequences_match_oracle(seed):
    import paper_2506_11510_gb300 as tv
    vol, kw = random_grid(seed)
    g = gpu_grid(vol, kw)
    ref = O.Grid(vol, **kw)
    rng = np.random.default_rng(100 + seed)
    o, d = rays(rng, 4000)
    # fp32 rays on both sides
    o32, d32 = o.astype(np.float32), d.astype(np.float32)
    got = tv.tet_optical_depth(g, torch.from_numpy(o32).cuda(), torch.from_numpy(d32).cuda(), 2.0, seq_cap=2048)
    want = ref.optical_depth(o32.astype(np.float64), d32.astype(np.float64), 2.0, seq_cap=2048)
    tau = got["tau"].cpu().numpy().astype(np.float64)
    assert np.allclose(tau, want["tau"], rtol=2e-5, atol=1e-6)
    nondeg = (want["flags"] & 1) == 0
    gs, gl = got["seq"].cpu().numpy(), got["seq_len"].cpu().numpy()
    same = [np.array_equal(gs[i, :gl[i]], want["seq"][i, :want["seq_len"][i]]) for i in np.nonzero(nondeg)[0]]
    assert nondeg.mean() > 0.9 and np.mean(same) >= 0.999


def test_homogeneous_beer_lambert_axis_and_lattice_rays():
    import paper_2506_11510_gb300 as tv
    vol, kw = random_grid(3, value=0.5, theta=-1.0, max_depth=9)
    g = gpu_grid(vol, kw)
    rng = np.random.default_rng(4)
    o, d = rays(rng, 500)
    extra_o = np.array([[-1, 0.3, 0.7], [0.25, -1, 0.5], [0.5, 0.5, -2], [-1, -1, -1], [-1, 0.5, 0.5],
                        [0.125, 0.375, -1], [0.5, 2, 0.5], [2, 0.75, 0.25]])
    extra_d = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [1, 0, 0], [0, 0, 1], [0, -1, 0], [-1, 0, 0]],
                       np.float64)
    extra_d /= np.linalg.norm(extra_d, axis=1, keepdims=True)
    o = np.concatenate([o, extra_o]).astype(np.float32)
    d = np.concatenate([d, extra_d]).astype(np.float32)
    got = tv.tet_optical_depth(g, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), 2.0)
    tau = got["tau"].cpu().numpy()
    for r in range(len(o)):
        se = CK.slab(o[r].astype(np.float64), d[r].astype(np.float64) / np.linalg.norm(d[r]), (1, 1, 1))
        assert tau[r] == pytest.approx(2.0 * 0.5 * (se[1] - se[0]), rel=2e-5, abs=1e-6)


def test_import_export_round_trip_and_render_on_imported_grid():
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import workloads as W
    from tests.conftest import scene_volume
    s = W.scene("adaptive_small", density_format=1)
    vol = scene_volume("adaptive_small")
    ref = O.Grid.for_scene(s, vol)
    a = ref.export()
    dev = torch.device("cuda")
    g = tv.grid_import(s.box_min, s.voxel_size, s.dims, a.K, torch.from_numpy(a.codes.view(np.int64)).to(dev),
                       torch.from_numpy(a.nbr).to(dev), torch.from_numpy(a.nid).to(dev),
                       torch.from_numpy(a.plane).to(dev), torch.from_numpy(a.density).to(dev), density_format=1)
    ex = g.export(("codes", "nbr", "nid", "plane", "density"))
    assert np.array_equal(ex["codes"].cpu().numpy().view(np.uint64), a.codes)
    for k in ("nbr", "nid", "plane", "density"):
        assert np.array_equal(ex[k].cpu().numpy(), getattr(a, k)), k
    assert g.info.max_depth == a.max_depth
    built = tv.build_scene_grid(s, torch.from_numpy(vol).cuda())
    px, py, sm = W.random_path_ids(s, 2000, seed=9)
    x = tv.tet_trace_paths(g, s.camera, s.medium, 5, px, py, sm)["L"]
    y = tv.tet_trace_paths(built, s.camera, s.medium, 5, px, py, sm)["L"]
    assert torch.equal(x, y)


def test_corrupted_links_end_in_the_step_limit():
    """Every link of an imported grid points back to the cell itself: each walk
    is stopped by the per-segment step limit and reported, and the kernel returns."""
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import workloads as W
    vol, kw = random_grid(6, n=8, theta=-1.0, max_depth=3)
    a = O.Grid(vol, **kw).export()
    n = len(a.codes)
    self_links = np.repeat(np.arange(n, dtype=np.int32)[:, None], 4, axis=1)
    dev = torch.device("cuda")
    g = tv.grid_import((0, 0, 0), 1 / 8, (8, 8, 8), a.K, torch.from_numpy(a.codes.view(np.int64)).to(dev),
                       torch.from_numpy(self_links).to(dev), torch.from_numpy(a.nid).to(dev),
                       torch.from_numpy(a.plane).to(dev), torch.from_numpy(a.density).to(dev))
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 20.0, 4, 4)
    med = W.Medium(0.5, 0.0, 0.0, 4, (0, -1, 0), 0.0, 1.0)     # sigma 0: no collisions, walks to the limit
    out = tv.tet_trace_paths(g, cam, med, 1, [1, 2], [1, 2], [0, 0])
    torch.cuda.synchronize()
    assert bool(((out["flags"] & 8) != 0).all())
    stats = tv.new_stats()
    tv.tet_render(g, cam, med, 1, 1, stats=stats)
    assert tv.stats_dict(stats)["step_limit"] == 16
