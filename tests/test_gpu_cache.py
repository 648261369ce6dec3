"""The learned radiance cache on the GPU against the oracle: the fused BF16
tensor-core MLP (inference and training gradients) against the oracle network
evaluated with the same operand rounding, Adam, the tracer's cache queries and
vertex training samples against the oracle tracer, the cached frame against
its own per-path composition, and the white furnace with a constant cache."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as M
from paper_2506_11510_gb300 import workloads as W
from tests.conftest import scene_volume
from tests.test_gpu_render import all_paths

pytestmark = pytest.mark.gpu


def _net(seed):
    p = W.mlp_init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    p[M.O_B1:M.O_W2] = rng.normal(size=64) * 0.1
    p[M.O_B2:M.O_W3] = rng.normal(size=64) * 0.1
    p[M.O_B3:M.O_W4] = rng.normal(size=64) * 0.1
    p[M.O_W4:M.O_B4] *= 10
    p[M.O_B4] = 0.3
    return p.astype(np.float32)


def _scale(p, rec):
    """Per-row magnitude of the output's terms, sum |w4| |h3| + |b4| (oracle, fp64)."""
    _, c = M.forward(p.astype(np.float64), rec[:, 0:3], rec[:, 4:7], bf16_ops=True)
    P = M.unpack(p)
    return np.abs(c["h3"]) @ np.abs(P["w4"]) + abs(P["b4"])


@pytest.mark.parametrize("n", [1, 1000, 148 * 128 * 3 + 77])
def test_mlp_inference_matches_oracle(n):
    from paper_2506_11510_gb300 import cache as RC
    p = _net(21)
    rec = W.mlp_random_records(n, 22)
    y = RC.mlp_infer(torch.from_numpy(p).cuda(), torch.from_numpy(rec).cuda()).cpu().numpy().astype(np.float64)
    want, _ = M.forward(p.astype(np.float64), rec[:, 0:3].astype(np.float64), rec[:, 4:7].astype(np.float64),
                        bf16_ops=True)
    S = _scale(p, rec)
    err = np.abs(y - want) / S
    # fp32 accumulation against exact sums: an activation may round to the other bf16 neighbour
    assert np.all(np.isfinite(y))
    assert err.max() <= 2.0 ** -8, err.max()
    assert np.quantile(err, 0.99) <= 1e-4
    assert RC.timeouts() == 0


def test_mlp_inference_is_exact_for_a_constant_network():
    from paper_2506_11510_gb300 import cache as RC
    p = np.zeros(M.NUM_PARAMS, np.float32)
    p[M.O_B4] = 1.25
    rec = W.mlp_random_records(777, 3)
    y = RC.mlp_infer(torch.from_numpy(p).cuda(), torch.from_numpy(rec).cuda()).cpu().numpy()
    assert np.all(y == 1.25)


@pytest.mark.parametrize("n", [1000, 148 * 128 * 2 + 77])
def test_mlp_gradient_matches_oracle(n):
    """rc_mlp_grad (forward + backward, weight gradients accumulated in TMEM over
    a block's tiles) against the oracle's gradient with the same bf16 operands."""
    from paper_2506_11510_gb300 import cache as RC
    p = _net(31)
    rec = W.mlp_random_records(n, 32)
    grad = torch.zeros(M.NUM_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(3, dtype=torch.float32, device="cuda")
    RC.mlp_grad(torch.from_numpy(p).cuda(), torch.from_numpy(rec).cuda(), grad, loss)
    g = grad.cpu().numpy().astype(np.float64)
    lo = loss.cpu().numpy().astype(np.float64)
    r = rec.astype(np.float64)
    wl, wc, wg = M.loss_grad(p.astype(np.float64), r[:, 0:3], r[:, 4:7], r[:, 3], r[:, 7], bf16_ops=True)
    assert lo[1] == wc
    assert abs(lo[0] - wl) <= 1e-4 * wl
    for a, b in ((M.O_W1, M.O_B1), (M.O_B1, M.O_W2), (M.O_W2, M.O_B2), (M.O_B2, M.O_W3), (M.O_W3, M.O_B3),
                 (M.O_B3, M.O_W4), (M.O_W4, M.O_B4), (M.O_B4, M.NUM_PARAMS)):
        ref = wg[a:b]
        got = g[a:b]
        sc = np.abs(ref).max()
        assert sc > 0
        assert np.abs(got - ref).max() <= 2e-3 * sc, (a, np.abs(got - ref).max() / sc)
        assert np.linalg.norm(got - ref) <= 1e-3 * np.linalg.norm(ref), (a, np.linalg.norm(got - ref) /
                                                                         np.linalg.norm(ref))
    assert RC.timeouts() == 0


def test_adam_matches_oracle():
    from paper_2506_11510_gb300 import cache as RC
    rng = np.random.default_rng(7)
    P = M.NUM_PARAMS
    p, m, v = rng.normal(size=P), rng.normal(size=P) * 0.01, rng.uniform(0, 1e-3, P)
    g = rng.normal(size=P) * 3
    cnt, step, lr = 37.0, 3, 5e-3
    t = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    tp, tm, tv_, tg = t(p), t(m), t(v), t(g)
    loss = t([11.0, cnt, 0.0])
    RC.adam(tp, tm, tv_, tg, loss, step, lr)
    want_p, want_m, want_v = M.adam(p.astype(np.float32).astype(np.float64), m.astype(np.float32),
                                    v.astype(np.float32), g.astype(np.float32), cnt, step, lr)
    assert np.allclose(tp.cpu().numpy(), want_p, rtol=1e-6, atol=1e-6)
    # fp32 moments: rounding errors relative to the terms combined, not to the (possibly cancelling) result
    assert np.allclose(tm.cpu().numpy(), want_m, rtol=1e-6, atol=1e-7)
    assert np.allclose(tv_.cpu().numpy(), want_v, rtol=1e-6, atol=1e-8)
    assert np.all(tg.cpu().numpy() == 0)
    lo = loss.cpu().numpy()
    assert lo[0] == 0 and lo[1] == 0 and np.isclose(lo[2], 11.0 / cnt)


def test_random_training_paths():
    from paper_2506_11510_gb300 import cache as RC
    px, py, sm = RC.random_paths(5, 200000, 96, 80, 1000)
    px, py, sm = px.cpu().numpy(), py.cpu().numpy(), sm.cpu().numpy()
    assert px.min() >= 0 and px.max() < 96 and py.min() >= 0 and py.max() < 80
    assert np.array_equal(sm, 1000 + np.arange(200000))
    # uniform over the pixels: chi-square of the pixel counts
    counts = np.bincount(py * 96 + px, minlength=96 * 80)
    e = 200000 / (96 * 80)
    chi = ((counts - e) ** 2 / e).sum()
    dof = 96 * 80 - 1
    assert abs(chi - dof) < 5 * math.sqrt(2 * dof)
    # pixel i from Philox word 0 of counter (i, 0, 'RCAC', 0)
    for i in (0, 1, 12345):
        o = O.philox4x32_10((i, 0, 0x52434143, 0), (5, 0))
        pix = (o[0] * (96 * 80)) >> 32
        assert (px[i], py[i]) == (pix % 96, pix // 96)


@pytest.fixture(scope="module")
def scene_pair():
    import paper_2506_11510_gb300 as tv
    s = W.scene("adaptive_small")
    vol = scene_volume("adaptive_small")
    grid = tv.build_scene_grid(s, torch.from_numpy(vol).cuda())
    ref = O.Grid.for_scene(s, vol)
    return s, grid, ref


def _paths(s, n, seed):
    g = np.random.default_rng(seed)
    return (g.integers(0, s.camera.width, n).astype(np.int32), g.integers(0, s.camera.height, n).astype(np.int32),
            g.integers(0, 64, n).astype(np.int32))


@pytest.mark.parametrize("survive,start", [(0.0, 0), (0.5, 0), (0.5, 4)])
def test_cache_samples_match_oracle(scene_pair, survive, start):
    """Vertex training samples: positions, arrival directions, targets (the rest
    of the path per unit throughput) and validity per path and vertex; with
    survive = 0.5 the training paths end by Russian roulette after their last
    training vertex (from collision `start` on), with the oracle's decisions."""
    from paper_2506_11510_gb300 import cache as RC
    s, grid, ref = scene_pair
    px, py, sm = _paths(s, 4000, 3)
    J = 4 if survive == 0 else 2
    got, L = RC.cache_samples(grid, s.camera, s.medium, s.render_seed, px, py, sm, J, want_L=True, survive=survive,
                              roulette_from=start)
    got = got.cpu().numpy().astype(np.float64).reshape(-1, J, 8)
    want = ref.cache_paths(s.camera, s.medium, s.render_seed, px, py, sm, max_vertices=J, survive=survive,
                           roulette_from=start)
    wv = want["vertices"]
    same_valid = np.all(got[..., 7] == wv[..., 7], axis=1)
    pos = np.all(np.abs(got[..., 0:3] - wv[..., 0:3]) <= 1e-4, axis=(1, 2))
    drc = np.all(np.abs(got[..., 4:7] - wv[..., 4:7]) <= 1e-4, axis=(1, 2))
    tg = np.all(np.abs(got[..., 3] - wv[..., 3]) <= 1e-4 * np.maximum(np.abs(wv[..., 3]), 1e-3), axis=1)
    ok = same_valid & pos & drc & tg
    assert ok.mean() >= 0.999, (same_valid.mean(), pos.mean(), drc.mean(), tg.mean())
    assert wv[..., 7].sum() > (2000 if survive == 0 else 1000)
    if survive > 0:
        assert ((want["flags"] & 32) != 0).mean() > (0.05 if start == 0 else 0.005)   # the roulette ends paths
    Lo = want["L"]
    assert np.mean(np.abs(L.cpu().numpy() - Lo) <= 1e-4 * np.maximum(np.abs(Lo), 1e-6)) >= 0.999


@pytest.mark.parametrize("depth", [1, 2])
def test_cache_queries_match_oracle(scene_pair, depth):
    from paper_2506_11510_gb300 import cache as RC
    s, grid, ref = scene_pair
    px, py, sm = _paths(s, 4000, 4 + depth)
    got = RC.cache_queries(grid, s.camera, s.medium, s.render_seed, px, py, sm, depth).cpu().numpy()
    want = ref.cache_paths(s.camera, s.medium, s.render_seed, px, py, sm, cache_depth=depth)["query"]
    got = got.astype(np.float64)
    hit_same = (got[:, 3] > 0) == (want[:, 3] > 0)
    close = np.all(np.abs(got[:, [0, 1, 2, 4, 5, 6]] - want[:, [0, 1, 2, 4, 5, 6]]) <= 1e-4, axis=1)
    beta = np.abs(got[:, 3] - want[:, 3]) <= 1e-6
    Lc = np.abs(got[:, 7] - want[:, 7]) <= 1e-4 * np.maximum(np.abs(want[:, 7]), 1e-6)
    ok = hit_same & close & beta & Lc
    assert ok.mean() >= 0.999, (hit_same.mean(), close.mean(), beta.mean(), Lc.mean())
    assert (want[:, 3] > 0).mean() > 0.2


def test_cached_estimate_matches_oracle(scene_pair):
    """Per-path cached estimate L + beta max(R, 0): GPU queries and MLP against the
    oracle tracer and the oracle network with bf16 operands."""
    from paper_2506_11510_gb300 import cache as RC
    s, grid, ref = scene_pair
    p = _net(41)
    px, py, sm = _paths(s, 3000, 9)
    rec = RC.cache_queries(grid, s.camera, s.medium, s.render_seed, px, py, sm, 1)
    y = RC.mlp_infer(torch.from_numpy(p).cuda(), rec).cpu().numpy().astype(np.float64)
    rec = rec.cpu().numpy().astype(np.float64)
    got = rec[:, 7] + rec[:, 3] * np.maximum(y, 0)
    q = ref.cache_paths(s.camera, s.medium, s.render_seed, px, py, sm, cache_depth=1)["query"]
    yo, _ = M.forward(p.astype(np.float64), q[:, 0:3].astype(np.float32), q[:, 4:7].astype(np.float32),
                      bf16_ops=True)
    want = q[:, 7] + q[:, 3] * np.maximum(yo, 0)
    close = np.abs(got - want) <= 2e-3 * np.maximum(np.abs(want), 1e-3)
    assert close.mean() >= 0.999, close.mean()


def test_cached_frame_is_the_sum_of_its_paths(scene_pair):
    """tet_render_cached (tracer records, fused MLP completion, per-pixel sums)
    equals the per-path cached estimates of the same frame summed per pixel."""
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import cache as RC
    s, grid, ref = scene_pair
    p = torch.from_numpy(_net(43)).cuda()
    spp = 3
    stats = tv.new_stats()
    img, img2 = RC.render_cached(grid, s.camera, s.medium, spp, s.render_seed, 2, p, sample_offset=5, stats=stats)
    px, py, sm = all_paths(s.camera, spp)
    rec = RC.cache_queries(grid, s.camera, s.medium, s.render_seed, px, py, sm + 5, 2)
    y = RC.mlp_infer(p, rec)
    L = (rec[:, 7] + rec[:, 3] * torch.clamp(y, min=0)).double().cpu().numpy()
    pix = py.astype(np.int64) * s.camera.width + px
    want = np.bincount(pix, weights=L, minlength=s.camera.width * s.camera.height)
    want2 = np.bincount(pix, weights=L * L, minlength=s.camera.width * s.camera.height)
    g = img.cpu().numpy().ravel().astype(np.float64)
    g2 = img2.cpu().numpy().ravel().astype(np.float64)
    # the frame's shadow walks stop at optical depth 40 (trace mode walks to the boundary)
    close = np.abs(g - want) <= 1e-4 * np.maximum(np.abs(want), 1e-4)
    assert close.mean() >= 0.999, close.mean()
    assert np.mean(np.abs(g2 - want2) <= 1e-4 * np.maximum(np.abs(want2), 1e-4)) >= 0.999
    assert tv.stats_dict(stats)["paths"] == len(px)


def test_furnace_with_constant_cache_is_exact(scene_pair):
    """albedo 1, environment 1, no sun, cache R = 1: every path, cached or not, is
    worth exactly 1, so every pixel sums to spp exactly."""
    from paper_2506_11510_gb300 import cache as RC
    s, grid, _ = scene_pair
    med = W.Medium(1.0, 0.5, 64.0, 100000, s.medium.sun_dir, 0.0, 1.0)
    p = torch.zeros(M.NUM_PARAMS, dtype=torch.float32, device="cuda")
    p[M.O_B4] = 1.0
    for depth in (1, 2):
        img, _ = RC.render_cached(grid, s.camera, med, 4, 3, depth, p)
        assert torch.all(img == 4.0)


def test_training_lowers_the_loss(scene_pair):
    """Online training on the tracer's own vertices: the loss on held-out samples
    falls, and the cached frame's mean comes close to the plain frame's."""
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import cache as RC
    s, grid, _ = scene_pair
    rc = RC.RadianceCache(W.mlp_init_params(1, b4=0.1), lr=3e-3)
    # held-out samples
    hx, hy, hs = RC.random_paths(99, 4096, s.camera.width, s.camera.height, 1 << 28)
    held = RC.cache_samples(grid, s.camera, s.medium, s.render_seed, hx, hy, hs, 4)

    def held_loss():
        g = torch.zeros_like(rc.params)
        lo = torch.zeros(3, dtype=torch.float32, device="cuda")
        RC.mlp_grad(rc.params, held, g, lo)
        return float(lo[0] / lo[1])

    first = held_loss()
    for f in range(60):
        rc.train_frame(grid, s.camera, s.medium, s.render_seed, f, n_paths=1 << 12)
    last = held_loss()
    assert last < 0.7 * first, (first, last)
    plain, _ = tv.tet_render(grid, s.camera, s.medium, 64, s.render_seed)
    cached, _ = rc.render(grid, s.camera, s.medium, 64, s.render_seed, cache_depth=1)
    rel = abs(float(cached.mean()) - float(plain.mean())) / float(plain.mean())
    assert rel < 0.1, rel
    assert RC.timeouts() == 0
