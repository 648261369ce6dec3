"""Pins of the oracle's learned radiance cache: the bf16 rounding, the frequency
encoding, backpropagation (against finite differences), Adam (closed forms),
and the tracer's two cache uses -- paths that end into the cache and training
samples from path vertices -- against the white furnace, an exact Bernoulli
case in a homogeneous medium, and the decomposition of the plain estimator."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as M
from paper_2506_11510_gb300 import workloads as W
from tests.test_oracle_render import all_paths, camera_rays
from tests import _checks as CK


# ---------------------------------------------------------------------------
# bf16 rounding
# ---------------------------------------------------------------------------
def test_bf16_rounding_ties_to_even():
    u = 2.0 ** -7                                  # bf16 spacing in [1, 2)
    assert M.bf16(1.0) == 1.0
    assert M.bf16(1 + u / 2) == 1.0                # tie, even mantissa below
    assert M.bf16(1 + 1.5 * u) == 1 + 2 * u        # tie, even mantissa above
    assert M.bf16(1 + u / 2 + 2.0 ** -20) == 1 + u
    assert M.bf16(-3.0) == -3.0
    assert M.bf16(0.0) == 0.0


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(3).normal(size=20000) * np.exp(np.random.default_rng(4).uniform(-20, 20, 20000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x.astype(np.float32)), ref)


# ---------------------------------------------------------------------------
# frequency encoding
# ---------------------------------------------------------------------------
def _blocks(e):
    """Positional sin/cos blocks (3, 12, 2) and directional (3, 4, 2) of an encoding row."""
    pos = e[6:6 + 72].reshape(3, 12, 2)
    dr = e[78:78 + 24].reshape(3, 4, 2)
    return pos, dr


def test_encoding_special_points():
    e = M.encode(np.zeros((1, 3)), np.zeros((1, 3)))[0]
    pos, dr = _blocks(e)
    assert np.all(e[:6] == 0) and np.all(e[102:] == 0)
    assert np.allclose(pos[..., 0], 0) and np.allclose(pos[..., 1], 1)
    assert np.allclose(dr[..., 0], 0) and np.allclose(dr[..., 1], 1)
    # x = (1/2, 0, 0): sin(pi/2) = 1, cos(pi/2) = 0, then sin(2^l pi / 2) = 0 and cos = -1, 1, 1, ...
    e = M.encode(np.array([[0.5, 0, 0]]), np.array([[0, 0, 1.0]]))[0]
    pos, dr = _blocks(e)
    assert np.allclose(pos[0, :, 0], [1] + [0] * 11, atol=1e-12)
    assert np.allclose(pos[0, :, 1], [0, -1] + [1] * 10, atol=1e-12)
    assert np.allclose(pos[1:, :, 0], 0) and np.allclose(pos[1:, :, 1], 1)
    # d = e_z: sin(2^l pi) = 0, cos(pi) = -1, then 1
    assert np.allclose(dr[2, :, 0], 0, atol=1e-12) and np.allclose(dr[2, :, 1], [-1, 1, 1, 1])
    assert np.array_equal(e[:6], [0.5, 0, 0, 0, 0, 1])


def test_encoding_frequencies_double():
    """sin(2a) = 2 sin a cos a and cos(2a) = cos^2 a - sin^2 a between successive
    frequencies, for every axis of both blocks."""
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (50, 3))
    d = rng.normal(size=(50, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    for e in M.encode(x, d):
        for blk in _blocks(e):
            s, c = blk[..., 0], blk[..., 1]
            assert np.allclose(s[:, 1:], 2 * s[:, :-1] * c[:, :-1], atol=1e-9)
            assert np.allclose(c[:, 1:], c[:, :-1] ** 2 - s[:, :-1] ** 2, atol=1e-9)
    # the lowest frequency is pi: sin(pi x) > 0 inside (0, 1)
    e = M.encode(x, d)
    assert np.all(e[:, 6:78].reshape(-1, 3, 12, 2)[:, :, 0, 0] > 0)


# ---------------------------------------------------------------------------
# network and training
# ---------------------------------------------------------------------------
def _net(seed=11, n=7):
    p = W.mlp_init_params(seed).astype(np.float64)
    p[M.O_B1:M.O_W2] = np.random.default_rng(seed).normal(size=64) * 0.1
    p[M.O_B2:M.O_W3] = np.random.default_rng(seed + 1).normal(size=64) * 0.1
    p[M.O_B3:M.O_W4] = np.random.default_rng(seed + 2).normal(size=64) * 0.1
    p[M.O_W4:M.O_B4] *= 10
    r = W.mlp_random_records(n, seed + 3).astype(np.float64)
    return p, r


def test_gradient_matches_finite_differences():
    p, r = _net()
    x, d, t, v = r[:, 0:3], r[:, 4:7], r[:, 3], r[:, 7]
    _, cnt, g = M.loss_grad(p, x, d, t, v)
    assert cnt == v.sum()
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(len(p)):
        pp = p.copy(); pp[i] += h
        lp = M.loss_grad(pp, x, d, t, v)[0]
        pp[i] -= 2 * h
        lm = M.loss_grad(pp, x, d, t, v)[0]
        fd[i] = (lp - lm) / (2 * h)
    err = np.abs(fd - g)
    scale = np.abs(g).max()
    assert scale > 0
    # every parameter group has a non-zero gradient and matches
    for a, b in ((M.O_W1, M.O_B1), (M.O_B1, M.O_W2), (M.O_W2, M.O_B2), (M.O_B2, M.O_W3), (M.O_W3, M.O_B3),
                 (M.O_B3, M.O_W4), (M.O_W4, M.O_B4), (M.O_B4, M.NUM_PARAMS)):
        assert np.abs(g[a:b]).max() > 0
    assert np.quantile(err / scale, 0.999) < 1e-6
    assert err.max() / scale < 1e-4          # a kink of a ReLU may fall inside +-h


def test_invalid_rows_do_not_contribute():
    p, r = _net(n=16)
    x, d, t, v = r[:, 0:3], r[:, 4:7], r[:, 3], r[:, 7]
    l1, c1, g1 = M.loss_grad(p, x, d, t, v)
    keep = v > 0
    l2, c2, g2 = M.loss_grad(p, x[keep], d[keep], t[keep], v[keep])
    assert c1 == c2 and np.isclose(l1, l2) and np.allclose(g1, g2, atol=1e-12)


def test_bf16_network_is_close_to_fp64():
    p, r = _net(n=200)
    y64, c = M.forward(p, r[:, 0:3], r[:, 4:7])
    y16, _ = M.forward(p, r[:, 0:3], r[:, 4:7], bf16_ops=True)
    # scale of the output's terms; bf16 keeps 8 significant bits through three products
    S = np.abs(c["h3"]) @ np.abs(M.unpack(p)["w4"]) + abs(M.unpack(p)["b4"])
    assert np.all(np.abs(y16 - y64) <= 2.0 ** -4 * S)
    assert not np.array_equal(y16, y64)


def test_adam_constant_gradient_moves_by_lr():
    """With a constant gradient the bias-corrected moments are exactly g and g^2,
    so every step moves each parameter by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=100); g = rng.normal(size=100) * 10.0 ** rng.uniform(-3, 3, 100)
    lr, eps = 1e-2, 1e-8
    p, m, v = p0.copy(), np.zeros(100), np.zeros(100)
    for step in range(1, 6):
        p, m, v = M.adam(p, m, v, g * 4, 4, step, lr, eps=eps)   # mean gradient = g
        assert np.allclose(p, p0 - step * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)


def test_adam_first_step_is_sign_step():
    g = np.array([3.0, -1e-3, 0.0, 1e4])
    p, m, v = M.adam(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 1, 0.5, eps=0.0 + 1e-30)
    assert np.allclose(p, [-0.5, 0.5, 0.0, -0.5])


def test_training_fits_a_smooth_function():
    """A property of the whole trainer: Adam on the L2 loss fits t = 1 + 0.5 sin(2 pi x0)."""
    rng = np.random.default_rng(9)
    p = W.mlp_init_params(3).astype(np.float64)
    m = np.zeros_like(p); v = np.zeros_like(p)
    x = rng.uniform(0, 1, (512, 3)); d = np.tile([0, 0, 1.0], (512, 1))
    t = 1 + 0.5 * np.sin(2 * np.pi * x[:, 0])
    first = None
    for step in range(1, 301):
        loss, cnt, g = M.loss_grad(p, x, d, t, np.ones(512))
        first = first or loss / cnt
        p, m, v = M.adam(p, m, v, g, cnt, step, 3e-3)
    loss = M.loss_grad(p, x, d, t, np.ones(512))[0] / 512
    assert loss < 0.01 * first and loss < 2e-3


# ---------------------------------------------------------------------------
# the tracer's cache uses
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny_grid(tiny_volume):
    return O.Grid.for_scene(W.scene("tiny"), tiny_volume)


def test_furnace_cache_targets_and_queries_are_one(tiny_grid):
    """albedo 1, environment 1, no sun: the rest of every path is worth exactly 1,
    so every training target is 1, every query has throughput 1 and nothing
    gathered before it, and a cache returning 1 makes every path exactly 1."""
    s = W.scene("tiny")
    med = W.Medium(1.0, 0.3, 30.0, 100000, s.medium.sun_dir, 0.0, 1.0)
    px, py, sm = all_paths(s.camera, 1)
    r = tiny_grid.cache_paths(s.camera, med, 11, px, py, sm, cache_depth=0, max_vertices=6)
    ok = (r["flags"] & 2) == 0
    v = r["vertices"][ok]
    valid = v[..., 7] == 1
    assert valid.sum() > 1000
    assert np.all(v[..., 3][valid] == 1.0)
    assert np.all(v[~valid] == 0)
    for k in (1, 2):
        q = tiny_grid.cache_paths(s.camera, med, 11, px, py, sm, cache_depth=k)["query"]
        hit = q[:, 3] > 0
        assert hit.mean() > 0.1
        assert np.all(q[hit, 3] == 1.0) and np.all(q[hit, 7] == 0.0)
        assert np.all(q[~hit, 7] == 1.0)                       # escaped before: environment
        est = q[:, 7] + q[:, 3] * 1.0
        assert np.all(est == 1.0)
        x = q[hit, 0:3]
        assert np.all((x >= 0) & (x <= 1))
        assert np.allclose(np.linalg.norm(q[hit, 4:7], axis=1), 1)


def test_cache_beyond_bounce_limit_is_the_plain_path(tiny_grid):
    s = W.scene("tiny")
    px, py, sm = all_paths(s.camera, 1)
    plain = tiny_grid.render_paths(s.camera, s.medium, 7, px, py, sm)
    q = tiny_grid.cache_paths(s.camera, s.medium, 7, px, py, sm, cache_depth=s.medium.max_bounces)
    assert np.all(q["query"][:, 3] == 0)
    assert np.array_equal(q["query"][:, 7], plain["L"])
    assert np.array_equal(q["L"], plain["L"])


def test_cached_path_plus_its_own_target_is_the_plain_path(tiny_grid):
    """For a path that reaches collision k, the cached record (L so far, beta, x, d)
    with the exact rest of the same path (the training target of its vertex k-1)
    gives back the plain estimate: L_plain = L_k + beta_k * target_{k-1}."""
    s = W.scene("tiny")
    px, py, sm = all_paths(s.camera, 2)
    plain = tiny_grid.render_paths(s.camera, s.medium, 7, px, py, sm)
    vt = tiny_grid.cache_paths(s.camera, s.medium, 7, px, py, sm, max_vertices=4)["vertices"]
    for k in (1, 2, 3):
        q = tiny_grid.cache_paths(s.camera, s.medium, 7, px, py, sm, cache_depth=k)["query"]
        hit = q[:, 3] > 0
        assert hit.sum() > 200
        v = vt[hit, k - 1]
        assert np.all(v[:, 7] == 1)
        assert np.array_equal(q[hit, 0:3], v[:, 0:3]) and np.array_equal(q[hit, 4:7], v[:, 4:7])
        rec = q[hit, 7] + q[hit, 3] * v[:, 3]
        assert np.allclose(rec, plain["L"][hit], rtol=1e-12, atol=1e-15)
        assert np.array_equal(q[~hit, 7], plain["L"][~hit])
        # the throughput at collision k is albedo^k
        assert np.allclose(q[hit, 3], float(np.float32(s.medium.albedo)) ** k, rtol=1e-12)


def test_cache_bernoulli_in_homogeneous_slab():
    """Homogeneous medium, no sun, environment 1, cache depth 1: a path either
    escapes uncollided (estimate 1) or ends into the cache at its first collision
    with throughput albedo and nothing gathered; the collision probability of a
    camera ray is 1 - exp(-sigma rho chord)."""
    rho, sig, alb = 0.5, 3.0, 0.6
    vol = np.full((16, 16, 16), rho, np.float32)
    g = O.Grid(vol, (0, 0, 0), 1 / 16, theta=-1, max_depth=6)
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 48, 40)
    med = W.Medium(alb, 0.2, sig, 16, (0, -1, 0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 8)
    q = g.cache_paths(cam, med, 5, px, py, sm, cache_depth=1)["query"]
    hit = q[:, 3] > 0
    assert np.all(q[hit, 3] == np.float32(alb)) and np.all(q[hit, 7] == 0)
    assert np.all(q[~hit, 7] == 1.0)
    o, D = camera_rays(cam, 5, px, py, sm)
    p = np.empty(len(px))
    for i in range(len(px)):
        se = CK.slab(o, D[i], (1, 1, 1))
        p[i] = 0.0 if se is None else 1 - math.exp(-sig * rho * (se[1] - se[0]))
    sd = math.sqrt(np.sum(p * (1 - p)))
    assert abs(hit.sum() - p.sum()) < 4 * sd
    # the query point lies on the camera ray, inside the box
    for i in np.nonzero(hit)[0][:200]:
        x = q[i, 0:3]
        w = x - o
        assert np.allclose(np.cross(w, D[i]), 0, atol=1e-9)
        assert np.allclose(q[i, 4:7], D[i], atol=1e-12)


# ---------------------------------------------------------------------------
# Russian roulette on training paths after their last training vertex
# ---------------------------------------------------------------------------
def test_roulette_off_is_the_plain_path(tiny_grid):
    """survive 0 or 1 switches the roulette off: the same vertices, targets and estimates."""
    s = W.scene("tiny")
    px, py, sm = all_paths(s.camera, 1)
    plain = tiny_grid.cache_paths(s.camera, s.medium, 7, px, py, sm, max_vertices=2)
    for q in (0.0, 1.0):
        r = tiny_grid.cache_paths(s.camera, s.medium, 7, px, py, sm, max_vertices=2, survive=q)
        assert np.array_equal(r["vertices"], plain["vertices"]) and np.array_equal(r["L"], plain["L"])
        assert np.array_equal(r["flags"], plain["flags"])


def test_roulette_decision_rate_and_weight():
    """One roulette per path (bounce limit = training vertices + 1) in a furnace
    (albedo 1, environment 1, no sun): a path that reaches its last training vertex
    is ended with probability 1 - q (binomial, 4 sd); a survivor carries throughput
    1 / q, so it returns exactly 1 / q when it escapes and 0 when the bounce limit
    truncates it; a path that escapes before the roulette returns exactly 1."""
    q, J = 0.375, 2
    vol = np.full((16, 16, 16), 0.5, np.float32)
    g = O.Grid(vol, (0, 0, 0), 1 / 16, theta=-1, max_depth=6)
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 64, 64)
    med = W.Medium(1.0, 0.3, 8.0, J + 1, (0, -1, 0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 16)
    r = g.cache_paths(cam, med, 9, px, py, sm, max_vertices=J, survive=q)
    played = r["vertices"][:, J - 1, 7] == 1
    killed = (r["flags"] & 32) != 0
    assert np.all(~killed[~played])
    n, k = int(played.sum()), int(killed.sum())
    assert n > 5000
    assert abs(k - n * (1 - q)) <= 4 * math.sqrt(n * q * (1 - q))
    alive = played & ~killed
    esc = alive & ((r["flags"] & 2) == 0)
    assert np.all(r["L"][esc] == 1.0 / q) and np.all(r["L"][alive & ~esc] == 0)
    assert np.all(r["L"][killed] == 0) and np.all(r["L"][~played & ((r["flags"] & 6) == 0)] == 1)


def test_roulette_keeps_the_targets_unbiased(tiny_grid):
    """The same paths with and without the roulette (q = 1/2 after 2 vertices) on
    the tiny scene with sun and environment: for every vertex the mean of the
    target difference is zero within 4 sd / sqrt(n), and the roulette paths are
    shorter."""
    s = W.scene("tiny")
    px, py, sm = all_paths(s.camera, 16)
    med = W.Medium(0.9, 0.3, 30.0, 64, s.medium.sun_dir, s.medium.sun_irradiance, 0.5)
    a = tiny_grid.cache_paths(s.camera, med, 13, px, py, sm, max_vertices=2)
    b = tiny_grid.cache_paths(s.camera, med, 13, px, py, sm, max_vertices=2, survive=0.5)
    assert np.array_equal(a["vertices"][..., 7], b["vertices"][..., 7])
    for j in range(2):
        v = a["vertices"][:, j, 7] == 1
        d = b["vertices"][v, j, 3] - a["vertices"][v, j, 3]
        assert v.sum() > 5000 and np.any(d != 0)
        assert abs(d.mean()) <= 4 * d.std() / math.sqrt(d.size)
    dL = b["L"] - a["L"]
    assert abs(dL.mean()) <= 4 * dL.std() / math.sqrt(dL.size)
    assert ((b["flags"] & 32) != 0).mean() > 0.05


def test_roulette_start_beyond_every_path_is_the_plain_path(tiny_grid):
    """A roulette that starts at the bounce limit never plays: the same vertices,
    targets, estimates and flags as without it."""
    s = W.scene("tiny")
    px, py, sm = all_paths(s.camera, 1)
    plain = tiny_grid.cache_paths(s.camera, s.medium, 7, px, py, sm, max_vertices=2)
    r = tiny_grid.cache_paths(s.camera, s.medium, 7, px, py, sm, max_vertices=2, survive=0.5,
                              roulette_from=s.medium.max_bounces)
    assert np.array_equal(r["vertices"], plain["vertices"]) and np.array_equal(r["L"], plain["L"])
    assert np.array_equal(r["flags"], plain["flags"])


def test_roulette_start_collision():
    """Furnace (albedo 1, environment 1, no sun), 2 training vertices, bounce limit 5,
    roulette from collision 3: it is played once, after collision 3 (index), by the
    paths that get that far, so an escaping path returns exactly 1 (escaped before)
    or 1 / q (survived it) -- never 1 / q^2, as it would with roulettes after
    collisions 1 and 2 -- a killed one 0; the kill rate is 1 - q (binomial, 4 sd)."""
    q = 0.375
    vol = np.full((16, 16, 16), 0.5, np.float32)
    g = O.Grid(vol, (0, 0, 0), 1 / 16, theta=-1, max_depth=6)
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 64, 64)
    med = W.Medium(1.0, 0.3, 8.0, 5, (0, -1, 0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 16)
    r = g.cache_paths(cam, med, 9, px, py, sm, max_vertices=2, survive=q, roulette_from=3)
    killed = (r["flags"] & 32) != 0
    trunc = (r["flags"] & 2) != 0
    early = ~killed & ~trunc & (r["L"] == 1.0)
    played = ~early & ((r["flags"] & 4) == 0)        # (flag 4: missed the box)
    assert np.all(r["L"][killed] == 0) and np.all(r["L"][trunc] == 0)
    assert np.all(np.isin(r["L"][played & ~killed & ~trunc], [1.0 / q]))
    n, k = int(played.sum()), int(killed.sum())
    assert n > 3000
    assert abs(k - n * (1 - q)) <= 4 * math.sqrt(n * q * (1 - q))


def test_roulette_from_a_later_collision_keeps_the_targets_unbiased(tiny_grid):
    """As the roulette after the last vertex, but played from collision 2 on (1
    training vertex): the mean target difference is zero within 4 sd / sqrt(n), and
    paths ending by the roulette never do so before collision 2."""
    s = W.scene("tiny")
    px, py, sm = all_paths(s.camera, 16)
    med = W.Medium(0.9, 0.3, 30.0, 64, s.medium.sun_dir, s.medium.sun_irradiance, 0.5)
    a = tiny_grid.cache_paths(s.camera, med, 13, px, py, sm, max_vertices=1)
    b = tiny_grid.cache_paths(s.camera, med, 13, px, py, sm, max_vertices=1, survive=0.5, roulette_from=2)
    c = tiny_grid.cache_paths(s.camera, med, 13, px, py, sm, max_vertices=1, survive=0.5)
    v = a["vertices"][:, 0, 7] == 1
    d = b["vertices"][v, 0, 3] - a["vertices"][v, 0, 3]
    assert v.sum() > 5000 and np.any(d != 0)
    assert abs(d.mean()) <= 4 * d.std() / math.sqrt(d.size)
    # fewer paths end by the roulette when it starts later, and the rest of every path
    # up to collision 2 is the plain one's
    assert 0 < ((b["flags"] & 32) != 0).sum() < ((c["flags"] & 32) != 0).sum()
    assert not np.array_equal(b["L"], c["L"])
