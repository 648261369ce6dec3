"""Pins of the oracle's estimator (Sec. 3, Algorithm 1 with sun next-event
estimation): white furnace, exponential free flights (escape probability
exp(-tau)), single scattering against 1D quadrature, Henyey-Greenstein
sampling and density, on the tet grid and on the regular-grid comparator."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests import _checks as CK
from tests.conftest import scene_volume


def camera_rays(cam, seed, px, py, sm, cube=1.0, box_min=(0, 0, 0)):
    """Grid-space camera rays of the given paths (pinhole, y down, Philox jitter)."""
    f = np.subtract(cam.target, cam.pos); f = f / np.linalg.norm(f)
    r = np.cross(f, cam.up); r = r / np.linalg.norm(r)
    u = np.cross(r, f); u = u / np.linalg.norm(u)
    tanF = math.tan(math.radians(cam.fov_y_deg) / 2)
    asp = cam.width / cam.height
    o = (np.array(cam.pos) - np.array(box_min)) / cube
    D = []
    for x, y, s in zip(px, py, sm):
        pix = int(y) * cam.width + int(x)
        u0, u1 = O.uniform(seed, pix, int(s), 0), O.uniform(seed, pix, int(s), 1)
        fx, fy = (x + u0) / cam.width, (y + u1) / cam.height
        dd = f + (2 * fx - 1) * tanF * asp * r - (2 * fy - 1) * tanF * u
        D.append(dd / np.linalg.norm(dd))
    return o, np.array(D)


def all_paths(cam, spp):
    py, px, sm = np.meshgrid(np.arange(cam.height), np.arange(cam.width), np.arange(spp), indexing="ij")
    return px.ravel().astype(np.int32), py.ravel().astype(np.int32), sm.ravel().astype(np.int32)


def test_white_furnace(tiny_volume):
    """albedo 1, environment 1, no sun: every path that is not truncated returns exactly 1."""
    s = W.scene("tiny")
    g = O.Grid.for_scene(s, tiny_volume)
    med = W.Medium(1.0, 0.3, 30.0, 100000, s.medium.sun_dir, 0.0, 1.0)
    px, py, sm = all_paths(s.camera, 2)
    res = g.render_paths(s.camera, med, 11, px, py, sm)
    ok = (res["flags"] & 2) == 0
    assert ok.mean() > 0.999
    assert np.all(res["L"][ok] == 1.0)
    assert res["collisions"].max() > 20


def _homog(n=16, value=0.5):
    return np.full((n, n, n), value, np.float32)


@pytest.mark.parametrize("kind", ["tet", "dda"])
def test_escape_probability_is_exp_minus_tau(kind):
    """max_bounces 1, environment 1, sun off: L = 1 iff the camera ray crosses the
    medium without a collision, with probability exp(-sigma rho chord)."""
    vol = _homog()
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 40.0, 48, 40)
    med = W.Medium(0.7, 0.0, 3.0, 1, (0, -1, 0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 8)
    if kind == "tet":
        g = O.Grid(vol, (0, 0, 0), 1 / 16, theta=-1, max_depth=6)
        res = g.render_paths(cam, med, 5, px, py, sm)
    else:
        res = O.dda_render_paths(vol, (0, 0, 0), 1 / 16, cam, med, 5, px, py, sm)
    o, D = camera_rays(cam, 5, px, py, sm)
    p = np.empty(len(px))
    for i in range(len(px)):
        se = CK.slab(o, D[i], (1, 1, 1))
        p[i] = 1.0 if se is None else math.exp(-3.0 * 0.5 * (se[1] - se[0]))
    L = res["L"]
    assert set(np.unique(L)) <= {0.0, 1.0}
    sd = math.sqrt(np.sum(p * (1 - p)))
    assert abs(L.sum() - p.sum()) < 4 * sd


@pytest.mark.parametrize("kind", ["tet", "dda"])
def test_single_scattering_matches_quadrature(kind):
    """max_bounces 1, sun only: E[L | ray] = int_0^chord sigma e^{-sigma t} albedo
    p(d . w) E e^{-sigma s(t)} dt, s(t) the distance to the boundary towards the sun."""
    rho, sig, alb, gg, E = 0.5, 4.0, 0.7, 0.4, 2.0
    vol = _homog(value=rho)
    cam = W.Camera((0.5, 0.6, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 16, 16)
    sun = np.array([-1.0, -2.0, 0.5]); sun /= np.linalg.norm(sun)
    med = W.Medium(alb, gg, sig, 1, tuple(sun), E, 0.0)
    px, py, sm = all_paths(cam, 64)
    if kind == "tet":
        g = O.Grid(vol, (0, 0, 0), 1 / 16, theta=-1, max_depth=6)
        res = g.render_paths(cam, med, 9, px, py, sm)
    else:
        res = O.dda_render_paths(vol, (0, 0, 0), 1 / 16, cam, med, 9, px, py, sm)
    o, D = camera_rays(cam, 9, px, py, sm)
    w = -sun
    st = sig * rho
    # composite Gauss-Legendre, 128 panels x 8 nodes, vectorised over the rays
    xg, wg = np.polynomial.legendre.leggauss(8)
    q = np.zeros(len(px))
    t_in, t_len = np.zeros(len(px)), np.zeros(len(px))
    for i in range(len(px)):
        se = CK.slab(o, D[i], (1, 1, 1))
        if se is not None:
            t_in[i], t_len[i] = se[0], se[1] - se[0]
    P = 128
    a_ = (np.arange(P)[:, None] + (xg[None, :] + 1) / 2).reshape(-1) / P      # nodes in [0, 1]
    wq = np.tile(wg / 2, P) / P
    t = a_[None, :] * t_len[:, None]                                          # (R, M)
    X = o[None, None, :] + (t_in[:, None] + t)[:, :, None] * D[:, None, :]
    with np.errstate(divide="ignore"):
        sx = np.where(w > 0, (1 - X) / w, np.where(w < 0, (0 - X) / w, np.inf))
    s_exit = np.maximum(sx.min(axis=2), 0)
    ph = np.array([O.hg_pdf(gg, float(D[i] @ w)) for i in range(len(px))])
    f = st * np.exp(-st * t) * alb * ph[:, None] * E * np.exp(-st * s_exit)
    q = (f * wq[None, :]).sum(1) * t_len
    L = res["L"]
    diff = L - q
    assert abs(diff.mean()) < 4 * diff.std() / math.sqrt(len(L))
    assert np.all(res["collisions"] <= 1)


def test_heterogeneous_escape_probability_on_both_grids():
    """Random 8^3 medium: the probability that a camera ray escapes uncollided is
    exp(-tau), tau by brute-force clipping with every tetrahedron (tet grid) or
    every voxel (regular grid)."""
    rng = np.random.default_rng(7)
    vol = rng.uniform(0, 1, (8, 8, 8)).astype(np.float32)
    cam = W.Camera((0.4, 0.55, -1.4), (0.5, 0.5, 0.5), (0, 1, 0), 35.0, 24, 20)
    med = W.Medium(0.5, 0.0, 2.0, 1, (0, -1, 0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 16)
    o, D = camera_rays(cam, 21, px, py, sm)
    g = O.Grid(vol, (0, 0, 0), 1 / 8, theta=0.2, max_depth=9)
    a = g.export()
    tet = g.render_paths(cam, med, 21, px, py, sm)["L"]
    dda = O.dda_render_paths(vol, (0, 0, 0), 1 / 8, cam, med, 21, px, py, sm)["L"]
    # voxel boxes
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    lo = np.stack([i, j, k], -1).reshape(-1, 3) / 8.0
    hi = lo + 1 / 8.0
    rv = vol.reshape(-1).astype(np.float64)
    p_t, p_v = np.zeros(len(px)), np.zeros(len(px))
    for r in range(len(px)):
        se = CK.slab(o, D[r], (1, 1, 1))
        if se is None:
            p_t[r] = p_v[r] = 1.0
            continue
        t0, t1 = CK.clip_all_tets(a.verts, a.K, o, D[r])
        ch = np.maximum(np.minimum(t1, se[1]) - np.maximum(t0, se[0]), 0)
        p_t[r] = math.exp(-2.0 * np.sum(a.density * ch))
        with np.errstate(divide="ignore", invalid="ignore"):
            ta, tb = (lo - o) / D[r], (hi - o) / D[r]
        tn = np.nanmax(np.minimum(ta, tb), 1)
        tf = np.nanmin(np.maximum(ta, tb), 1)
        ch = np.maximum(np.minimum(tf, se[1]) - np.maximum(tn, se[0]), 0)
        p_v[r] = math.exp(-2.0 * np.sum(rv * ch))
    for L, p in ((tet, p_t), (dda, p_v)):
        sd = math.sqrt(np.sum(p * (1 - p)))
        assert abs(L.sum() - p.sum()) < 4 * sd


@pytest.mark.parametrize("g", [-0.3, 0.0, 0.5, 0.9])
def test_henyey_greenstein_sampling(g):
    rng = np.random.default_rng(int(g * 100) + 50)
    n = 20000
    d = rng.normal(size=3); d /= np.linalg.norm(d)
    u = rng.uniform(0, 1, (n, 2))
    cos = np.empty(n)
    for i in range(n):
        w = O.hg_sample(g, u[i, 0], u[i, 1], d)
        assert abs(np.linalg.norm(w) - 1) < 1e-12
        cos[i] = np.dot(w, d)
    # E[cos] = g
    assert abs(cos.mean() - g) < 4 * cos.std() / math.sqrt(n) + 1e-12
    # chi^2 of the cos histogram against the density 2 pi p(cos)
    edges = np.linspace(-1, 1, 41)
    obs, _ = np.histogram(cos, edges)
    pdf = lambda c: 2 * math.pi * O.hg_pdf(g, c)
    exp = np.array([integrate.quad(pdf, a, b)[0] for a, b in zip(edges[:-1], edges[1:])]) * n
    keep = exp > 5
    chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4
    # the azimuth about d is uniform (any orthonormal frame of d: here Gram-Schmidt on e_x or e_y)
    a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    t = a - (a @ d) * d; t /= np.linalg.norm(t)
    b = np.cross(d, t)
    W_ = np.array([O.hg_sample(g, u[i, 0], u[i, 1], d) for i in range(n)])
    phi = np.mod(np.arctan2(W_ @ b, W_ @ t), 2 * math.pi)
    obs, _ = np.histogram(phi, np.linspace(0, 2 * math.pi, 17))
    chi2 = np.sum((obs - n / 16) ** 2 / (n / 16))
    assert stats.chi2.sf(chi2, 15) > 1e-4


@pytest.mark.parametrize("g", [-0.5, 0.0, 0.3, 0.95])
def test_henyey_greenstein_density_normalised(g):
    tot = integrate.quad(lambda c: 2 * math.pi * O.hg_pdf(g, c), -1, 1, points=[1.0], limit=200)[0]
    assert tot == pytest.approx(1.0, abs=1e-9)
    if g == 0:
        assert O.hg_pdf(0.0, 0.3) == pytest.approx(1 / (4 * math.pi))


@pytest.mark.parametrize("heterogeneous", [False, True])
def test_collision_distances_are_exponential(heterogeneous):
    """Free flights (Algorithm 1, SampleFreePath + MarchThroughCells): in a medium
    that is homogeneous along each ray, the distance s from the entry point to
    the first collision, given a collision, has F(s) = (1 - e^{-mu s}) / (1 - e^{-mu l})
    (l the chord); the probability transforms u = F(s) of all paths are uniform
    (Kolmogorov-Smirnov).  The heterogeneous case has densities 0.2 and 0.8 in the
    halves x < 1/2 and x >= 1/2 (cell faces lie on x = 1/2 at this depth) and uses
    the rays that stay in one half, each with its own rate."""
    rho, sig = 0.5, 3.0
    n = 16
    vol = np.full((n, n, n), rho, np.float32)
    if heterogeneous:
        vol[:, :, : n // 2] = 0.2
        vol[:, :, n // 2:] = 0.8
    g = O.Grid(vol, (0, 0, 0), 1 / n, theta=-1, max_depth=6)
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 8.0, 40, 40)   # nearly parallel to +z
    med = W.Medium(0.7, 0.0, sig, 4, (0, -1, 0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 32)
    q = g.cache_paths(cam, med, 17, px, py, sm, cache_depth=1)["query"]
    hit = q[:, 3] > 0
    o, D = camera_rays(cam, 17, px, py, sm)
    u = []
    for i in np.nonzero(hit)[0]:
        se = CK.slab(o, D[i], (1, 1, 1))
        t_in, chord = se[0], se[1] - se[0]
        xa, xb = (o + t_in * D[i])[0], (o + se[1] * D[i])[0]
        if (xa < 0.5) != (xb < 0.5):
            continue                                    # the ray crosses x = 1/2
        x = q[i, 0:3]                                   # grid position (domain extent 1)
        s = float(np.dot(x - (o + t_in * D[i]), D[i]))
        xi = int(min(max(np.floor(xa * n), 0), n - 1))
        mu = sig * float(vol[0, 0, xi])
        u.append((1 - math.exp(-mu * s)) / (1 - math.exp(-mu * chord)))
    u = np.array(u)
    assert len(u) > 10000
    assert np.all((u >= 0) & (u <= 1 + 1e-12))
    assert stats.kstest(u, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("kind", ["tet", "dda"])
def test_image_orientation(kind):
    """The pixel convention (y down, right = forward x up): a camera on the -z side
    looking along +z with up +y sees world x < 1/2 on the right of the image and
    y > 1/2 in its top rows.  An absorbing block filling x < 1/2, y > 1/2 through
    the whole depth darkens exactly the top-right quadrant; every other ray crosses
    empty space and returns the environment, 1.  A mirrored axis or a flipped row
    order anywhere in the camera model moves the dark quadrant."""
    vol = np.zeros((16, 16, 16), np.float32)
    vol[:, 8:, :8] = 1.0                                  # [z][y][x]: y > 1/2, x < 1/2
    cam = W.Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 12, 16)   # every ray meets the front face
    med = W.Medium(0.0, 0.0, 60.0, 4, (0.0, -1.0, 0.0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 2)
    if kind == "tet":
        L = O.Grid(vol, (0, 0, 0), 1 / 16, theta=0.1, max_depth=9).render_paths(cam, med, 5, px, py, sm)["L"]
    else:
        L = O.dda_render_paths(vol, (0, 0, 0), 1 / 16, cam, med, 5, px, py, sm)["L"]
    right, top = px >= cam.width // 2, py < cam.height // 2
    dark = right & top
    assert np.all(L[~dark] == 1.0)
    assert L[dark].max() < 1e-6


def test_albedo_multiplies_once_per_collision():
    """No sun, environment 1: a path that escapes after k collisions returns exactly
    albedo^k (the throughput is multiplied by the albedo at every collision), and a
    truncated path returns 0."""
    vol = _homog(value=0.8)
    cam = W.Camera((0.5, 0.6, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 30.0, 16, 16)
    alb = 0.75
    med = W.Medium(alb, 0.2, 6.0, 12, (0.0, -1.0, 0.0), 0.0, 1.0)
    px, py, sm = all_paths(cam, 8)
    res = O.Grid(vol, (0, 0, 0), 1 / 16, theta=-1, max_depth=6).render_paths(cam, med, 13, px, py, sm)
    trunc = (res["flags"] & 2) != 0
    k = res["collisions"][~trunc].astype(np.int64)
    assert k.max() >= 4 and trunc.any()
    assert np.allclose(res["L"][~trunc], alb ** k, rtol=1e-12, atol=0)
    assert np.all(res["L"][trunc] == 0.0)
