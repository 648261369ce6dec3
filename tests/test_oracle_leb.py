"""Pins of the oracle's grid construction (Sec. 2) against what the paper and the
geometry fix: the 24-tetrahedron control cube, uniform counts, conformity,
exact volumes, longest-edge refinement, 18 face orientations, brute-force
density statistics, order independence and minimality of the closure."""
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests import _checks as CK
from tests.conftest import control_cube_tets, paper_count, scene_volume


def uniform_grid(dims, depth, value=0.5):
    vol = np.full(dims[::-1], value, np.float32)
    return O.Grid(vol, (0, 0, 0), 1.0 / min(dims), theta=-1.0, max_depth=depth)


@pytest.mark.parametrize("depth", [0, 1, 2, 3, 5, 8])
def test_uniform_counts_and_invariants(depth):
    g = uniform_grid((16, 16, 16), depth)
    a = g.export()
    assert len(a.codes) == 6 * 2 ** depth
    assert np.all(O.code_depth(a.codes) == depth)
    CK.check_grid(a)


def test_tiny_scene_is_uniform_depth_12(tiny_volume):
    s = W.scene("tiny")
    a = O.Grid.for_scene(s, tiny_volume).export()
    assert len(a.codes) == 24576                     # 6 * 2^12
    CK.check_grid(a)
    assert set(np.unique(a.nid)) == set(range(paper_count("face_orientations")))   # Sec. 3
    assert a.nbr.shape[1] == paper_count("max_neighbours")


def test_depth2_is_the_24_halfedge_control_cube():
    """Sec. 2: the control cube is tessellated into 24 tetrahedra, one per halfedge:
    the halfedge's two vertices, the centre of the face carrying it and the cube centre."""
    g = uniform_grid((8, 8, 8), 2)
    a = g.export()
    S = 1 << a.K
    assert len(a.codes) == paper_count("control_cube_tets")
    # the same tetrahedra as the paper's list (tests/golden), vertex sets compared
    want = control_cube_tets()
    assert len(want) == len(set(want)) == paper_count("control_cube_tets")
    got = {frozenset(tuple(int(c) // (S // 2) for c in v) for v in T) for T in a.verts}
    assert all(int(c) % (S // 2) == 0 for T in a.verts for v in T for c in v)
    assert got == set(want)
    seen = set()
    for T in a.verts:
        pts = {tuple(int(c) for c in v) for v in T}
        centre = (S // 2,) * 3
        assert centre in pts
        corners = [p for p in pts if all(c in (0, S) for c in p)]
        assert len(corners) == 2
        e0, e1 = corners
        diff = [i for i in range(3) if e0[i] != e1[i]]
        assert len(diff) == 1                         # a cube edge
        face = [p for p in pts if p != centre and p not in corners]
        assert len(face) == 1
        fc = face[0]
        assert sorted(fc).count(S // 2) == 2          # a face centre
        fixed = [i for i in range(3) if fc[i] != S // 2][0]
        assert e0[fixed] == e1[fixed] == fc[fixed]    # the face carries the edge
        seen.add((tuple(sorted([e0, e1])), fc))
    assert len(seen) == 24                            # 12 edges x 2 faces each


@pytest.mark.parametrize("name", ["adaptive_small", "production_small"])
def test_adaptive_scene_invariants(name):
    s = W.scene(name)
    a = O.Grid.for_scene(s, scene_volume(name)).export()
    CK.check_grid(a)
    assert a.max_depth <= s.max_depth
    assert len(np.unique(O.code_depth(a.codes))) > 5   # genuinely adaptive


def test_empty_volume_keeps_the_roots():
    vol = np.zeros((16, 16, 16), np.float32)
    s = W.scene("adaptive_small")
    g = O.Grid(vol, (0, 0, 0), 1 / 16, camera=s.camera, footprint_px=1.0, theta=0.5, max_depth=12)
    a = g.export()
    assert len(a.codes) == 6 and np.all(a.density == 0)
    CK.check_grid(a)


def test_codes_follow_the_bisection_rule():
    """Replaying Maubach's rule along each code's path bits from its Kuhn root gives the
    exported vertices (independent replay in Python)."""
    s = W.scene("adaptive_small")
    a = O.Grid.for_scene(s, scene_volume("adaptive_small")).export()
    S = 1 << a.K
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    rng = np.random.default_rng(0)
    for i in rng.choice(len(a.codes), 300, replace=False):
        code = int(a.codes[i])
        root, depth = code >> 56, code & 63
        bits = (code >> 6) & ((1 << 50) - 1)
        cube, perm = divmod(root, 6)
        C = a.cubes
        base = [(cube % C[0]) * S, (cube // C[0] % C[1]) * S, (cube // (C[0] * C[1])) * S]
        x = [tuple(base)]
        cur = list(base)
        for ax in perms[perm]:
            cur[ax] += S
            x.append(tuple(cur))
        k = 3
        for d in range(depth):
            b = (bits >> (49 - d)) & 1
            z = tuple((p + q) // 2 for p, q in zip(x[0], x[k]))
            x = (x[:k] if b == 0 else x[1:k + 1]) + [z] + x[k + 1:]
            k = k - 1 if k > 1 else 3
        assert [tuple(v) for v in a.verts[i].tolist()] == x
        assert int(a.tag[i]) == k


def _brute_stats(vol_q, verts, K, n):
    """D by testing every voxel centre of the volume against the closed tetrahedron
    (exact integer orientations)."""
    nz, ny, nx = vol_q.shape
    h = 1 << (K - int(np.log2(n)) - 1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    P = np.stack([(2 * i + 1) * h, (2 * j + 1) * h, (2 * k + 1) * h], -1).reshape(-1, 3).astype(np.int64)
    v = verts.astype(np.int64)
    inside = np.ones(len(P), bool)
    for f in range(4):
        q = [v[t] for t in range(4) if t != f]
        nrm = np.cross(q[1] - q[0], q[2] - q[0])
        sref = np.sign(nrm @ (v[f] - q[0]))
        sp = np.sign((P - q[0]) @ nrm)
        inside &= (sp == 0) | (sp == sref)
    vals = vol_q.reshape(-1)[inside]
    if len(vals) == 0:
        cen = v.sum(0)
        idx = [min(max(int(c) >> (K + 2 - int(np.log2(n))), 0), dim - 1) for c, dim in zip(cen, (nx, ny, nz))]
        vals = np.array([vol_q[idx[2], idx[1], idx[0]]])
    return len(vals), int(vals.sum()), int(vals.min()), int(vals.max())


def test_density_statistics_by_brute_force():
    s = W.scene("adaptive_small")
    vol = scene_volume("adaptive_small")
    a = O.Grid.for_scene(s, vol).export()
    q = np.clip(np.rint(vol.astype(np.float64) * 2 ** 24), 0, 2 ** 24).astype(np.int64)
    rng = np.random.default_rng(1)
    depth = O.code_depth(a.codes)
    picks = list(rng.choice(len(a.codes), 60, replace=False)) + list(np.nonzero(depth == depth.min())[0][:4])
    for i in picks:
        c, sm, mn, mx = _brute_stats(q, a.verts[i], a.K, a.voxels_per_cube)
        assert (a.count[i], a.sum[i], a.qmin[i], a.qmax[i]) == (c, sm, mn, mx)
        mean = np.float32(np.float64(sm) / (np.float64(c) * 2.0 ** 24))
        assert a.density[i] == mean
        assert a.majorant[i] == np.float32(mx / 2.0 ** 24)


@pytest.mark.parametrize("fmt,dtype", [(1, torch.bfloat16), (2, torch.float16)])
def test_density_storage_rounding(fmt, dtype):
    """Stored densities are the fp32 mean rounded to nearest-even in bf16 / fp16
    (checked against torch's own conversions)."""
    s = W.scene("adaptive_small", density_format=fmt)
    vol = scene_volume("adaptive_small")
    a32 = O.Grid.for_scene(W.scene("adaptive_small"), vol).export()
    a = O.Grid.for_scene(s, vol).export()
    assert np.array_equal(a.codes, a32.codes)
    ref = torch.from_numpy(a32.density).to(dtype).to(torch.float32).numpy()
    assert np.array_equal(a.density, ref)


def test_variation_criterion_exact():
    """Sec. 2 criterion 1 with the camera criterion off: split <=> depth < max and
    (max - min) / mean > theta, evaluated in exact rationals from the statistics."""
    s = W.scene("adaptive_small")
    vol = scene_volume("adaptive_small")
    rng = np.random.default_rng(2)
    pts = rng.uniform(0, 1, (200, 3))
    for theta in (0.0, 0.5, 1.75):
        pr = O.path_profile(vol, s.box_min, s.voxel_size, None, 0.0, theta, 12, 0, pts)
        th = Fraction(int(round(theta * 65536)), 65536)
        for p in range(len(pts)):
            for d in range(13):
                c, sm, mn, mx = (int(pr["count"][p, d]), int(pr["sum"][p, d]), int(pr["qmin"][p, d]),
                                 int(pr["qmax"][p, d]))
                want = d < 12 and sm > 0 and Fraction(mx - mn) / Fraction(sm, c) > th
                assert bool(pr["split"][p, d]) == want


def _camera_frame(cam):
    f = np.subtract(cam.target, cam.pos); f = f / np.linalg.norm(f)
    r = np.cross(f, cam.up); r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    return np.array(cam.pos, np.float64), f, r, u


def _code_vertices(code, cubes=(1, 1, 1)):
    """Vertices (in cubes) of an LEB code, replayed from its Kuhn root."""
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    root, d, bits = code >> 56, code & 63, (code >> 6) & ((1 << 50) - 1)
    cube = root // 6
    base = np.array([cube % cubes[0], cube // cubes[0] % cubes[1], cube // (cubes[0] * cubes[1])], np.float64)
    x = [base.copy()]
    cur = base.copy()
    for ax in perms[root % 6]:
        cur = cur.copy(); cur[ax] += 1; x.append(cur)
    k = 3
    for dd in range(d):
        b = (bits >> (49 - dd)) & 1
        z = (x[0] + x[k]) / 2
        x = (x[:k] if b == 0 else x[1:k + 1]) + [z] + x[k + 1:]
        k = k - 1 if k > 1 else 3
    return np.array(x)


def test_camera_criterion_bounds():
    """Sec. 2 criterion 2 through the image: with the variation criterion off,
    (a) a cell whose four vertices project into the image over more than 4 pixels
    is split (the footprint bounds the projected extent from above, to within a
    factor 1 + tan(half fov)); (b) a cell whose vertices all project beyond one
    image edge, or lie behind the eye, is not; (c) splitting is monotone down the
    hierarchy: a cell the criterion keeps has children it keeps."""
    s = W.with_camera(W.scene("adaptive_small"), fov_y_deg=15.0)    # narrow: much of the box out of view
    vol = scene_volume("adaptive_small")
    cam = s.camera
    eye, f, r, u = _camera_frame(cam)
    tanF = np.tan(np.radians(cam.fov_y_deg) / 2)
    rng = np.random.default_rng(3)
    pts = np.concatenate([rng.uniform(0, 1, (150, 3)), rng.uniform(0, 1, (50, 3)) * [1, 0.05, 1]])
    md = 18
    pr = O.path_profile(vol, s.box_min, s.voxel_size, cam, 1.0, -1.0, md, 0, pts)
    sp = pr["split"].astype(bool)
    assert np.all(sp[:, 1:md] <= sp[:, 0:md - 1])                       # (c)
    big = outside = 0
    for p in range(len(pts)):
        for d in range(md):
            X = _code_vertices(int(pr["codes"][p, d]))      # grid space == world space (box at 0, cube 1)
            rel = X - eye
            zc, xc, yc = rel @ f, rel @ r, rel @ u
            if np.all(zc < 1e-3):
                assert not sp[p, d]; outside += 1
                continue
            if np.any(zc <= 1e-3):
                continue
            pxs = (xc / (zc * tanF * cam.width / cam.height) + 1) * cam.width / 2
            pys = (yc / (zc * tanF) + 1) * cam.height / 2
            if np.all(pxs < 0) or np.all(pxs > cam.width) or np.all(pys < 0) or np.all(pys > cam.height):
                assert not sp[p, d]; outside += 1                         # (b)
                continue
            ext = max(pxs.max() - pxs.min(), pys.max() - pys.min())
            inside = np.all((pxs > 0) & (pxs < cam.width) & (pys > 0) & (pys < cam.height))
            if ext > 4 and inside:
                assert sp[p, d]; big += 1                                # (a)
    assert big > 10 and outside > 10


def _python_random_order_build(s, vol, seed):
    """Independent Python closure with a random, sequential split order: sweep the
    leaves in a shuffled order and bisect at once every leaf that the criterion
    selects or that has a vertex at one of its edge midpoints, until a sweep
    splits nothing.  The criterion of a cell is read from the oracle's descent
    profile at its centroid."""
    rnd = random.Random(seed)
    K = O.Grid(vol, s.box_min, s.voxel_size, max_depth=s.max_depth, theta=-1).info()["K"]
    S = 1 << K
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    leaves = {}
    for r, perm in enumerate(perms):
        x = [(0, 0, 0)]
        cur = [0, 0, 0]
        for ax in perm:
            cur[ax] += S
            x.append(tuple(cur))
        leaves[(r, 0, 0)] = (x, 3)

    crit_cache = {}

    def crit(key, x):
        if key not in crit_cache:
            cen = np.array(x, np.float64).mean(0)[None] * 2.0 ** (-K)
            pr = O.path_profile(vol, s.box_min, s.voxel_size, s.camera, s.footprint_px, s.variation_threshold,
                                s.max_depth, 0, cen)
            crit_cache[key] = bool(pr["split"][0, key[1]])
        return crit_cache[key]

    verts = {v for x, _ in leaves.values() for v in x}

    def marked(key, x):
        if crit(key, x):
            return True
        for i in range(4):
            for j in range(i + 1, 4):
                sm = [p + q for p, q in zip(x[i], x[j])]
                if all(c % 2 == 0 for c in sm) and tuple(c // 2 for c in sm) in verts:
                    return True
        return False

    changed = True
    while changed:
        changed = False
        keys = list(leaves)
        rnd.shuffle(keys)
        for key in keys:
            if key not in leaves or not marked(key, leaves[key][0]):
                continue
            x, k = leaves.pop(key)
            z = tuple((p + q) // 2 for p, q in zip(x[0], x[k]))
            verts.add(z)
            kk = k - 1 if k > 1 else 3
            r, d, path = key
            leaves[(r, d + 1, path << 1)] = (x[:k] + [z] + x[k + 1:], kk)
            leaves[(r, d + 1, (path << 1) | 1)] = (x[1:k + 1] + [z] + x[k + 1:], kk)
            changed = True
    codes = sorted((r << 56) | (((path << (56 - d)) & ((1 << 56) - 1)) if d else 0) | d for r, d, path in leaves)
    return np.array(codes, np.uint64), leaves, K


def test_order_independence_and_minimality():
    s = W.scene("adaptive_small", dims=(16, 16, 16), voxel_size=1 / 16, max_depth=9)
    vol = scene_volume("adaptive_small", dims=(16, 16, 16), voxel_size=1 / 16, max_depth=9)
    ref = O.Grid.for_scene(s, vol).export()
    for seed in (0, 1):
        codes, leaves, K = _python_random_order_build(s, vol, seed)
        assert np.array_equal(codes, ref.codes)
    # minimality: a sibling pair whose parent the criterion does not split exists only
    # because its split vertex z is shared with another cell (merging would hang z)
    byk = {}
    for i, c in enumerate(ref.codes):
        byk[int(c)] = i
    owners = {}
    for i in range(len(ref.codes)):
        for v in ref.verts[i]:
            owners.setdefault(tuple(int(c) for c in v), set()).add(i)
    checked = 0
    for i, c in enumerate(ref.codes):
        c = int(c)
        d = c & 63
        if d == 0 or (c >> (56 - d)) & 1:
            continue
        sib = c | (1 << (56 - d))
        if sib not in byk:
            continue
        j = byk[sib]
        # z sits at the parent's tag position k in both children; a child's tag is k - 1 (or 3 if k = 1)
        kp = int(ref.tag[i]) % 3 + 1
        z = tuple(int(v) for v in ref.verts[i][kp])
        assert z == tuple(int(v) for v in ref.verts[j][kp])
        par = ({tuple(int(v) for v in a) for a in ref.verts[i]} | {tuple(int(v) for v in b) for b in ref.verts[j]}) - {z}
        assert len(par) == 4
        parent_code = (c & ~((1 << (57 - d)) - 1)) | (d - 1)
        cen = np.array(sorted(par), np.float64).mean(0)[None] * 2.0 ** (-ref.K)
        pr = O.path_profile(vol, s.box_min, s.voxel_size, s.camera, s.footprint_px, s.variation_threshold,
                            s.max_depth, 0, cen)
        assert int(pr["codes"][0, d - 1]) == parent_code
        if not pr["split"][0, d - 1]:
            assert len(owners[z] - {i, j}) > 0, "closure split a cell it did not need to"
            checked += 1
    assert checked > 0
