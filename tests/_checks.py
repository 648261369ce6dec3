"""Structural checks of a tetrahedral grid that hold at any size (numpy only).

They follow what the paper states about LEB grids: conforming (every interior
face shared by exactly two cells, Sec. 1), at most four neighbours, a
refinement edge that is the longest edge (Sec. 2), and 18 face orientations
(Sec. 3).  Used both to pin the oracle and to check GPU-built grids.
"""
import numpy as np

P9 = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, -1, 0],
               [0, 1, 1], [0, 1, -1], [1, 0, 1], [1, 0, -1]], np.int64)


def face_vertices(verts, f):
    idx = [i for i in range(4) if i != f]
    return verts[:, idx, :]


def six_volumes(verts):
    v = verts.astype(np.int64)
    a, b, c = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]
    return np.abs(np.einsum("ni,ni->n", a, np.cross(b, c)))


def check_volumes(verts, codes, K, cubes):
    """6 vol(T) = 6 vol(root) / 2^depth exactly, and the cells tile the domain."""
    depth = (codes & np.uint64(63)).astype(np.int64)
    sv = six_volumes(verts)
    expect = (np.int64(1) << np.int64(3 * K)) >> depth
    assert np.array_equal(sv, expect), "cell volume differs from root volume / 2^depth"
    assert int(sv.sum()) == 6 * int(np.prod(cubes)) * (1 << (3 * K)), "cells do not tile the domain"


def check_longest_edge(verts, tag):
    """The refinement edge x0-x_tag is the unique longest edge."""
    v = verts.astype(np.int64)
    L = {}
    for i in range(4):
        for j in range(i + 1, 4):
            d = v[:, i] - v[:, j]
            L[(i, j)] = (d * d).sum(1)
    ref = np.choose(tag - 1, [L[(0, 1)], L[(0, 2)], L[(0, 3)]])
    others_max = np.zeros_like(ref)
    for (i, j), l in L.items():
        is_ref = (i == 0) & (j == tag)
        others_max = np.maximum(others_max, np.where(is_ref, 0, l))
    assert np.all(ref > others_max), "refinement edge is not the unique longest edge"


def _face_keys(verts):
    """(N, 4, 9) sorted vertex triples of every face."""
    N = len(verts)
    keys = np.empty((N, 4, 9), np.int64)
    for f in range(4):
        fv = face_vertices(verts, f).astype(np.int64)            # (N,3,3)
        packed = (fv[:, :, 0] << 42) | (fv[:, :, 1] << 21) | fv[:, :, 2]
        order = np.argsort(packed, axis=1)
        fv = np.take_along_axis(fv, order[:, :, None], axis=1)
        keys[:, f, :] = fv.reshape(N, 9)
    return keys


def check_conforming(verts, nbr, K, cubes):
    """Every face is shared by exactly two cells, or lies on the domain boundary and
    belongs to one; neighbour links are symmetric and join the shared face."""
    N = len(verts)
    keys = _face_keys(verts)
    flat = keys.reshape(-1, 9)
    _, inv, cnt = np.unique(flat, axis=0, return_inverse=True, return_counts=True)
    mult = cnt[inv.reshape(-1)].reshape(N, 4)
    assert mult.max() <= 2, "a face is shared by more than two cells"
    boundary = mult == 1
    lim = np.array(cubes, np.int64) << K
    on_bnd = np.zeros((N, 4), bool)
    for a in range(3):
        xa = keys[:, :, a::3]
        on_bnd |= np.all(xa == 0, axis=2) | np.all(xa == lim[a], axis=2)
    assert np.all(on_bnd[boundary]), "a face with one cell lies inside the domain (hanging face)"
    assert np.array_equal(boundary, nbr < 0), "boundary links differ from unshared faces"
    i, f = np.nonzero(nbr >= 0)
    j = nbr[i, f]
    back = nbr[j]                                        # (M,4)
    hits = back == i[:, None]
    assert np.all(hits.sum(1) == 1), "neighbour links are not symmetric"
    g = np.argmax(hits, axis=1)
    assert np.array_equal(keys[i, f], keys[j, g]), "linked cells do not share the face"
    assert np.all(nbr < N)


def check_normals(verts, nid, plane, K):
    """nid = p + 9 s names the outward face normal (-1)^s P9[p]; plane = P9[p] . v for
    the face's vertices (in cubes)."""
    v = verts.astype(np.int64)
    assert nid.max() < 18
    for f in range(4):
        fv = face_vertices(v, f)
        n = np.cross(fv[:, 1] - fv[:, 0], fv[:, 2] - fv[:, 0])
        out = np.einsum("ni,ni->n", n, v[:, f] - fv[:, 0]) > 0
        n[out] = -n[out]
        p = nid[:, f].astype(np.int64) % 9
        s = np.where(nid[:, f] >= 9, -1, 1)
        expect = P9[p] * s[:, None]
        # n must be a positive multiple of expect
        scale = np.abs(n).max(1)
        assert np.all(scale > 0)
        assert np.array_equal(n, expect * scale[:, None]), "normal id does not match the face"
        for k in range(3):
            c = np.einsum("ni,ni->n", P9[p], fv[:, k]).astype(np.float64) * 2.0 ** (-K)
            assert np.array_equal(c.astype(np.float32), plane[:, f]), "plane offset differs"


def check_codes(codes):
    """Codes are unique and in depth-first pre-order (sorted)."""
    assert np.all(codes[1:] > codes[:-1]), "codes not strictly increasing"


def check_grid(arr, K=None, cubes=None):
    K = arr.K if K is None else K
    cubes = arr.cubes if cubes is None else cubes
    check_codes(arr.codes)
    check_volumes(arr.verts, arr.codes, K, cubes)
    check_longest_edge(arr.verts, arr.tag)
    check_conforming(arr.verts, arr.nbr, K, cubes)
    check_normals(arr.verts, arr.nid, arr.plane, K)


# ---------------------------------------------------------------------------
# brute-force ray clipping against every cell (tiny grids only)
# ---------------------------------------------------------------------------
def clip_all_tets(verts, K, o, d):
    """Parametric interval [t0, t1] of the ray o + t d inside every tetrahedron
    (grid space, cubes), from the four face half-spaces."""
    v = verts.astype(np.float64) * 2.0 ** (-K)
    t0 = np.full(len(v), -np.inf)
    t1 = np.full(len(v), np.inf)
    for f in range(4):
        fv = face_vertices(v, f)
        n = np.cross(fv[:, 1] - fv[:, 0], fv[:, 2] - fv[:, 0])
        out = np.einsum("ni,ni->n", n, v[:, f] - fv[:, 0]) > 0
        n[out] = -n[out]                                   # outward
        c = np.einsum("ni,ni->n", n, fv[:, 0])
        nd = n @ d
        no = n @ o
        # inside: n.(o + t d) <= c
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (c - no) / nd
        pos = nd > 0
        neg = nd < 0
        t1 = np.where(pos, np.minimum(t1, t), t1)
        t0 = np.where(neg, np.maximum(t0, t), t0)
        zero = nd == 0
        t1 = np.where(zero & (no > c), -np.inf, t1)
    return t0, t1


def slab(o, d, hi):
    """Entry/exit parameters of the ray in the box [0, hi]."""
    tn, tf = 0.0, np.inf
    for a in range(3):
        if d[a] == 0:
            if o[a] < 0 or o[a] > hi[a]:
                return None
            continue
        t1, t2 = (0 - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        tn, tf = max(tn, min(t1, t2)), min(tf, max(t1, t2))
    return (tn, tf) if tn < tf else None
