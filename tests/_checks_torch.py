"""Structural grid checks that hold at any size, on torch tensors (run on the
GPU for the 50 M-cell production grid).  Same properties as tests/_checks.py:
exact volumes that tile the domain, longest-edge refinement, symmetric
neighbour links that join identical faces (hence every interior face is shared
by exactly two cells), boundary faces on the domain boundary, orientation ids
and plane offsets that match the geometry."""
import torch

P9 = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, -1, 0], [0, 1, 1], [0, 1, -1], [1, 0, 1], [1, 0, -1]]
FACE = [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]


def _sorted_face(v, f):
    """(n, 3, 3) vertices of face f, sorted lexicographically (packed key order)."""
    fv = v[:, FACE[f], :]
    key = (fv[:, :, 0] << 42) | (fv[:, :, 1] << 21) | fv[:, :, 2]
    order = torch.argsort(key, dim=1)
    return torch.gather(fv, 1, order[:, :, None].expand(-1, -1, 3))


def check_grid_torch(ex, K, cubes, chunk=1 << 22):
    codes, verts, tag, nbr, nid, plane = (ex["codes"], ex["verts"], ex["tag"], ex["nbr"], ex["nid"], ex["plane"])
    N = codes.shape[0]
    dev = codes.device
    # codes strictly increasing as unsigned 64-bit numbers (flip the sign bit for a signed compare)
    sc = codes ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=dev)
    assert bool((sc[1:] > sc[:-1]).all()), "codes not strictly increasing"
    depth = codes & 63
    total6 = 0
    P = torch.tensor(P9, dtype=torch.int64, device=dev)
    lim = torch.tensor(cubes, dtype=torch.int64, device=dev) << K
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        v = verts[a:b].to(torch.int64)
        e1, e2, e3 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]
        six = torch.abs((e1 * torch.cross(e2, e3, dim=1)).sum(1))
        expect = (torch.ones_like(six) << (3 * K)) >> depth[a:b]
        assert bool((six == expect).all()), "cell volume != root volume / 2^depth"
        total6 += int(six.sum())
        # refinement edge x0 - x_tag is the unique longest edge
        L = {}
        for i in range(4):
            for j in range(i + 1, 4):
                d = v[:, i] - v[:, j]
                L[(i, j)] = (d * d).sum(1)
        t = tag[a:b].to(torch.int64)
        ref = torch.where(t == 1, L[(0, 1)], torch.where(t == 2, L[(0, 2)], L[(0, 3)]))
        om = torch.zeros_like(ref)
        for (i, j), l in L.items():
            is_ref = (i == 0) & (t == j)
            om = torch.maximum(om, torch.where(is_ref, torch.zeros_like(l), l))
        assert bool((ref > om).all()), "refinement edge is not the unique longest edge"
        # faces: normals, planes, links
        for f in range(4):
            fv = v[:, FACE[f], :]
            n = torch.cross(fv[:, 1] - fv[:, 0], fv[:, 2] - fv[:, 0], dim=1)
            out = ((n * (v[:, f] - fv[:, 0])).sum(1) > 0)
            n = torch.where(out[:, None], -n, n)
            idf = nid[a:b, f].to(torch.int64)
            p = idf % 9
            sgn = torch.where(idf >= 9, -1, 1)
            want = P[p] * sgn[:, None]
            scale = n.abs().max(1).values
            assert bool((scale > 0).all())
            assert bool((n == want * scale[:, None]).all()), "orientation id does not match the face"
            c = (P[p] * fv[:, 0]).sum(1).to(torch.float64) * 2.0 ** (-K)
            assert bool((c.to(torch.float32) == plane[a:b, f]).all()), "plane offset differs"
            j = nbr[a:b, f].to(torch.int64)
            bnd = j < 0
            # boundary faces lie on the domain boundary
            if bool(bnd.any()):
                fb = fv[bnd]
                onb = torch.zeros(fb.shape[0], dtype=torch.bool, device=dev)
                for ax in range(3):
                    xa = fb[:, :, ax]
                    onb |= (xa == 0).all(1) | (xa == lim[ax]).all(1)
                assert bool(onb.all()), "a boundary link on an interior face"
            ii = torch.arange(a, b, device=dev)[~bnd]
            jj = j[~bnd]
            assert bool((jj < N).all())
            back = nbr[jj].to(torch.int64) == ii[:, None]
            assert bool((back.sum(1) == 1).all()), "neighbour links are not symmetric"
            g = torch.argmax(back.to(torch.int64), dim=1)
            mine = _sorted_face(v[~bnd], f)
            vj = verts[jj].to(torch.int64)
            theirs = torch.empty_like(mine)
            for gg in range(4):
                m = g == gg
                if bool(m.any()):
                    theirs[m] = _sorted_face(vj[m], gg)
            assert bool((mine == theirs).all()), "linked cells do not share the face"
    assert total6 == 6 * int(cubes[0] * cubes[1] * cubes[2]) * (1 << (3 * K)), "cells do not tile the domain"
