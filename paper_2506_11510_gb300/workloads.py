"""Seeded synthetic workloads: density volumes, cameras, media and build settings.

The paper renders OpenVDB assets (the Disney *cloud* and an explosion, Sec. 4)
that are not available here; procedural clouds of the same shape stand in for
them.  This module holds none of the method's arithmetic (no bisection, no
walk, no estimator): it only produces inputs, and both the CUDA path and the
CPU oracle take their inputs from it.

Every generator is integer-exact (hashed value noise and Worley noise in fixed
point, int64 tensor ops only), so evaluating it on the CPU or on a CUDA device
gives bit-identical volumes.  The density of voxel (i, j, k) is q / 2**24 with
an integer q in [0, 2**24], stored as float32 (exact).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import torch

MASK32 = 0xFFFFFFFF
ONE16 = 1 << 16
ONE24 = 1 << 24


# ----------------------------------------------------------------------------
# integer hashing and noise (fixed point, 16 fractional bits)
# ----------------------------------------------------------------------------
def _mix32(h: torch.Tensor) -> torch.Tensor:
    # xor-shift-multiply finaliser; every product stays below 2**63
    h = h ^ (h >> 16)
    h = (h * 0x7FEB352D) & MASK32
    h = h ^ (h >> 15)
    h = (h * 0x4C6CA68B) & MASK32
    h = h ^ (h >> 16)
    return h


def _hash3(ix, iy, iz, seed: int) -> torch.Tensor:
    h = (ix * 0x1B873593 + iy * 0x5BD1E995 + iz * 0x68E31DA4 + (seed & 0xFFFF) * 0x3C6EF372) & MASK32
    return _mix32(h)


def _smooth16(f: torch.Tensor) -> torch.Tensor:
    # 3f^2 - 2f^3 with f, result in [0, 2**16]
    return (((f * f) >> 16) * (3 * ONE16 - 2 * f)) >> 16


def value_noise(X, Y, Z, seed: int) -> torch.Tensor:
    """Trilinear value noise at fixed-point lattice coordinates; result in [0, 65535]."""
    ix, iy, iz = X >> 16, Y >> 16, Z >> 16
    wx, wy, wz = _smooth16(X & 0xFFFF), _smooth16(Y & 0xFFFF), _smooth16(Z & 0xFFFF)

    def corner(dx, dy, dz):
        return _hash3(ix + dx, iy + dy, iz + dz, seed) >> 16

    def lerp(a, b, w):
        return a + (((b - a) * w) >> 16)

    x00 = lerp(corner(0, 0, 0), corner(1, 0, 0), wx)
    x10 = lerp(corner(0, 1, 0), corner(1, 1, 0), wx)
    x01 = lerp(corner(0, 0, 1), corner(1, 0, 1), wx)
    x11 = lerp(corner(0, 1, 1), corner(1, 1, 1), wx)
    y0 = lerp(x00, x10, wy)
    y1 = lerp(x01, x11, wy)
    return lerp(y0, y1, wz)


def fbm(X, Y, Z, octaves: int, seed: int) -> torch.Tensor:
    """Fractal sum of value noise, lacunarity 2, gain 1/2; result in [0, 65535]."""
    acc = torch.zeros_like(X)
    for o in range(octaves):
        acc = acc + (value_noise(X << o, Y << o, Z << o, seed + 101 * o) << (octaves - 1 - o))
    return acc // ((1 << octaves) - 1)


def worley_f1sq(X, Y, Z, seed: int) -> torch.Tensor:
    """Squared distance to the nearest of one hashed feature point per lattice cell,
    in units of 2**-16 lattice cells squared, clamped to [0, 65535]."""
    ix, iy, iz = X >> 16, Y >> 16, Z >> 16
    best = torch.full_like(X, 1 << 40)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                cx, cy, cz = ix + dx, iy + dy, iz + dz
                h = _hash3(cx, cy, cz, seed)
                fx = (cx << 16) + (h & 0xFFFF)
                fy = (cy << 16) + ((h >> 16) & 0xFFFF)
                fz = (cz << 16) + (_mix32(h ^ 0x5F3759DF) & 0xFFFF)
                d2 = (fx - X) ** 2 + (fy - Y) ** 2 + (fz - Z) ** 2
                best = torch.minimum(best, d2)
    return torch.clamp(best >> 16, max=ONE16 - 1)


def _coords(n0: int, n1: int, n_ref: int, freq: int, device) -> torch.Tensor:
    """Fixed-point lattice coordinate of voxel centres n0..n1-1 for `freq` lattice
    cells across `n_ref` voxels: ((2i+1)/2) * freq / n_ref * 2**16, exact."""
    i = torch.arange(n0, n1, dtype=torch.int64, device=device)
    assert (freq << 15) % n_ref == 0
    return (2 * i + 1) * ((freq << 15) // n_ref)


# ----------------------------------------------------------------------------
# scene recipes
# ----------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Camera:
    pos: Tuple[float, float, float]
    target: Tuple[float, float, float]
    up: Tuple[float, float, float]
    fov_y_deg: float
    width: int
    height: int


@dataclasses.dataclass(frozen=True)
class Medium:
    albedo: float
    g: float
    sigma_scale: float          # extinction per world unit at density 1
    max_bounces: int
    sun_dir: Tuple[float, float, float]   # direction the light travels
    sun_irradiance: float
    env_radiance: float


@dataclasses.dataclass(frozen=True)
class Scene:
    name: str
    dims: Tuple[int, int, int]            # (nx, ny, nz)
    recipe: str
    volume_seed: int
    box_min: Tuple[float, float, float]
    voxel_size: float
    camera: Camera
    medium: Medium
    spp: int
    render_seed: int
    footprint_px: float                   # <= 0: camera criterion off
    variation_threshold: float            # < 0: density-variation criterion off
    max_depth: int
    density_format: int                   # 0 fp32, 1 bf16, 2 fp16

    @property
    def paths_per_frame(self) -> int:
        return self.camera.width * self.camera.height * self.spp


def _norm(v):
    n = math.sqrt(sum(x * x for x in v))
    return tuple(x / n for x in v)


SCENES = {
    # 32^3 fBm-perturbed sphere, uniform LEB depth 12 (24,576 tets), 64x64 at 4 spp
    "tiny": Scene(
        name="tiny", dims=(32, 32, 32), recipe="sphere", volume_seed=1,
        box_min=(0.0, 0.0, 0.0), voxel_size=1.0 / 32,
        camera=Camera((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 40.0, 64, 64),
        medium=Medium(0.8, 0.3, 10.0, 8, _norm((-1.0, -1.0, 1.0)), math.pi, 0.0),
        spp=4, render_seed=7, footprint_px=0.0, variation_threshold=-1.0,
        max_depth=12, density_format=0),
    # 256^3 fBm cloud (~40% occupancy), adaptive LEB for a 512^2 view at 1-pixel footprint
    "adaptive": Scene(
        name="adaptive", dims=(256, 256, 256), recipe="cloud", volume_seed=2,
        box_min=(0.0, 0.0, 0.0), voxel_size=1.0 / 256,
        camera=Camera((0.5, 0.4, -1.2), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, 512, 512),
        medium=Medium(0.9, 0.5, 64.0, 64, _norm((-1.0, -1.0, 1.0)), 3.0, 0.25),
        spp=32, render_seed=8, footprint_px=1.0, variation_threshold=0.5,
        max_depth=27, density_format=0),
    # the adaptive recipe at 64^3 / 96x80 (ragged against 32-wide tiles), for fast parity runs
    "adaptive_small": Scene(
        name="adaptive_small", dims=(64, 64, 64), recipe="cloud", volume_seed=4,
        box_min=(0.0, 0.0, 0.0), voxel_size=1.0 / 64,
        camera=Camera((0.5, 0.4, -1.2), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, 96, 80),
        medium=Medium(0.9, 0.5, 64.0, 64, _norm((-1.0, -1.0, 1.0)), 3.0, 0.25),
        spp=3, render_seed=18, footprint_px=1.0, variation_threshold=0.5,
        max_depth=21, density_format=0),
    # the production recipe (fBm x Worley, BF16) on a 2x2x1-cube 128x128x64 volume
    "production_small": Scene(
        name="production_small", dims=(128, 128, 64), recipe="wispy", volume_seed=5,
        box_min=(0.0, 0.0, 0.0), voxel_size=1.0 / 64,
        camera=Camera((1.0, 1.0, -2.6), (1.0, 1.0, 0.5), (0.0, 1.0, 0.0), 45.0, 72, 66),
        medium=Medium(0.95, 0.7, 64.0, 128, _norm((-1.0, -1.0, 1.0)), 3.0, 0.25),
        spp=2, render_seed=19, footprint_px=1.0, variation_threshold=0.5,
        max_depth=21, density_format=1),
    # 1024x1024x512 sparse fBm x Worley cloud (~20% occupancy), 1024^2 at 32 spp, BF16 density
    "production": Scene(
        name="production", dims=(1024, 1024, 512), recipe="wispy", volume_seed=3,
        box_min=(0.0, 0.0, 0.0), voxel_size=1.0 / 512,
        camera=Camera((1.0, 1.0, -2.6), (1.0, 1.0, 0.5), (0.0, 1.0, 0.0), 45.0, 1024, 1024),
        medium=Medium(0.95, 0.7, 64.0, 128, _norm((-1.0, -1.0, 1.0)), 3.0, 0.25),
        spp=32, render_seed=9, footprint_px=1.0, variation_threshold=2.0,
        max_depth=30, density_format=1),
}


def scene(name: str, **overrides) -> Scene:
    s = SCENES[name]
    return dataclasses.replace(s, **overrides) if overrides else s


def with_camera(s: Scene, **cam) -> Scene:
    return dataclasses.replace(s, camera=dataclasses.replace(s.camera, **cam))


def with_medium(s: Scene, **med) -> Scene:
    return dataclasses.replace(s, medium=dataclasses.replace(s.medium, **med))


# ----------------------------------------------------------------------------
# volume generation
# ----------------------------------------------------------------------------
def _field_sphere(X, Y, Z, n: int, seed: int):
    # soft ball of radius 0.35 around the centre, perturbed by 4-octave fBm of amplitude 1/2
    i, j, k = X, Y, Z  # voxel indices here
    dx, dy, dz = 2 * i + 1 - n, 2 * j + 1 - n, 2 * k + 1 - n   # units of 1/(2n)
    r2 = dx * dx + dy * dy + dz * dz
    ball = ONE24 - (r2 * ONE24 * 100) // (49 * n * n)         # 1 - r^2/0.35^2
    cx = _coords_from_index(i, n, n, 4)
    cy = _coords_from_index(j, n, n, 4)
    cz = _coords_from_index(k, n, n, 4)
    f = fbm(cx, cy, cz, 4, seed)
    return torch.clamp(ball + (f - 32768) * 256, 0, ONE24)


def _coords_from_index(i, n_ref, _n, freq):
    return (2 * i + 1) * ((freq << 15) // n_ref)


def _cloud_field(i, j, k, dims, seed):
    nx, ny, nz = dims
    n_ref = max(dims)
    X, Y, Z = (_coords_from_index(i, n_ref, nx, 4), _coords_from_index(j, n_ref, ny, 4),
               _coords_from_index(k, n_ref, nz, 4))
    f = fbm(X, Y, Z, 6, seed)
    # soft ellipsoid, semi-axes 0.50, 0.45, 0.50 of the volume extent
    dx, dy, dz = 2 * i + 1 - nx, 2 * j + 1 - ny, 2 * k + 1 - nz
    e = (dx * dx * ONE16) // (nx * nx * 4 * 50 * 50 // 10000) \
        + (dy * dy * ONE16) // (ny * ny * 4 * 45 * 45 // 10000) \
        + (dz * dz * ONE16) // (nz * nz * 4 * 50 * 50 // 10000)
    shell = torch.clamp(ONE16 - e, 0, ONE16)
    return (f * shell) >> 16


def _wispy_field(i, j, k, dims, seed):
    nx, ny, nz = dims
    n_ref = max(dims)
    X, Y, Z = (_coords_from_index(i, n_ref, nx, 8), _coords_from_index(j, n_ref, ny, 8),
               _coords_from_index(k, n_ref, nz, 8))
    f = fbm(X, Y, Z, 6, seed)
    WX, WY, WZ = (_coords_from_index(i, n_ref, nx, 4), _coords_from_index(j, n_ref, ny, 4),
                  _coords_from_index(k, n_ref, nz, 4))
    w = worley_f1sq(WX, WY, WZ, seed + 7)
    blob = torch.clamp(ONE16 - w * 2, 0, ONE16)
    # fade towards the volume faces so the cloud stays inside the box
    def fade(idx, n):
        d = torch.minimum(idx, n - 1 - idx)
        return torch.clamp((d * ONE16) // max(1, n // 16), 0, ONE16)
    edge = (fade(i, nx) * fade(j, ny) >> 16) * fade(k, nz) >> 16
    return (((f * blob) >> 16) * edge) >> 16


def _grid_idx(z0, z1, ny, nx, device):
    k = torch.arange(z0, z1, dtype=torch.int64, device=device).view(-1, 1, 1)
    j = torch.arange(ny, dtype=torch.int64, device=device).view(1, -1, 1)
    i = torch.arange(nx, dtype=torch.int64, device=device).view(1, 1, -1)
    return i, j, k


def _field(recipe, i, j, k, dims, seed):
    if recipe == "cloud":
        return _cloud_field(i, j, k, dims, seed)
    if recipe == "wispy":
        return _wispy_field(i, j, k, dims, seed)
    raise ValueError(recipe)


def _quantile_levels(recipe, dims, seed, device, occupancy):
    """Threshold T (so that about `occupancy` of the voxels exceed it) and a
    top level P, taken from a strided subsample of the field with an exact
    integer histogram."""
    nx, ny, nz = dims
    stride = max(1, min(dims) // 64)
    i = torch.arange(0, nx, stride, dtype=torch.int64, device=device).view(1, 1, -1)
    j = torch.arange(0, ny, stride, dtype=torch.int64, device=device).view(1, -1, 1)
    hist = torch.zeros(ONE16, dtype=torch.int64, device=device)
    for k0 in range(0, nz, stride * 16):
        k = torch.arange(k0, min(nz, k0 + stride * 16), stride, dtype=torch.int64, device=device).view(-1, 1, 1)
        f = _field(recipe, i, j, k, dims, seed).reshape(-1)
        hist += torch.bincount(f, minlength=ONE16)
    cdf = torch.cumsum(hist, 0)
    total = int(cdf[-1])
    t = int(torch.searchsorted(cdf, torch.tensor([int(total * (1.0 - occupancy))], device=device)).item())
    p = int(torch.searchsorted(cdf, torch.tensor([int(total * 0.995)], device=device)).item())
    return t, max(p, t + 1)


_OCC = {"cloud": 0.40, "wispy": 0.20}


def make_volume(s: Scene, device="cpu", z_range: Optional[Tuple[int, int]] = None) -> torch.Tensor:
    """Density volume float32[nz][ny][nx] (or the z-slab `z_range` of it), values q / 2**24."""
    nx, ny, nz = s.dims
    z0, z1 = z_range if z_range is not None else (0, nz)
    out = torch.empty((z1 - z0, ny, nx), dtype=torch.float32, device=device)
    levels = None
    if s.recipe in _OCC:
        levels = _quantile_levels(s.recipe, s.dims, s.volume_seed, device, _OCC[s.recipe])
    slab = max(1, (1 << 23) // (nx * ny))
    for a in range(z0, z1, slab):
        b = min(z1, a + slab)
        i, j, k = _grid_idx(a, b, ny, nx, device)
        if s.recipe == "sphere":
            q = _field_sphere(i, j, k, nx, s.volume_seed)
        else:
            t, p = levels
            f = _field(s.recipe, i, j, k, s.dims, s.volume_seed)
            x = torch.clamp(((f - t) * ONE16) // (p - t), 0, ONE16)
            if s.recipe == "wispy":
                q = (x * x * (3 * ONE16 - 2 * x)) >> 24   # smoothstep: thin soft edges
            else:
                q = x << 8
        out[a - z0:b - z0] = (q.to(torch.float64) / ONE24).to(torch.float32)
    return out


def uniform_volume(dims, value: float, device="cpu") -> torch.Tensor:
    nx, ny, nz = dims
    q = round(value * ONE24)
    return torch.full((nz, ny, nx), q / ONE24, dtype=torch.float32, device=device)


def random_path_ids(s: Scene, n: int, seed: int):
    """Seeded sample of (px, py, sample) triples of the scene's frame."""
    g = torch.Generator().manual_seed(seed)
    px = torch.randint(0, s.camera.width, (n,), generator=g, dtype=torch.int32)
    py = torch.randint(0, s.camera.height, (n,), generator=g, dtype=torch.int32)
    sm = torch.randint(0, s.spp, (n,), generator=g, dtype=torch.int32)
    return px, py, sm


def mlp_init_params(seed: int, num_params: int = 16641, b4: float = 0.0):
    """Seeded initial parameters of the radiance cache's MLP (flat fp32 vector in
    the layout W1[64][128], b1[64], W2[64][64], b2, W3[64][64], b3, w4[64], b4):
    weights uniform in +-sqrt(6 / fan_in) (He et al. 2015), biases zero."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_out, fan_in in ((64, 128), (64, 64), (64, 64)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    parts.append(rng.uniform(-math.sqrt(6.0 / 64), math.sqrt(6.0 / 64), 64) * 0.1)
    parts.append(np.array([b4]))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == num_params
    return p


def mlp_random_records(n: int, seed: int):
    """Seeded cache records [n][8]: x in [0,1]^3 at 0..2, a unit direction at 4..6,
    a target / weight in 3 and a valid flag in 7 (1 for 7 of every 8 rows)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.zeros((n, 8), np.float32)
    r[:, 0:3] = rng.uniform(0, 1, (n, 3))
    d = rng.normal(size=(n, 3))
    r[:, 4:7] = d / np.linalg.norm(d, axis=1, keepdims=True)
    r[:, 3] = rng.uniform(0, 2, n)
    r[:, 7] = (np.arange(n) % 8 != 7).astype(np.float32)
    return r


def make_channels(s: Scene, device="cpu", z_range: Optional[Tuple[int, int]] = None):
    """Extra channel volumes of a scene, float32[nz][ny][nx] each with values
    q / 2**24 (integer-exact like the density): temperature (a hot core fading
    outwards, broken up by fBm: the explosion-style asset), albedo in [0.5, 1]
    and anisotropy a in [0.35, 0.95] (g = 2a - 1 in [-0.3, 0.9]), both from
    low-frequency value noise."""
    nx, ny, nz = s.dims
    z0, z1 = z_range if z_range is not None else (0, nz)
    shape = (z1 - z0, ny, nx)
    temp = torch.empty(shape, dtype=torch.float32, device=device)
    alb = torch.empty_like(temp)
    ani = torch.empty_like(temp)
    n_ref = max(s.dims)
    slab = max(1, (1 << 22) // (nx * ny))
    for a in range(z0, z1, slab):
        b = min(z1, a + slab)
        i, j, k = _grid_idx(a, b, ny, nx, device)
        dx, dy, dz = 2 * i + 1 - nx, 2 * j + 1 - ny, 2 * k + 1 - nz
        r2 = (dx * dx * ONE16) // (nx * nx) + (dy * dy * ONE16) // (ny * ny) + (dz * dz * ONE16) // (nz * nz)
        core = torch.clamp(ONE16 - (r2 * 4) // 3, 0, ONE16)                    # 1 - r^2 / 0.75 (r in box units)
        X, Y, Z = (_coords_from_index(i, n_ref, nx, 4), _coords_from_index(j, n_ref, ny, 4),
                   _coords_from_index(k, n_ref, nz, 4))
        f = fbm(X, Y, Z, 4, s.volume_seed + 31)
        t16 = (core * f) >> 16                                               # [0, 2^16)
        temp[a - z0:b - z0] = ((t16 << 8).to(torch.float64) / ONE24).to(torch.float32)
        L1 = (_coords_from_index(i, n_ref, nx, 2), _coords_from_index(j, n_ref, ny, 2),
              _coords_from_index(k, n_ref, nz, 2))
        va = value_noise(*L1, s.volume_seed + 57)                              # [0, 65535]
        vg = value_noise(*L1, s.volume_seed + 83)
        qa = (ONE24 >> 1) + (va << 7)                                          # 0.5 + va / 2^17 * ... in [0.5, 1)
        qg = (ONE24 * 35) // 100 + ((vg * ((ONE24 * 60) // 100)) >> 16)        # [0.35, 0.95)
        alb[a - z0:b - z0] = (qa.to(torch.float64) / ONE24).to(torch.float32)
        ani[a - z0:b - z0] = (qg.to(torch.float64) / ONE24).to(torch.float32)
    return temp, alb, ani


def batch_scenes(n: int = 64, seed: int = 100, max_dim: int = 384):
    """A heterogeneous batch: n cloud scenes (volume seeds seed..seed+n-1) with
    cubic volumes of 64..max_dim voxels per edge, square views of 128..1024
    pixels and 4..64 spp (each log-uniform), HG g uniform in [-0.3, 0.8],
    albedo in [0.8, 0.95], up to 32 bounces, fp32 densities, adaptive grids
    (1-pixel footprint, threshold 0.5)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = [d for d in (64, 96, 128, 192, 256, 384, 512) if d <= max_dim]
    out = []
    for k in range(n):
        d = dims[int(rng.integers(0, len(dims)))]
        res = int(round(2 ** rng.uniform(7, 10) / 16)) * 16
        spp = int(round(2 ** rng.uniform(2, 6)))
        g = float(rng.uniform(-0.3, 0.8))
        alb = float(rng.uniform(0.8, 0.95))
        depth = 3 * int(math.log2(d)) + 3
        cam = Camera((0.5, 0.4, -1.2), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, res, res)
        med = Medium(alb, g, 64.0, 32, _norm((-1.0, -1.0, 1.0)), 3.0, 0.25)
        out.append(Scene(name="batch%d" % k, dims=(d, d, d), recipe="cloud", volume_seed=seed + k,
                         box_min=(0.0, 0.0, 0.0), voxel_size=1.0 / d, camera=cam, medium=med, spp=spp,
                         render_seed=1000 + k, footprint_px=1.0, variation_threshold=0.5, max_depth=depth,
                         density_format=0))
    return out
