"""Python API over the C ABI, on torch tensors (device memory and streams only).

Every function forwards to one C entry point of libtetvol.so; the computation
runs in the library's CUDA kernels.  Inputs must already be CUDA tensors of the
documented dtype and layout; outputs are allocated as torch tensors.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _native as N


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need(t: torch.Tensor, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t


def camera_struct(cam) -> N.TgCamera:
    c = N.TgCamera()
    c.pos[:] = [float(v) for v in cam.pos]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.fov_y_deg = float(cam.fov_y_deg)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def medium_struct(med) -> N.TgMedium:
    m = N.TgMedium()
    m.albedo = float(med.albedo); m.g = float(med.g); m.sigma_scale = float(med.sigma_scale)
    m.max_bounces = int(med.max_bounces)
    m.sun_dir[:] = [float(v) for v in med.sun_dir]
    m.sun_irradiance = float(med.sun_irradiance); m.env_radiance = float(med.env_radiance)
    return m


def volume_desc(density: torch.Tensor, box_min, voxel_size) -> N.TgVolumeDesc:
    nz, ny, nx = density.shape
    v = N.TgVolumeDesc()
    v.box_min[:] = [float(x) for x in box_min]
    v.voxel_size = float(voxel_size)
    v.nx, v.ny, v.nz = int(nx), int(ny), int(nz)
    return v


@dataclass
class GridInfo:
    num_tets: int
    max_depth: int
    bytes: int
    K: int
    rounds: int


class Grid:
    """A device-resident tetrahedral grid owned by libtetvol (tg_grid)."""

    def __init__(self, handle: C.c_void_p, desc: N.TgVolumeDesc, density_format: int):
        self._h = handle
        self.desc = desc
        self.density_format = density_format
        self.info = self._info()

    def _info(self) -> GridInfo:
        n, md, b, K, r = C.c_int64(), C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32()
        N.check(N.lib().tg_grid_info(self._h, C.byref(n), C.byref(md), C.byref(b), C.byref(K), C.byref(r)),
                "tg_grid_info")
        return GridInfo(n.value, md.value, b.value, K.value, r.value)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            N.lib().tg_grid_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def export(self, fields: Sequence[str] = ("codes", "verts", "tag", "nbr", "nid", "plane", "density",
                                             "majorant", "count", "sum", "qmin", "qmax")) -> dict:
        n = self.info.num_tets
        dev = torch.device("cuda", torch.cuda.current_device())
        spec = {"codes": ((n,), torch.int64), "verts": ((n, 4, 3), torch.int32), "tag": ((n,), torch.int32),
                "nbr": ((n, 4), torch.int32), "nid": ((n, 4), torch.uint8), "plane": ((n, 4), torch.float32),
                "density": ((n,), torch.float32), "majorant": ((n,), torch.float32),
                "count": ((n,), torch.int32), "sum": ((n,), torch.int64), "qmin": ((n,), torch.int32),
                "qmax": ((n,), torch.int32)}
        out = {k: torch.empty(spec[k][0], dtype=spec[k][1], device=dev) for k in fields}
        order = ["codes", "verts", "tag", "nbr", "nid", "plane", "density", "majorant", "count", "sum", "qmin", "qmax"]
        N.check(N.lib().tg_grid_export(self._h, *[_ptr(out.get(k)) for k in order], _stream()), "tg_grid_export")
        return out


    def channels(self, density: torch.Tensor, temperature=None, albedo=None, aniso=None):
        """Per-cell channel means and voxel majorants (tg_grid_channels)."""
        for t, nm in ((density, "density"), (temperature, "temperature"), (albedo, "albedo"), (aniso, "aniso")):
            if t is not None:
                _need(t, torch.float32, nm, (self.desc.nz, self.desc.ny, self.desc.nx))
        N.check(N.lib().tg_grid_channels(self._h, _ptr(density), _ptr(temperature), _ptr(albedo), _ptr(aniso),
                                         _stream()), "tg_grid_channels")

    def export_channels(self):
        n = self.info.num_tets
        dev = torch.device("cuda", torch.cuda.current_device())
        chan = torch.empty((n, 4), dtype=torch.float32, device=dev)
        vmaj = torch.empty(n, dtype=torch.float32, device=dev)
        N.check(N.lib().tg_grid_export_channels(self._h, _ptr(chan), _ptr(vmaj), _stream()),
                "tg_grid_export_channels")
        return chan, vmaj


def ext_struct(flags: int, emission_scale: float = 0.0, density: Optional[torch.Tensor] = None) -> N.TgExt:
    x = N.TgExt()
    x.flags = int(flags)
    x.emission_scale = float(emission_scale)
    if density is not None:
        _need(density, torch.float32, "density")
    x.density = _ptr(density).value if density is not None else None
    return x


def _need_volume(t: torch.Tensor, name: str = "density"):
    """A volume a build reads once: a CUDA tensor, or a pinned (page-locked) host
    tensor that the device reads in place."""
    if isinstance(t, torch.Tensor) and not t.is_cuda and t.is_pinned():
        if t.dtype != torch.float32:
            raise TypeError("%s must be float32, got %s" % (name, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        return t
    return _need(t, torch.float32, name)


def leb_build(density: torch.Tensor, box_min, voxel_size, camera=None, footprint_px: float = 0.0,
              variation_threshold: float = -1.0, max_depth: int = 12, density_format: int = 0) -> Grid:
    """Sec. 2: build the adaptive conforming LEB grid of a density volume float32[nz][ny][nx]
    (a CUDA tensor, or a pinned host tensor that the build reads in place)."""
    _need_volume(density)
    if density.dim() != 3:
        raise ValueError("density must be [nz, ny, nx]")
    desc = volume_desc(density, box_min, voxel_size)
    cam = C.byref(camera_struct(camera)) if camera is not None else None
    h = C.c_void_p()
    N.check(N.lib().leb_build(_ptr(density), C.byref(desc), cam, float(footprint_px), float(variation_threshold),
                              int(max_depth), int(density_format), _stream(), C.byref(h)), "leb_build")
    return Grid(h, desc, density_format)


def leb_rebuild(prev: Grid, density: torch.Tensor, box_min, voxel_size, camera=None, footprint_px: float = 0.0,
                variation_threshold: float = -1.0, max_depth: int = 12, density_format: int = 0) -> Grid:
    """leb_build for a new camera on the volume `prev` was built from, reusing its node statistics."""
    _need_volume(density)
    desc = volume_desc(density, box_min, voxel_size)
    cam = C.byref(camera_struct(camera)) if camera is not None else None
    h = C.c_void_p()
    N.check(N.lib().leb_rebuild(prev.handle, _ptr(density), C.byref(desc), cam, float(footprint_px),
                                float(variation_threshold), int(max_depth), int(density_format), _stream(),
                                C.byref(h)), "leb_rebuild")
    return Grid(h, desc, density_format)


def rebuild_scene_grid(prev: Grid, scene, density: torch.Tensor) -> Grid:
    return leb_rebuild(prev, density, scene.box_min, scene.voxel_size, scene.camera, scene.footprint_px,
                       scene.variation_threshold, scene.max_depth, scene.density_format)


def build_scene_grid(scene, density: torch.Tensor) -> Grid:
    return leb_build(density, scene.box_min, scene.voxel_size, scene.camera, scene.footprint_px,
                     scene.variation_threshold, scene.max_depth, scene.density_format)


def grid_import(box_min, voxel_size, dims, K: int, codes, nbr, nid, plane, density, density_format=0) -> Grid:
    """Wrap grid arrays (device tensors, export layout) into a Grid for rendering."""
    n = codes.shape[0]
    _need(codes, torch.int64, "codes", (n,)); _need(nbr, torch.int32, "nbr", (n, 4))
    _need(nid, torch.uint8, "nid", (n, 4)); _need(plane, torch.float32, "plane", (n, 4))
    _need(density, torch.float32, "density", (n,))
    desc = N.TgVolumeDesc()
    desc.box_min[:] = [float(x) for x in box_min]
    desc.voxel_size = float(voxel_size)
    desc.nx, desc.ny, desc.nz = [int(x) for x in dims]
    h = C.c_void_p()
    N.check(N.lib().tg_grid_import(C.byref(desc), int(K), int(n), _ptr(codes), _ptr(nbr), _ptr(nid), _ptr(plane),
                                   _ptr(density), int(density_format), _stream(), C.byref(h)), "tg_grid_import")
    return Grid(h, desc, density_format)


def release_build_memory():
    """Return the device memory that builds keep for later builds (tg_release_build_memory)."""
    N.check(N.lib().tg_release_build_memory(), "tg_release_build_memory")


def new_stats(device=None) -> torch.Tensor:
    """Zeroed device tg_stats (8 x uint64 counters, as int64)."""
    return torch.zeros(len(N.STATS_FIELDS), dtype=torch.int64, device=device or "cuda")


def stats_dict(stats: torch.Tensor) -> dict:
    return dict(zip(N.STATS_FIELDS, [int(v) for v in stats.cpu()]))


def _accum(camera, accum_sum, accum_sumsq, want_sq):
    dev = torch.device("cuda", torch.cuda.current_device())
    if accum_sum is None:
        accum_sum = torch.zeros((camera.height, camera.width), dtype=torch.float32, device=dev)
    if accum_sumsq is None and want_sq:
        accum_sumsq = torch.zeros((camera.height, camera.width), dtype=torch.float32, device=dev)
    _need(accum_sum, torch.float32, "accum_sum", (camera.height, camera.width))
    if accum_sumsq is not None:
        _need(accum_sumsq, torch.float32, "accum_sumsq", (camera.height, camera.width))
    return accum_sum, accum_sumsq


def tet_render(grid: Grid, camera, medium, spp: int, seed: int, sample_offset: int = 0, accum_sum=None,
               accum_sumsq=None, stats: Optional[torch.Tensor] = None, want_sq: bool = True):
    """Sec. 3, Algorithm 1: accumulate spp paths per pixel into (accum_sum, accum_sumsq)."""
    s, s2 = _accum(camera, accum_sum, accum_sumsq, want_sq)
    if stats is not None:
        _need(stats, torch.int64, "stats", (len(N.STATS_FIELDS),))
    N.check(N.lib().tet_render(grid.handle, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                               int(spp), C.c_uint64(seed), int(sample_offset), _ptr(s), _ptr(s2), _ptr(stats),
                               _stream()), "tet_render")
    return s, s2


def grid_render(density: torch.Tensor, box_min, voxel_size, camera, medium, spp: int, seed: int,
                sample_offset: int = 0, accum_sum=None, accum_sumsq=None, stats=None, want_sq: bool = True):
    """The regular-grid (3D DDA) comparator with the same estimator."""
    _need(density, torch.float32, "density")
    desc = volume_desc(density, box_min, voxel_size)
    s, s2 = _accum(camera, accum_sum, accum_sumsq, want_sq)
    if stats is not None:
        _need(stats, torch.int64, "stats", (len(N.STATS_FIELDS),))
    N.check(N.lib().grid_render(_ptr(density), C.byref(desc), C.byref(camera_struct(camera)),
                                C.byref(medium_struct(medium)), int(spp), C.c_uint64(seed), int(sample_offset),
                                _ptr(s), _ptr(s2), _ptr(stats), _stream()), "grid_render")
    return s, s2


def _paths(px, py, sample):
    dev = torch.device("cuda", torch.cuda.current_device())
    px = torch.as_tensor(px, dtype=torch.int32).to(dev).contiguous()
    py = torch.as_tensor(py, dtype=torch.int32).to(dev).contiguous()
    sm = torch.as_tensor(sample, dtype=torch.int32).to(dev).contiguous()
    return px, py, sm, dev


def tet_trace_paths(grid: Grid, camera, medium, seed: int, px, py, sample, seq_cap: int = 0) -> dict:
    px, py, sm, dev = _paths(px, py, sample)
    n = px.numel()
    out = dict(L=torch.empty(n, dtype=torch.float32, device=dev), flags=torch.empty(n, dtype=torch.int32, device=dev),
               collisions=torch.empty(n, dtype=torch.int32, device=dev),
               steps=torch.empty(n, dtype=torch.int64, device=dev))
    seq = seq_len = None
    if seq_cap:
        seq = torch.full((n, seq_cap), -2, dtype=torch.int32, device=dev)
        seq_len = torch.zeros(n, dtype=torch.int32, device=dev)
        out.update(seq=seq, seq_len=seq_len)
    N.check(N.lib().tet_trace_paths(grid.handle, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                    C.c_uint64(seed), n, _ptr(px), _ptr(py), _ptr(sm), _ptr(out["L"]),
                                    _ptr(out["flags"]), _ptr(out["collisions"]), _ptr(out["steps"]), _ptr(seq),
                                    int(seq_cap), _ptr(seq_len), _stream()), "tet_trace_paths")
    return out


def grid_trace_paths(density, box_min, voxel_size, camera, medium, seed: int, px, py, sample) -> dict:
    _need(density, torch.float32, "density")
    desc = volume_desc(density, box_min, voxel_size)
    px, py, sm, dev = _paths(px, py, sample)
    n = px.numel()
    out = dict(L=torch.empty(n, dtype=torch.float32, device=dev), flags=torch.empty(n, dtype=torch.int32, device=dev),
               collisions=torch.empty(n, dtype=torch.int32, device=dev),
               steps=torch.empty(n, dtype=torch.int64, device=dev))
    N.check(N.lib().grid_trace_paths(_ptr(density), C.byref(desc), C.byref(camera_struct(camera)),
                                     C.byref(medium_struct(medium)), C.c_uint64(seed), n, _ptr(px), _ptr(py),
                                     _ptr(sm), _ptr(out["L"]), _ptr(out["flags"]), _ptr(out["collisions"]),
                                     _ptr(out["steps"]), _stream()), "grid_trace_paths")
    return out


def tet_optical_depth(grid: Grid, origins: torch.Tensor, dirs: torch.Tensor, sigma: float, seq_cap: int = 0) -> dict:
    n = origins.shape[0]
    _need(origins, torch.float32, "origins", (n, 3)); _need(dirs, torch.float32, "dirs", (n, 3))
    dev = origins.device
    out = dict(tau=torch.empty(n, dtype=torch.float32, device=dev), steps=torch.empty(n, dtype=torch.int64, device=dev))
    seq = seq_len = None
    if seq_cap:
        seq = torch.full((n, seq_cap), -2, dtype=torch.int32, device=dev)
        seq_len = torch.zeros(n, dtype=torch.int32, device=dev)
        out.update(seq=seq, seq_len=seq_len)
    N.check(N.lib().tet_optical_depth(grid.handle, n, _ptr(origins), _ptr(dirs), float(sigma), _ptr(out["tau"]),
                                      _ptr(out["steps"]), _ptr(seq), int(seq_cap), _ptr(seq_len), _stream()),
            "tet_optical_depth")
    return out


def tet_render_ext(grid: Grid, camera, medium, flags: int, spp: int, seed: int, emission_scale: float = 0.0,
                   density: Optional[torch.Tensor] = None, sample_offset: int = 0, accum_sum=None, accum_sumsq=None,
                   stats: Optional[torch.Tensor] = None, want_sq: bool = True):
    """tet_render with the extended medium: per-cell emission / albedo / g, or the voxel
    medium `density` tracked against the cells' voxel majorants (flags TG_EXT_*)."""
    s, s2 = _accum(camera, accum_sum, accum_sumsq, want_sq)
    if stats is not None:
        _need(stats, torch.int64, "stats", (len(N.STATS_FIELDS),))
    x = ext_struct(flags, emission_scale, density)
    N.check(N.lib().tet_render_ext(grid.handle, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                   C.byref(x), int(spp), C.c_uint64(seed), int(sample_offset), _ptr(s), _ptr(s2),
                                   _ptr(stats), _stream()), "tet_render_ext")
    return s, s2


def tet_trace_ext_paths(grid: Grid, camera, medium, flags: int, seed: int, px, py, sample, emission_scale=0.0,
                        density: Optional[torch.Tensor] = None) -> dict:
    px, py, sm, dev = _paths(px, py, sample)
    n = px.numel()
    out = dict(L=torch.empty(n, dtype=torch.float32, device=dev), flags=torch.empty(n, dtype=torch.int32, device=dev),
               collisions=torch.empty(n, dtype=torch.int32, device=dev),
               steps=torch.empty(n, dtype=torch.int64, device=dev))
    x = ext_struct(flags, emission_scale, density)
    N.check(N.lib().tet_trace_ext_paths(grid.handle, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                        C.byref(x), C.c_uint64(seed), n, _ptr(px), _ptr(py), _ptr(sm),
                                        _ptr(out["L"]), _ptr(out["flags"]), _ptr(out["collisions"]),
                                        _ptr(out["steps"]), _stream()), "tet_trace_ext_paths")
    return out


class Batch:
    """Many jobs (grid, camera, medium, spp, seed, image) rendered by one persistent
    launch captured in a CUDA graph (tg_batch_*); render() adds one frame of every job."""

    def __init__(self, jobs, autotune: bool = True):
        """jobs: sequence of (grid, camera, medium, spp, seed, accum_sum, accum_sumsq or None[, sample_offset])."""
        arr = (N.TgJob * len(jobs))()
        self._keep = []
        for k, j in enumerate(jobs):
            grid, cam, med, spp, seed, s, s2 = j[:7]
            off = j[7] if len(j) > 7 else 0
            _need(s, torch.float32, "accum_sum", (cam.height, cam.width))
            if s2 is not None:
                _need(s2, torch.float32, "accum_sumsq", (cam.height, cam.width))
            arr[k].grid = grid.handle.value
            arr[k].cam = camera_struct(cam)
            arr[k].med = medium_struct(med)
            arr[k].spp = int(spp)
            arr[k].sample_offset = int(off)
            arr[k].seed = int(seed)
            arr[k].accum_sum = s.data_ptr()
            arr[k].accum_sumsq = s2.data_ptr() if s2 is not None else None
            self._keep.append((grid, s, s2))
        self._h = C.c_void_p()
        self.n = len(jobs)
        N.check(N.lib().tg_batch_create(arr, self.n, 1 if autotune else 0, _stream(), C.byref(self._h)),
                "tg_batch_create")

    def render(self):
        N.check(N.lib().tg_batch_render(self._h, _stream()), "tg_batch_render")

    def info(self):
        knobs = (C.c_int32 * 4)()
        ms = (C.c_double * self.n)()
        N.check(N.lib().tg_batch_info(self._h, knobs, ms), "tg_batch_info")
        return dict(zip(("regen_min", "ev_min", "blocks_per_sm", "order"), list(knobs))), list(ms)

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().tg_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
