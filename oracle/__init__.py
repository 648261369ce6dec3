"""Python binding of the CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg; the product path never imports it.  It takes
numpy arrays and calls the plain C++ oracle through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "lib", "liboracle.so")
SRC = os.path.join(HERE, "oracle.cpp")


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/lib/liboracle.so (plain g++, OpenMP)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


class _Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class _Medium(C.Structure):
    _fields_ = [("albedo", C.c_float), ("g", C.c_float), ("sigma_scale", C.c_float),
                ("max_bounces", C.c_int32), ("sun_dir", C.c_float * 3),
                ("sun_irradiance", C.c_float), ("env_radiance", C.c_float)]


class _Ext(C.Structure):
    _fields_ = [("flags", C.c_int32), ("emission_scale", C.c_float), ("density", C.c_void_p)]


def camera_struct(cam) -> _Camera:
    c = _Camera()
    c.pos[:] = list(cam.pos); c.target[:] = list(cam.target); c.up[:] = list(cam.up)
    c.fov_y_deg = cam.fov_y_deg; c.width = cam.width; c.height = cam.height
    return c


def medium_struct(med) -> _Medium:
    m = _Medium()
    m.albedo = med.albedo; m.g = med.g; m.sigma_scale = med.sigma_scale
    m.max_bounces = med.max_bounces; m.sun_dir[:] = list(med.sun_dir)
    m.sun_irradiance = med.sun_irradiance; m.env_radiance = med.env_radiance
    return m


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
        _lib.orc_build.restype = C.c_int
        _lib.orc_uniform.restype = C.c_double
        _lib.orc_hg_pdf.restype = C.c_double
        _lib.orc_grid_free.restype = None
        _lib.orc_render_ext_paths.argtypes = None
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f3(v):
    return (C.c_float * 3)(*[float(x) for x in v])


class OracleError(RuntimeError):
    pass


def _check(st):
    if st != 0:
        raise OracleError("oracle status %d" % st)


@dataclass
class GridArrays:
    codes: np.ndarray
    verts: np.ndarray
    tag: np.ndarray
    nbr: np.ndarray
    nid: np.ndarray
    plane: np.ndarray
    density: np.ndarray
    majorant: np.ndarray
    count: np.ndarray
    sum: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    K: int
    max_depth: int
    rounds: int
    cubes: tuple
    voxels_per_cube: int


class Grid:
    """An oracle-built grid (host memory, owned by the oracle library)."""

    def __init__(self, volume: np.ndarray, box_min, voxel_size, camera=None, footprint_px=0.0,
                 theta=-1.0, max_depth=12, density_format=0, max_rounds=0, nthreads=0):
        L = lib()
        vol = np.ascontiguousarray(volume, dtype=np.float32)
        nz, ny, nx = vol.shape
        self._h = C.c_void_p()
        cam = C.byref(camera_struct(camera)) if camera is not None else None
        st = L.orc_build(_p(vol), nx, ny, nz, _f3(box_min), C.c_float(voxel_size), cam,
                         C.c_float(footprint_px), C.c_float(theta), max_depth, density_format,
                         max_rounds, nthreads, C.byref(self._h))
        _check(st)

    @classmethod
    def for_scene(cls, s, volume: np.ndarray, nthreads=0, **kw):
        args = dict(box_min=s.box_min, voxel_size=s.voxel_size, camera=s.camera,
                    footprint_px=s.footprint_px, theta=s.variation_threshold,
                    max_depth=s.max_depth, density_format=s.density_format, nthreads=nthreads)
        args.update(kw)
        return cls(volume, **args)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().orc_grid_free(self._h)
            self._h = None

    def info(self):
        n = C.c_int64(); md = C.c_int32(); K = C.c_int32(); r = C.c_int32()
        cubes = (C.c_int32 * 3)(); vpc = C.c_int32()
        _check(lib().orc_grid_info(self._h, C.byref(n), C.byref(md), C.byref(K), C.byref(r), cubes, C.byref(vpc)))
        return dict(num_tets=n.value, max_depth=md.value, K=K.value, rounds=r.value,
                    cubes=tuple(cubes), voxels_per_cube=vpc.value)

    def export(self) -> GridArrays:
        inf = self.info()
        N = inf["num_tets"]
        a = GridArrays(
            codes=np.empty(N, np.uint64), verts=np.empty((N, 4, 3), np.int32), tag=np.empty(N, np.int32),
            nbr=np.empty((N, 4), np.int32), nid=np.empty((N, 4), np.uint8), plane=np.empty((N, 4), np.float32),
            density=np.empty(N, np.float32), majorant=np.empty(N, np.float32), count=np.empty(N, np.uint32),
            sum=np.empty(N, np.uint64), qmin=np.empty(N, np.uint32), qmax=np.empty(N, np.uint32),
            K=inf["K"], max_depth=inf["max_depth"], rounds=inf["rounds"], cubes=inf["cubes"],
            voxels_per_cube=inf["voxels_per_cube"])
        _check(lib().orc_grid_export(self._h, _p(a.codes), _p(a.verts), _p(a.tag), _p(a.nbr), _p(a.nid),
                                     _p(a.plane), _p(a.density), _p(a.majorant), _p(a.count), _p(a.sum),
                                     _p(a.qmin), _p(a.qmax)))
        return a

    def render_paths(self, camera, medium, seed, px, py, sample, seq_cap=0, nthreads=0):
        px = np.ascontiguousarray(px, np.int32); py = np.ascontiguousarray(py, np.int32)
        sm = np.ascontiguousarray(sample, np.int32)
        n = len(px)
        L = np.empty(n, np.float64); flags = np.empty(n, np.int32); coll = np.empty(n, np.int32)
        steps = np.empty(n, np.int64)
        seq = np.full((n, seq_cap), -2, np.int32) if seq_cap else None
        seq_len = np.zeros(n, np.int32) if seq_cap else None
        _check(lib().orc_render_paths(self._h, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                      C.c_uint64(seed), C.c_int64(n), _p(px), _p(py), _p(sm), _p(L), _p(flags),
                                      _p(coll), _p(steps), _p(seq), seq_cap, _p(seq_len), nthreads))
        out = dict(L=L, flags=flags, collisions=coll, steps=steps)
        if seq_cap:
            out.update(seq=seq, seq_len=seq_len)
        return out

    def cache_paths(self, camera, medium, seed, px, py, sample, cache_depth=0, max_vertices=0, nthreads=0,
                    survive=0.0, roulette_from=0):
        """The radiance cache's uses of the tracer: cached-path records (cache_depth > 0,
        query [n][8]) and training samples from path vertices (vertices [n][max_vertices][8]);
        survive in (0, 1): Russian roulette after the last training vertex, at collisions
        roulette_from and later (0-based)."""
        px = np.ascontiguousarray(px, np.int32); py = np.ascontiguousarray(py, np.int32)
        sm = np.ascontiguousarray(sample, np.int32)
        n = len(px)
        q = np.zeros((n, 8), np.float64) if cache_depth > 0 else None
        v = np.zeros((n, max_vertices, 8), np.float64) if max_vertices > 0 else None
        L = np.empty(n, np.float64); flags = np.empty(n, np.int32)
        _check(lib().orc_cache_paths(self._h, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                     C.c_uint64(seed), C.c_int64(n), _p(px), _p(py), _p(sm), cache_depth, _p(q),
                                     max_vertices, _p(v), _p(L), _p(flags), C.c_float(survive),
                                     int(roulette_from), nthreads))
        return dict(query=q, vertices=v, L=L, flags=flags)

    def channels(self, density, temperature=None, albedo=None, aniso=None, nthreads=0):
        """Per-tet channel means and voxel majorants (orc_grid_channels)."""
        c = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
        d, t, a_, g = c(density), c(temperature), c(albedo), c(aniso)
        self._keep = (d, t, a_, g)
        _check(lib().orc_grid_channels(self._h, _p(d), _p(t), _p(a_), _p(g), nthreads))

    def export_channels(self):
        n = self.info()["num_tets"]
        chan = np.empty((n, 3), np.float32); vmaj = np.empty(n, np.float32)
        _check(lib().orc_grid_export_channels(self._h, _p(chan), _p(vmaj)))
        return chan, vmaj

    def render_ext_paths(self, camera, medium, seed, px, py, sample, flags, emission_scale=0.0, density=None,
                         nthreads=0):
        """The extended estimator (emission, per-tet albedo / g, voxel medium with delta tracking)."""
        px = np.ascontiguousarray(px, np.int32); py = np.ascontiguousarray(py, np.int32)
        sm = np.ascontiguousarray(sample, np.int32)
        n = len(px)
        vox = np.ascontiguousarray(density, np.float32) if density is not None else None
        ext = _Ext()
        ext.flags = flags; ext.emission_scale = emission_scale
        ext.density = vox.ctypes.data_as(C.c_void_p) if vox is not None else None
        L = np.empty(n, np.float64); fl = np.empty(n, np.int32); coll = np.empty(n, np.int32)
        steps = np.empty(n, np.int64)
        _check(lib().orc_render_ext_paths(self._h, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                          C.byref(ext), C.c_uint64(seed), C.c_int64(n), _p(px), _p(py), _p(sm),
                                          _p(L), _p(fl), _p(coll), _p(steps), nthreads))
        return dict(L=L, flags=fl, collisions=coll, steps=steps)

    def render(self, camera, medium, spp, seed, sample_offset=0, nthreads=0):
        s = np.zeros((camera.height, camera.width), np.float64)
        s2 = np.zeros_like(s)
        steps = C.c_int64()
        _check(lib().orc_render(self._h, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)), spp,
                                C.c_uint64(seed), sample_offset, _p(s), _p(s2), C.byref(steps), nthreads))
        return s, s2, steps.value

    def optical_depth(self, origins, dirs, sigma, seq_cap=0):
        o = np.ascontiguousarray(origins, np.float64); d = np.ascontiguousarray(dirs, np.float64)
        n = len(o)
        tau = np.empty(n, np.float64); steps = np.empty(n, np.int64); mft = np.empty(n, np.int32)
        flags = np.empty(n, np.int32)
        seq = np.full((n, seq_cap), -2, np.int32) if seq_cap else None
        seq_len = np.zeros(n, np.int32) if seq_cap else None
        _check(lib().orc_optical_depth(self._h, C.c_int64(n), _p(o), _p(d), C.c_double(sigma), _p(tau),
                                       _p(steps), _p(mft), _p(flags), _p(seq), seq_cap, _p(seq_len)))
        out = dict(tau=tau, steps=steps, max_faces_tested=mft, flags=flags)
        if seq_cap:
            out.update(seq=seq, seq_len=seq_len)
        return out

    def locate(self, points):
        p = np.ascontiguousarray(points, np.float64)
        out = np.empty(len(p), np.int32)
        _check(lib().orc_locate(self._h, C.c_int64(len(p)), _p(p), _p(out)))
        return out


def dda_render_paths(volume, box_min, voxel_size, camera, medium, seed, px, py, sample, nthreads=0):
    vol = np.ascontiguousarray(volume, np.float32)
    nz, ny, nx = vol.shape
    px = np.ascontiguousarray(px, np.int32); py = np.ascontiguousarray(py, np.int32)
    sm = np.ascontiguousarray(sample, np.int32)
    n = len(px)
    L = np.empty(n, np.float64); flags = np.empty(n, np.int32); coll = np.empty(n, np.int32)
    steps = np.empty(n, np.int64)
    _check(lib().orc_dda_paths(_p(vol), nx, ny, nz, _f3(box_min), C.c_float(voxel_size),
                               C.byref(camera_struct(camera)), C.byref(medium_struct(medium)), C.c_uint64(seed),
                               C.c_int64(n), _p(px), _p(py), _p(sm), _p(L), _p(flags), _p(coll), _p(steps),
                               nthreads))
    return dict(L=L, flags=flags, collisions=coll, steps=steps)


def dda_render(volume, box_min, voxel_size, camera, medium, spp, seed, sample_offset=0, nthreads=0):
    vol = np.ascontiguousarray(volume, np.float32)
    nz, ny, nx = vol.shape
    s = np.zeros((camera.height, camera.width), np.float64)
    s2 = np.zeros_like(s)
    steps = C.c_int64()
    _check(lib().orc_dda_render(_p(vol), nx, ny, nz, _f3(box_min), C.c_float(voxel_size),
                                C.byref(camera_struct(camera)), C.byref(medium_struct(medium)), spp,
                                C.c_uint64(seed), sample_offset, _p(s), _p(s2), C.byref(steps), nthreads))
    return s, s2, steps.value


def path_profile(volume, box_min, voxel_size, camera, footprint_px, theta, max_depth, density_format,
                 points, nthreads=0):
    vol = np.ascontiguousarray(volume, np.float32)
    nz, ny, nx = vol.shape
    p = np.ascontiguousarray(points, np.float64)
    n = len(p)
    lv = max_depth + 1
    out = dict(codes=np.empty((n, lv), np.uint64), count=np.empty((n, lv), np.uint32),
               sum=np.empty((n, lv), np.uint64), qmin=np.empty((n, lv), np.uint32),
               qmax=np.empty((n, lv), np.uint32), density=np.empty((n, lv), np.float32),
               split=np.empty((n, lv), np.uint8))
    cam = C.byref(camera_struct(camera)) if camera is not None else None
    _check(lib().orc_path_profile(_p(vol), nx, ny, nz, _f3(box_min), C.c_float(voxel_size), cam,
                                  C.c_float(footprint_px), C.c_float(theta), max_depth, density_format,
                                  C.c_int64(n), _p(p), _p(out["codes"]), _p(out["count"]), _p(out["sum"]),
                                  _p(out["qmin"]), _p(out["qmax"]), _p(out["density"]), _p(out["split"]),
                                  nthreads))
    return out


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr); k = (C.c_uint32 * 2)(*key); o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(o)


def uniform(seed, pixel, sample, slot):
    return lib().orc_uniform(C.c_uint64(seed), C.c_uint32(pixel), C.c_uint32(sample), C.c_uint32(slot))


def hg_sample(g, u1, u2, d):
    di = (C.c_double * 3)(*d); do = (C.c_double * 3)()
    lib().orc_hg_sample(C.c_double(g), C.c_double(u1), C.c_double(u2), di, do)
    return tuple(do)


def hg_pdf(g, cos_theta):
    return lib().orc_hg_pdf(C.c_double(g), C.c_double(cos_theta))


def code_depth(codes):
    return (np.asarray(codes, np.uint64) & np.uint64(63)).astype(np.int64)
