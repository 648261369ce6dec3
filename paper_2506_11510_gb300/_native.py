"""ctypes binding of libtetvol.so (the C ABI declared in include/tetvol.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

TG_OK, TG_EINVAL, TG_ENOMEM, TG_ECUDA, TG_ESTEPLIMIT, TG_EROUNDLIMIT, TG_EGRID = 0, -1, -2, -3, -4, -5, -6


class TgCamera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class TgMedium(C.Structure):
    _fields_ = [("albedo", C.c_float), ("g", C.c_float), ("sigma_scale", C.c_float),
                ("max_bounces", C.c_int32), ("sun_dir", C.c_float * 3),
                ("sun_irradiance", C.c_float), ("env_radiance", C.c_float)]


class TgVolumeDesc(C.Structure):
    _fields_ = [("box_min", C.c_float * 3), ("voxel_size", C.c_float),
                ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class TgJob(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("cam", TgCamera), ("med", TgMedium), ("spp", C.c_int32),
                ("sample_offset", C.c_int32), ("seed", C.c_uint64), ("accum_sum", C.c_void_p),
                ("accum_sumsq", C.c_void_p)]


class TgExt(C.Structure):
    _fields_ = [("flags", C.c_int32), ("emission_scale", C.c_float), ("density", C.c_void_p)]


STATS_FIELDS = ("paths", "tet_steps", "shadow_steps", "collisions", "escapes", "truncated", "step_limit", "misses")

# name -> (restype, argtypes)
_VP, _I32, _I64, _U64, _F = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float
SIGNATURES = {
    "leb_build": (C.c_int, [_VP, C.POINTER(TgVolumeDesc), C.POINTER(TgCamera), _F, _F, _I32, _I32, _VP,
                            C.POINTER(_VP)]),
    "leb_rebuild": (C.c_int, [_VP, _VP, C.POINTER(TgVolumeDesc), C.POINTER(TgCamera), _F, _F, _I32, _I32, _VP,
                              C.POINTER(_VP)]),
    "tg_grid_info": (C.c_int, [_VP, C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I64), C.POINTER(_I32),
                               C.POINTER(_I32)]),
    "tg_grid_export": (C.c_int, [_VP] + [_VP] * 12 + [_VP]),
    "tg_grid_import": (C.c_int, [C.POINTER(TgVolumeDesc), _I32, _I64, _VP, _VP, _VP, _VP, _VP, _I32, _VP,
                                 C.POINTER(_VP)]),
    "tg_grid_free": (None, [_VP]),
    "tet_render": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), _I32, _U64, _I32, _VP, _VP, _VP, _VP]),
    "grid_render": (C.c_int, [_VP, C.POINTER(TgVolumeDesc), C.POINTER(TgCamera), C.POINTER(TgMedium), _I32, _U64,
                              _I32, _VP, _VP, _VP, _VP]),
    "tet_trace_paths": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), _U64, _I64, _VP, _VP, _VP, _VP,
                                  _VP, _VP, _VP, _VP, _I32, _VP, _VP]),
    "grid_trace_paths": (C.c_int, [_VP, C.POINTER(TgVolumeDesc), C.POINTER(TgCamera), C.POINTER(TgMedium), _U64,
                                   _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "tet_optical_depth": (C.c_int, [_VP, _I64, _VP, _VP, _F, _VP, _VP, _VP, _I32, _VP, _VP]),
    "tg_release_build_memory": (C.c_int, []),
    "tet_render_noalloc": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), _I32, _U64, _I32, _VP, _VP,
                                     _VP]),
    "tg_grid_channels": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "tg_grid_export_channels": (C.c_int, [_VP, _VP, _VP, _VP]),
    "tet_render_ext": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), C.POINTER(TgExt), _I32, _U64, _I32,
                                 _VP, _VP, _VP, _VP]),
    "tet_trace_ext_paths": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), C.POINTER(TgExt), _U64, _I64,
                                      _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "tg_batch_create": (C.c_int, [C.POINTER(TgJob), _I32, _I32, _VP, C.POINTER(_VP)]),
    "tg_batch_render": (C.c_int, [_VP, _VP]),
    "tg_batch_info": (C.c_int, [_VP, C.POINTER(_I32), C.POINTER(C.c_double)]),
    "tg_batch_free": (None, [_VP]),
    "tg_random_paths": (C.c_int, [_U64, _I64, _I32, _I32, _I32, _VP, _VP, _VP, _VP]),
    "tet_cache_samples": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), _U64, _I64, _VP, _VP, _VP, _I32,
                                    _VP, _VP, C.c_float, _I32, _VP]),
    "tet_cache_queries": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), _U64, _I64, _VP, _VP, _VP, _I32,
                                    _VP, _VP]),
    "rc_mlp_infer": (C.c_int, [_VP, _VP, _I64, _VP, _VP]),
    "rc_mlp_grad": (C.c_int, [_VP, _VP, _I64, _VP, _VP, _VP]),
    "rc_adam": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _I32, _F, _F, _F, _F, _VP]),
    "tet_render_cached": (C.c_int, [_VP, C.POINTER(TgCamera), C.POINTER(TgMedium), _I32, _U64, _I32, _I32, _VP, _VP,
                                    _VP, _VP, _VP]),
    "rc_timeouts": (C.c_int, [C.POINTER(_I64)]),
    "tg_error_string": (C.c_char_p, [C.c_int]),
}

RC_NUM_PARAMS = 16641

_lib = None


class TetvolError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = lib().tg_error_string(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s (status %d)" % (what, msg, status))


def lib(path: str | None = None):
    """Load libtetvol.so from the package's lib/ folder (built by _build.build())."""
    global _lib
    if _lib is None:
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError("libtetvol.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_2506_11510_gb300._build" % p)
        L = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, what):
    if status != TG_OK:
        raise TetvolError(status, what)
