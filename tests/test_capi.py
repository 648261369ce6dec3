"""The C-ABI library loads on any machine (no GPU needed) and exports every
entry point that include/tetvol.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tetvol.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("leb_build", "tet_render", "grid_render", "tg_grid_export", "tg_grid_info", "tg_grid_free",
              "tg_error_string", "tet_trace_paths", "tet_optical_depth", "tg_grid_import", "grid_trace_paths"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2506_11510_gb300 import _build, _native
    _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for n in declared_functions():
        assert hasattr(lib, n), "libtetvol.so does not export %s" % n
    assert set(_native.SIGNATURES) == set(declared_functions())


def test_error_strings_without_a_gpu():
    from paper_2506_11510_gb300 import _native as N
    L = N.lib()
    assert L.tg_error_string(0) == b"ok"
    assert L.tg_error_string(-6) == b"grid is not conforming"
    assert L.tg_error_string(12345) == b"unknown status"


def test_argument_checks_need_no_gpu():
    """Invalid arguments are rejected before any CUDA call."""
    import ctypes as C
    from paper_2506_11510_gb300 import _native as N
    L = N.lib()
    out = C.c_void_p()
    desc = N.TgVolumeDesc()
    desc.nx = desc.ny = desc.nz = 8
    desc.voxel_size = 0.125
    assert L.leb_build(None, C.byref(desc), None, 0.0, -1.0, 4, 0, None, C.byref(out)) == N.TG_EINVAL
    assert L.leb_build(C.c_void_p(16), C.byref(desc), None, 0.0, -1.0, 51, 0, None, C.byref(out)) == N.TG_EINVAL
    assert L.leb_build(C.c_void_p(16), C.byref(desc), None, 0.0, -1.0, 4, 3, None, C.byref(out)) == N.TG_EINVAL
    assert L.tet_render(None, None, None, 1, 0, 0, None, None, None, None) == N.TG_EINVAL
    assert L.tg_grid_info(None, None, None, None, None, None) == N.TG_EINVAL


def test_radiance_cache_argument_checks_need_no_gpu():
    import ctypes as C
    from paper_2506_11510_gb300 import _native as N
    L = N.lib()
    cam, med = N.TgCamera(), N.TgMedium()
    cam.width = cam.height = 8
    cam.fov_y_deg = 40.0
    med.max_bounces = 4
    fake = C.c_void_p(256)
    assert L.rc_adam(fake, fake, fake, fake, fake, 0, 1e-3, 0.9, 0.99, 1e-8, None) == N.TG_EINVAL    # step < 1
    assert L.rc_adam(fake, fake, fake, fake, fake, 1, 0.0, 0.9, 0.99, 1e-8, None) == N.TG_EINVAL     # lr
    assert L.rc_adam(fake, fake, fake, fake, fake, 1, 1e-3, 1.0, 0.99, 1e-8, None) == N.TG_EINVAL    # beta1
    assert L.rc_mlp_infer(None, fake, 4, fake, None) == N.TG_EINVAL
    assert L.rc_mlp_infer(fake, None, 4, fake, None) == N.TG_EINVAL
    assert L.rc_mlp_grad(fake, fake, -1, fake, fake, None) == N.TG_EINVAL
    assert L.rc_mlp_grad(fake, fake, 0, None, fake, None) == N.TG_EINVAL
    assert L.tet_render_cached(None, C.byref(cam), C.byref(med), 1, 0, 0, 1, fake, fake, None, None,
                               None) == N.TG_EINVAL
    assert L.tet_render_cached(fake, C.byref(cam), C.byref(med), 1, 0, 0, 0, fake, fake, None, None,
                               None) == N.TG_EINVAL                                               # depth 0
    assert L.tet_cache_queries(fake, C.byref(cam), C.byref(med), 0, 4, fake, fake, fake, 0, fake,
                               None) == N.TG_EINVAL
    assert L.tet_cache_samples(fake, C.byref(cam), C.byref(med), 0, 4, fake, fake, fake, 65, fake, None, 0.0, 0,
                               None) == N.TG_EINVAL                                               # > 64 vertices
    for q in (-0.5, 1.5, float("nan")):                                                           # survival
        assert L.tet_cache_samples(fake, C.byref(cam), C.byref(med), 0, 4, fake, fake, fake, 4, fake, None, q, 0,
                                   None) == N.TG_EINVAL
    assert L.tet_cache_samples(fake, C.byref(cam), C.byref(med), 0, 4, fake, fake, fake, 4, fake, None, 0.5, -1,
                               None) == N.TG_EINVAL                                               # roulette start
    assert L.tg_random_paths(0, 4, 0, 8, 0, fake, fake, fake, None) == N.TG_EINVAL
    assert L.tg_random_paths(0, 4, 8, 8, (1 << 31) - 2, fake, fake, fake, None) == N.TG_EINVAL
    assert L.rc_mlp_grad(fake, fake, 0, fake, fake, None) == N.TG_OK                              # nothing to do
    assert N.RC_NUM_PARAMS == 64 * 128 + 64 + 2 * (64 * 64 + 64) + 64 + 1


def test_rebuild_batch_and_channel_argument_checks_need_no_gpu():
    import ctypes as C
    from paper_2506_11510_gb300 import _native as N
    L = N.lib()
    desc = N.TgVolumeDesc()
    desc.nx = desc.ny = desc.nz = 8
    desc.voxel_size = 0.125
    out = C.c_void_p()
    fake = C.c_void_p(256)
    assert L.leb_rebuild(None, fake, C.byref(desc), None, 0.0, -1.0, 4, 0, None, C.byref(out)) == N.TG_EINVAL
    assert L.leb_rebuild(fake, None, C.byref(desc), None, 0.0, -1.0, 4, 0, None, C.byref(out)) == N.TG_EINVAL
    assert L.leb_rebuild(fake, fake, C.byref(desc), None, 0.0, -1.0, 51, 0, None, C.byref(out)) == N.TG_EINVAL
    assert L.tg_batch_create(None, 1, 0, None, C.byref(out)) == N.TG_EINVAL
    jobs = (N.TgJob * 1)()
    assert L.tg_batch_create(jobs, 0, 0, None, C.byref(out)) == N.TG_EINVAL          # no jobs
    assert L.tg_batch_create(jobs, 257, 0, None, C.byref(out)) == N.TG_EINVAL        # too many
    assert L.tg_batch_create(jobs, 1, 0, None, C.byref(out)) == N.TG_EINVAL          # NULL grid
    assert L.tg_batch_render(None, None) == N.TG_EINVAL
    assert L.tg_batch_info(None, None, None) == N.TG_EINVAL
    assert L.tg_grid_channels(None, fake, None, None, None, None) == N.TG_EINVAL
    assert L.tg_grid_channels(fake, None, None, None, None, None) == N.TG_EINVAL
    assert L.tg_grid_export_channels(None, None, None, None) == N.TG_EINVAL
    cam, med = N.TgCamera(), N.TgMedium()
    cam.width = cam.height = 8
    cam.fov_y_deg = 40.0
    med.max_bounces = 4
    ext = N.TgExt()
    assert L.tet_render_ext(None, C.byref(cam), C.byref(med), C.byref(ext), 1, 0, 0, fake, None, None,
                            None) == N.TG_EINVAL
    assert L.tet_trace_ext_paths(None, C.byref(cam), C.byref(med), C.byref(ext), 0, 1, fake, fake, fake, None,
                                 None, None, None, None) == N.TG_EINVAL


def test_training_bounce_limit_changes_only_the_limit():
    """RadianceCache.train(max_bounces=k) traces its training paths in the same
    medium with the collision limit k (host logic, no GPU)."""
    import types
    from paper_2506_11510_gb300 import cache as RC, workloads as W
    m = W.scene("production").medium
    c = RC.with_max_bounces(m, 16)
    assert c.max_bounces == 16 and m.max_bounces == 128
    assert (c.albedo, c.g, c.sigma_scale, c.sun_dir, c.sun_irradiance, c.env_radiance) == \
        (m.albedo, m.g, m.sigma_scale, m.sun_dir, m.sun_irradiance, m.env_radiance)
    o = types.SimpleNamespace(albedo=.5, g=.1, sigma_scale=2., max_bounces=9, sun_dir=(0, 0, 1), sun_irradiance=1.,
                              env_radiance=0.)
    assert RC.with_max_bounces(o, 3).max_bounces == 3 and o.max_bounces == 9
    with pytest.raises(ValueError):
        RC.with_max_bounces(m, 0)


def test_sample_ranges_beyond_int32_are_refused_without_a_gpu():
    """A frame's sample indices [offset, offset + spp) must stay int32: a range past
    INT32_MAX would wrap and repeat other samples' random streams, so every render
    entry point refuses it before touching the grid or the device."""
    import ctypes as C
    from paper_2506_11510_gb300 import _native as N
    L = N.lib()
    cam, med = N.TgCamera(), N.TgMedium()
    cam.width = cam.height = 8
    cam.fov_y_deg = 40.0
    med.max_bounces = 4
    desc = N.TgVolumeDesc()
    desc.nx = desc.ny = desc.nz = 8
    desc.voxel_size = 0.125
    fake = C.c_void_p(256)              # never dereferenced: the range check comes first
    ext = N.TgExt()
    top = (1 << 31) - 1
    for spp, off in ((2, top - 1), (1, top), (top, 1)):
        assert L.tet_render(fake, C.byref(cam), C.byref(med), spp, 0, off, fake, None, None, None) == N.TG_EINVAL
        assert L.tet_render_noalloc(fake, C.byref(cam), C.byref(med), spp, 0, off, fake, None, None) == N.TG_EINVAL
        assert L.grid_render(fake, C.byref(desc), C.byref(cam), C.byref(med), spp, 0, off, fake, None, None,
                             None) == N.TG_EINVAL
        assert L.tet_render_ext(fake, C.byref(cam), C.byref(med), C.byref(ext), spp, 0, off, fake, None, None,
                                None) == N.TG_EINVAL
        assert L.tet_render_cached(fake, C.byref(cam), C.byref(med), spp, 0, off, 1, fake, fake, None, None,
                                   None) == N.TG_EINVAL
