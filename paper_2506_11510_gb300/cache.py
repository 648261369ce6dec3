"""The learned radiance cache on torch tensors (device memory and streams only).

A 3 x 64 MLP R(x, d) over a frequency encoding of position and direction ends
paths after one or two collisions; it is trained online on the tracer's own
path vertices.  Every function forwards to libtetvol.so (include/tetvol.h):
the tracer, the fused tensor-core MLP kernels and Adam all run there.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import types
from typing import Optional

import torch

from . import _native as N
from .api import Grid, _accum, _need, _paths, _ptr, _stream, camera_struct, medium_struct

NUM_PARAMS = N.RC_NUM_PARAMS


def random_paths(seed: int, n: int, width: int, height: int, sample_base: int, device=None):
    """n training paths, pixels uniform over the image (tg_random_paths)."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    px = torch.empty(n, dtype=torch.int32, device=dev)
    py = torch.empty_like(px)
    sm = torch.empty_like(px)
    N.check(N.lib().tg_random_paths(C.c_uint64(seed), n, width, height, sample_base, _ptr(px), _ptr(py), _ptr(sm),
                                    _stream()), "tg_random_paths")
    return px, py, sm


def cache_samples(grid: Grid, camera, medium, seed: int, px, py, sample, max_vertices: int, out=None,
                  want_L: bool = False, survive: float = 0.0, roulette_from: int = 0):
    """Training samples [n * max_vertices][8] (x, target, d, valid) from full paths;
    survive in (0, 1): Russian roulette after a path's last training vertex, played
    after collisions roulette_from and later (0-based)."""
    px, py, sm, dev = _paths(px, py, sample)
    n = px.numel()
    samples = out if out is not None else torch.empty((n * max_vertices, 8), dtype=torch.float32, device=dev)
    _need(samples, torch.float32, "samples", (n * max_vertices, 8))
    L = torch.empty(n, dtype=torch.float32, device=dev) if want_L else None
    N.check(N.lib().tet_cache_samples(grid.handle, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                      C.c_uint64(seed), n, _ptr(px), _ptr(py), _ptr(sm), int(max_vertices),
                                      _ptr(samples), _ptr(L), float(survive), int(roulette_from), _stream()),
            "tet_cache_samples")
    return (samples, L) if want_L else samples


def cache_queries(grid: Grid, camera, medium, seed: int, px, py, sample, cache_depth: int):
    """Cached-estimator records [n][8] (x, beta, d, L) of the listed paths."""
    px, py, sm, dev = _paths(px, py, sample)
    n = px.numel()
    rec = torch.empty((n, 8), dtype=torch.float32, device=dev)
    N.check(N.lib().tet_cache_queries(grid.handle, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                      C.c_uint64(seed), n, _ptr(px), _ptr(py), _ptr(sm), int(cache_depth), _ptr(rec),
                                      _stream()), "tet_cache_queries")
    return rec


def mlp_infer(params: torch.Tensor, rec: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """R(x, d) of every record (fused BF16 tensor-core kernel, FP32 accumulation)."""
    _need(params, torch.float32, "params", (NUM_PARAMS,))
    n = rec.shape[0]
    _need(rec, torch.float32, "rec", (n, 8))
    y = out if out is not None else torch.empty(n, dtype=torch.float32, device=rec.device)
    N.check(N.lib().rc_mlp_infer(_ptr(params), _ptr(rec), n, _ptr(y), _stream()), "rc_mlp_infer")
    return y


def mlp_grad(params: torch.Tensor, samples: torch.Tensor, grad: torch.Tensor, loss: torch.Tensor):
    """grad += d/dparams sum valid (R - target)^2; loss[0] += that sum, loss[1] += count."""
    _need(params, torch.float32, "params", (NUM_PARAMS,))
    n = samples.shape[0]
    _need(samples, torch.float32, "samples", (n, 8))
    _need(grad, torch.float32, "grad", (NUM_PARAMS,))
    _need(loss, torch.float32, "loss", (3,))
    N.check(N.lib().rc_mlp_grad(_ptr(params), _ptr(samples), n, _ptr(grad), _ptr(loss), _stream()), "rc_mlp_grad")


def adam(params, m, v, grad, loss, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.99,
         eps: float = 1e-8):
    """One Adam step on grad / max(loss[1], 1); clears grad and loss[0:2], loss[2] = mean loss."""
    for t, nm in ((params, "params"), (m, "m"), (v, "v"), (grad, "grad")):
        _need(t, torch.float32, nm, (NUM_PARAMS,))
    _need(loss, torch.float32, "loss", (3,))
    N.check(N.lib().rc_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), _ptr(loss), int(step), float(lr),
                            float(beta1), float(beta2), float(eps), _stream()), "rc_adam")


def render_cached(grid: Grid, camera, medium, spp: int, seed: int, cache_depth: int, params: torch.Tensor,
                  sample_offset: int = 0, accum_sum=None, accum_sumsq=None, stats=None, want_sq: bool = True):
    """A frame of the cached estimator (tet_render_cached), accumulated (+=)."""
    _need(params, torch.float32, "params", (NUM_PARAMS,))
    s, s2 = _accum(camera, accum_sum, accum_sumsq, want_sq)
    if stats is not None:
        _need(stats, torch.int64, "stats", (len(N.STATS_FIELDS),))
    N.check(N.lib().tet_render_cached(grid.handle, C.byref(camera_struct(camera)), C.byref(medium_struct(medium)),
                                      int(spp), C.c_uint64(seed), int(sample_offset), int(cache_depth),
                                      _ptr(params), _ptr(s), _ptr(s2), _ptr(stats), _stream()),
            "tet_render_cached")
    return s, s2


def with_max_bounces(medium, max_bounces: int):
    """The medium with another collision limit (training paths may be cut shorter
    than the rendered ones)."""
    if int(max_bounces) < 1:
        raise ValueError("max_bounces must be >= 1")
    if dataclasses.is_dataclass(medium):
        return dataclasses.replace(medium, max_bounces=int(max_bounces))
    fields = ("albedo", "g", "sigma_scale", "max_bounces", "sun_dir", "sun_irradiance", "env_radiance")
    d = {k: getattr(medium, k) for k in fields}
    d["max_bounces"] = int(max_bounces)
    return types.SimpleNamespace(**d)


def timeouts() -> int:
    c = C.c_int64()
    N.check(N.lib().rc_timeouts(C.byref(c)), "rc_timeouts")
    return c.value


class RadianceCache:
    """Online-trained radiance cache: parameters, Adam state, and one training
    round per frame on samples from the tracer's own path vertices."""

    def __init__(self, init_params, device=None, lr: float = 2e-3, beta1: float = 0.9, beta2: float = 0.99,
                 eps: float = 1e-8):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        p = torch.as_tensor(init_params, dtype=torch.float32)
        if p.shape != (NUM_PARAMS,):
            raise ValueError("init_params must have %d entries" % NUM_PARAMS)
        self.params = p.to(dev).contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(3, dtype=torch.float32, device=dev)
        self.step = 0
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps
        self._buf = None

    def train(self, grid: Grid, camera, medium, seed: int, rounds: int = 1, first_round: int = 0,
              n_paths: int = 1 << 14, max_vertices: int = 4, batches: int = 4, sample_base: int = 1 << 24,
              max_bounces: Optional[int] = None, survive: float = 0.0, roulette_from: int = 0):
        """`rounds` training rounds: each traces n_paths full paths at uniform
        pixels (sample indices disjoint from rendering's) and takes `batches`
        Adam steps on their n_paths * max_vertices vertex samples.  The paths
        of all rounds are traced in one launch, then the steps run in order.
        max_bounces, when given, cuts the training paths at that many collisions
        (their targets then miss what lies beyond; the launch no longer waits
        for the longest paths of the medium's own limit).  survive in (0, 1)
        ends the training paths sooner without biasing them: after their last
        training vertex they go on with that probability, throughput divided
        by it (Russian roulette); roulette_from > 0 plays it only after that
        collision (0-based), so that only the long tail of paths is cut."""
        if max_bounces is not None:
            medium = with_max_bounces(medium, max_bounces)
        total = rounds * n_paths
        px, py, sm = random_paths(seed ^ (0x9E3779B97F4A7C15 * (first_round + 1) & 0xFFFFFFFFFFFFFFFF), total,
                                  camera.width, camera.height,
                                  sample_base + (first_round * n_paths) % (1 << 29))
        nslot = total * max_vertices
        if self._buf is None or self._buf.shape[0] < nslot:
            self._buf = torch.empty((nslot, 8), dtype=torch.float32, device=self.params.device)
        buf = self._buf[:nslot]
        cache_samples(grid, camera, medium, seed, px, py, sm, max_vertices, out=buf, survive=survive,
                      roulette_from=roulette_from)
        per_round = n_paths * max_vertices
        per = (per_round + batches - 1) // batches
        for r in range(rounds):
            rb = buf[r * per_round:(r + 1) * per_round]
            for b in range(batches):
                chunk = rb[b * per:(b + 1) * per]
                if chunk.shape[0] == 0:
                    continue
                mlp_grad(self.params, chunk, self.grad, self.loss)
                self.step += 1
                adam(self.params, self.m, self.v, self.grad, self.loss, self.step, self.lr, self.beta1,
                     self.beta2, self.eps)
        return self.loss            # loss[2]: mean loss of the last step (device)

    def train_frame(self, grid: Grid, camera, medium, seed: int, frame: int, **kw):
        """One training round (the per-frame update of progressive rendering)."""
        return self.train(grid, camera, medium, seed, rounds=1, first_round=frame, **kw)

    def render(self, grid: Grid, camera, medium, spp: int, seed: int, cache_depth: int = 1, sample_offset: int = 0,
               accum_sum=None, accum_sumsq=None, stats=None):
        return render_cached(grid, camera, medium, spp, seed, cache_depth, self.params, sample_offset, accum_sum,
                             accum_sumsq, stats)
