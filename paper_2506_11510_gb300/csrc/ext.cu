// The extended medium: extra per-cell channels (temperature -> emission,
// albedo, g) and the voxel medium tracked against per-cell voxel majorants
// (tet_render_ext, tet_trace_ext_paths).
#include "walk_tet.cuh"

namespace tv {

static int ext_setup(const GridImpl& G, const tg_ext* x, EstParams& ep) {
  if (!x || (x->flags & ~15) || x->flags == 0) return TG_EINVAL;
  const int need = (x->flags & 7) | ((x->flags & EXT_VOXEL) ? 8 : 0);
  if ((need & ~G.chan_mask) != 0) return TG_EINVAL;             // channels not computed (tg_grid_channels)
  if ((x->flags & EXT_VOXEL) && !x->density) return TG_EINVAL;
  if ((x->flags & EXT_EMISSION) && !(x->emission_scale >= 0.f)) return TG_EINVAL;
  ep.ext_flags = x->flags;
  ep.emission_scale = x->emission_scale;
  ep.chan = G.chan;
  ep.vmaj = G.vmaj;
  ep.voxel = x->density;
  for (int a = 0; a < 3; ++a) ep.vdim[a] = G.nvox[a];
  ep.vn = (float)G.n_per_cube;
  return TG_OK;
}

}  // namespace tv

using namespace tv;

extern "C" {

int tet_render_ext(const tg_grid* g, const tg_camera* cam, const tg_medium* med, const tg_ext* ext, int32_t spp,
                   uint64_t seed, int32_t sample_offset, float* accum_sum, float* accum_sumsq, tg_stats* stats,
                   void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || !samples_ok(spp, sample_offset) || !accum_sum) return TG_EINVAL;
  try {
    const GridImpl& G = g->impl;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    EstParams ep = est_params(G, *cam, *med, seed);
    const int s = ext_setup(G, ext, ep);
    if (s != TG_OK) return s;
    if (spp == 0 || G.n == 0) return TG_OK;
    ep.spp = spp;
    ep.sample_offset = sample_offset;
    ep.total = (long long)cam->width * cam->height * spp;
    CallCounter counter(st);
    ep.counter = counter.p;
    ep.sum = accum_sum;
    ep.sumsq = accum_sumsq;
    ep.stats = stats;
    run_tet<MODE_RENDER, true>(G, ep, st);
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int tet_trace_ext_paths(const tg_grid* g, const tg_camera* cam, const tg_medium* med, const tg_ext* ext,
                        uint64_t seed, int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                        float* L, int32_t* flags, int32_t* collisions, int64_t* steps, void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || n < 0 || (n > 0 && (!px || !py || !sample))) return TG_EINVAL;
  try {
    const GridImpl& G = g->impl;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    EstParams ep = est_params(G, *cam, *med, seed);
    const int s = ext_setup(G, ext, ep);
    if (s != TG_OK) return s;
    if (n == 0) return TG_OK;
    ep.spp = 1;
    ep.total = n;
    CallCounter counter(st);
    ep.counter = counter.p;
    ep.px = px; ep.py = py; ep.ps = sample;
    ep.outL = L; ep.outFlags = flags; ep.outColl = collisions; ep.outSteps = steps;
    run_tet<MODE_TRACE, true>(G, ep, st);
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

}  // extern "C"
