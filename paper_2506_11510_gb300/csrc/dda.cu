// grid_render / grid_trace_paths: the regular-grid comparator, the same
// estimator as tet_render walking voxels with a 3D DDA.
#include <mutex>
#include <vector>

#include "walk_voxel.cuh"

namespace tv {

static bool vol_setup(const tg_volume_desc* v, VoxParams* p, double* cube, float box_min[3]) {
  if (!v || v->nx <= 0 || v->ny <= 0 || v->nz <= 0 || !(v->voxel_size > 0)) return false;
  if ((long long)v->nx * v->ny * v->nz >= (1ll << 31)) return false;
  int n = 1;
  while (v->nx % (2 * n) == 0 && v->ny % (2 * n) == 0 && v->nz % (2 * n) == 0 && n < (1 << 18)) n *= 2;
  p->nx = v->nx; p->ny = v->ny; p->nz = v->nz;
  p->n_f = (float)n;
  p->inv_n = 1.0f / (float)n;
  p->C[0] = v->nx / n; p->C[1] = v->ny / n; p->C[2] = v->nz / n;
  *cube = (double)v->voxel_size * (double)n;
  for (int a = 0; a < 3; ++a) box_min[a] = v->box_min[a];
  return true;
}

static EstParams dda_est(const tg_camera& cam, const tg_medium& med, uint64_t seed, double cube,
                         const float box_min[3]) {
  EstParams ep;
  std::memset(&ep, 0, sizeof ep);
  ep.cam = camera_setup(cam, box_min, cube);
  ep.med = medium_setup(med, cube);
  ep.seed = seed;
  ep.regen_min = TV_REGEN_MIN;
  ep.ev_min = TV_EV_MIN;
  for (int a = 0; a < 3; ++a) ep.ext[a] = 1.0f;
  return ep;
}

}  // namespace tv

using namespace tv;

extern "C" {

int grid_render(const float* density, const tg_volume_desc* vol, const tg_camera* cam, const tg_medium* med,
                int32_t spp, uint64_t seed, int32_t sample_offset, float* accum_sum, float* accum_sumsq,
                tg_stats* stats, void* cuda_stream) {
  VoxParams p;
  double cube;
  float bmin[3];
  if (!density || !accum_sum || !camera_ok(cam) || !medium_ok(med) || !samples_ok(spp, sample_offset) ||
      !vol_setup(vol, &p, &cube, bmin))
    return TG_EINVAL;
  try {
    if (spp == 0) return TG_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    p.rho = density;
    EstParams ep = dda_est(*cam, *med, seed, cube, bmin);
    ep.spp = spp;
    ep.sample_offset = sample_offset;
    ep.total = (long long)cam->width * cam->height * spp;
    CallCounter counter(st);
    ep.counter = counter.p;
    ep.sum = accum_sum;
    ep.sumsq = accum_sumsq;
    ep.stats = stats;
    launch_estimate<VoxelWalker, MODE_RENDER>(p, ep, st);
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int grid_trace_paths(const float* density, const tg_volume_desc* vol, const tg_camera* cam, const tg_medium* med,
                     uint64_t seed, int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample, float* L,
                     int32_t* flags, int32_t* collisions, int64_t* steps, void* cuda_stream) {
  VoxParams p;
  double cube;
  float bmin[3];
  if (!density || !camera_ok(cam) || !medium_ok(med) || n < 0 || (n > 0 && (!px || !py || !sample)) ||
      !vol_setup(vol, &p, &cube, bmin))
    return TG_EINVAL;
  try {
    if (n == 0) return TG_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    p.rho = density;
    EstParams ep = dda_est(*cam, *med, seed, cube, bmin);
    ep.spp = 1;
    ep.total = n;
    CallCounter counter(st);
    ep.counter = counter.p;
    ep.px = px; ep.py = py; ep.ps = sample;
    ep.outL = L; ep.outFlags = flags; ep.outColl = collisions; ep.outSteps = steps;
    launch_estimate<VoxelWalker, MODE_TRACE>(p, ep, st);
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

}  // extern "C"
