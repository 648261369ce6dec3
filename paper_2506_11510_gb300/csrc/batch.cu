// Batched heterogeneous rendering: many grids, cameras, media and images in
// one persistent launch (k_estimate<TetWalker<FMT, true>, MODE_RENDER, false,
// true>), captured in a CUDA graph, with launch knobs chosen by timing a small
// set of candidates (tg_batch_create).
#include <algorithm>
#include <cmath>
#include <vector>

#include "walk_tet.cuh"

namespace tv {

using Job = BatchJob<TetParams>;

// The direction table of each job's sun (the one thread per job the tables need)
__global__ void k_sun_tables(Job* jobs, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const MedF& m = jobs[i].med;
  float inv[TET_NID];
  tet_dir_table(ff3{ff_make(m.sun_w[0]), ff_make(m.sun_w[1]), ff_make(m.sun_w[2])}, jobs[i].wp.invK, inv);
  for (int q = 0; q < TET_NID; ++q) jobs[i].sun_inv[q] = inv[q];
}

struct Knobs {
  int regen_min, ev_min, blocks_per_sm, order;    // order 0: as given, 1: costliest jobs first
};

}  // namespace tv

struct tg_batch {
  int device = 0;
  int fmt = 0;
  int n = 0;
  std::vector<tv::Job> host;                     // the jobs in the caller's order
  std::vector<int> perm;                         // launch order (perm[k] = caller index)
  tv::DevBuf<tv::Job> table;
  tv::DevBuf<unsigned long long> done, times;
  tv::DevBuf<float> scratch;                     // tuning renders go here
  tv::Knobs knobs{TV_REGEN_MIN, TV_EV_MIN, 0, 0};
  long long total = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~tg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

namespace tv {

// Lay the jobs out in launch order (with their first path ids) and upload.
static void upload(tg_batch& b, const Knobs& k, bool to_scratch, cudaStream_t st) {
  std::vector<int> perm(b.n);
  for (int i = 0; i < b.n; ++i) perm[i] = i;
  if (k.order == 1) {
    std::vector<double> cost(b.n);
    for (int i = 0; i < b.n; ++i)
      cost[i] = (double)b.host[i].paths * std::cbrt((double)std::max<long long>(1, b.host[i].wp.n));
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  }
  std::vector<Job> t(b.n);
  long long base = 0;
  for (int k2 = 0; k2 < b.n; ++k2) {
    t[k2] = b.host[perm[k2]];
    t[k2].base = base;
    base += t[k2].paths;
    if (to_scratch) {
      t[k2].sum = b.scratch.p;
      t[k2].sumsq = nullptr;
    }
  }
  b.perm = perm;
  TV_CUDA(cudaMemcpyAsync(b.table.p, t.data(), sizeof(Job) * b.n, cudaMemcpyHostToDevice, st));
  k_sun_tables<<<(b.n + 63) / 64, 64, 0, st>>>(b.table.p, b.n);
  TV_LAUNCH();
}

static void launch(tg_batch& b, const Knobs& k, cudaStream_t st) {
  EstParams ep;
  std::memset(&ep, 0, sizeof ep);
  ep.regen_min = k.regen_min;
  ep.ev_min = k.ev_min;
  ep.total = b.total;
  ep.counter = b.done.p + b.n;                   // the launch's path counter
  ep.jobs = b.table.p;
  ep.njobs = b.n;
  ep.job_done = b.done.p;
  ep.job_time = b.times.p;
  ep.med = b.host[0].med;                        // unused by a batch launch
  ep.cam = b.host[0].cam;
  TV_CUDA(cudaMemsetAsync(b.done.p, 0, sizeof(unsigned long long) * (b.n + 1), st));
  TV_CUDA(cudaMemsetAsync(b.times.p, 0xFF, sizeof(unsigned long long) * (b.n + 1), st));
  const TetParams& wp = b.host[0].wp;
  switch (b.fmt) {
    case TG_DENSITY_BF16:
      launch_estimate<TetWalker<TG_DENSITY_BF16, true>, MODE_RENDER, false, true>(wp, ep, st, k.blocks_per_sm);
      break;
    case TG_DENSITY_FP16:
      launch_estimate<TetWalker<TG_DENSITY_FP16, true>, MODE_RENDER, false, true>(wp, ep, st, k.blocks_per_sm);
      break;
    default:
      launch_estimate<TetWalker<TG_DENSITY_FP32, true>, MODE_RENDER, false, true>(wp, ep, st, k.blocks_per_sm);
  }
}

static void capture(tg_batch& b, cudaStream_t user) {
  if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
  if (b.graph) { cudaGraphDestroy(b.graph); b.graph = nullptr; }
  cudaStream_t cs;
  TV_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  TV_CUDA(cudaStreamSynchronize(user));
  try {
    TV_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    launch(b, b.knobs, cs);
    TV_CUDA(cudaStreamEndCapture(cs, &b.graph));
    TV_CUDA(cudaGraphInstantiate(&b.exec, b.graph, 0));
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    throw;
  }
  TV_CUDA(cudaStreamDestroy(cs));
}

}  // namespace tv

using namespace tv;

extern "C" {

int tg_batch_create(const tg_job* jobs, int32_t njobs, int32_t autotune, void* cuda_stream, tg_batch** out) {
  if (!jobs || !out || njobs < 1 || njobs > BATCH_MAX_JOBS) return TG_EINVAL;
  int fmt = -1;
  long long total = 0, maxpix = 0;
  for (int i = 0; i < njobs; ++i) {
    const tg_job& j = jobs[i];
    if (!j.grid || !camera_ok(&j.cam) || !medium_ok(&j.med) || j.spp < 1 || !samples_ok(j.spp, j.sample_offset) || !j.accum_sum)
      return TG_EINVAL;
    if (j.grid->impl.n == 0) return TG_EINVAL;
    if (fmt >= 0 && j.grid->impl.fmt != fmt) return TG_EINVAL;   // one density format per batch
    fmt = j.grid->impl.fmt;
    total += (long long)j.cam.width * j.cam.height * j.spp;
    maxpix = std::max(maxpix, (long long)j.cam.width * j.cam.height);
  }
  tg_batch* b = new (std::nothrow) tg_batch();
  if (!b) return TG_ENOMEM;
  try {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    TV_CUDA(cudaGetDevice(&b->device));
    b->fmt = fmt;
    b->n = njobs;
    b->total = total;
    b->host.resize(njobs);
    for (int i = 0; i < njobs; ++i) {
      const tg_job& j = jobs[i];
      const GridImpl& G = j.grid->impl;
      Job& h = b->host[i];
      std::memset(&h, 0, sizeof h);
      h.wp = tet_params(G);
      h.cam = camera_setup(j.cam, G.box_min, G.cube);
      h.med = medium_setup(j.med, G.cube);
      h.sum = j.accum_sum;
      h.sumsq = j.accum_sumsq;
      h.seed = j.seed;
      h.paths = (long long)j.cam.width * j.cam.height * j.spp;
      h.spp = j.spp;
      h.sample_offset = j.sample_offset;
    }
    b->table.alloc(njobs);
    b->done.alloc(njobs + 1);
    b->times.alloc(njobs + 1);
    if (autotune) {
      // timed trial launches render into a scratch image
      b->scratch.alloc((size_t)maxpix);
      int dev = 0, per_sm = 0;
      TV_CUDA(cudaGetDevice(&dev));
      const size_t shm = TetWalker<TG_DENSITY_FP32, true>::smem_bytes();
      TV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, k_estimate<TetWalker<TG_DENSITY_FP32, true>, MODE_RENDER, false, true>, EST_BLOCK, shm));
      cudaEvent_t e0, e1;
      TV_CUDA(cudaEventCreate(&e0));
      TV_CUDA(cudaEventCreate(&e1));
      auto trial = [&](const Knobs& k) {
        upload(*b, k, true, st);
        TV_CUDA(cudaEventRecord(e0, st));
        launch(*b, k, st);
        TV_CUDA(cudaEventRecord(e1, st));
        TV_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
      };
      // coordinate descent over the knobs, one pass: each knob in turn takes the
      // value that times fastest with the others held
      Knobs cur = b->knobs;
      float best = trial(cur);
      const int bps_alt = std::max(1, per_sm - 1);
      for (int knob = 0; knob < 4; ++knob) {
        std::vector<int> values;
        if (knob == 0) values = {4, 8, 16};
        else if (knob == 1) values = {8, 12, 16};
        else if (knob == 2) values = {0, bps_alt};
        else values = {0, 1};
        for (int v : values) {
          Knobs k = cur;
          if (knob == 0) { if (v == k.regen_min) continue; k.regen_min = v; }
          else if (knob == 1) { if (v == k.ev_min) continue; k.ev_min = v; }
          else if (knob == 2) { if (v == k.blocks_per_sm) continue; k.blocks_per_sm = v; }
          else { if (v == k.order) continue; k.order = v; }
          const float ms = trial(k);
          if (ms < best) { best = ms; cur = k; }
        }
      }
      b->knobs = cur;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      b->scratch.alloc(0);
    }
    upload(*b, b->knobs, false, st);
    capture(*b, st);
  } catch (const Error& e) {
    delete b;
    return e.code;
  }
  *out = b;
  return TG_OK;
}

int tg_batch_render(tg_batch* b, void* cuda_stream) {
  if (!b || !b->exec) return TG_EINVAL;
  if (cudaGraphLaunch(b->exec, (cudaStream_t)cuda_stream) != cudaSuccess) return TG_ECUDA;
  return TG_OK;
}

int tg_batch_info(const tg_batch* b, int32_t* knobs, double* job_ms) {
  if (!b) return TG_EINVAL;
  if (knobs) {
    knobs[0] = b->knobs.regen_min; knobs[1] = b->knobs.ev_min; knobs[2] = b->knobs.blocks_per_sm;
    knobs[3] = b->knobs.order;
  }
  if (job_ms) {
    std::vector<unsigned long long> t(b->n + 1);
    if (cudaMemcpy(t.data(), b->times.p, sizeof(unsigned long long) * (b->n + 1), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return TG_ECUDA;
    for (int k = 0; k < b->n; ++k) job_ms[b->perm[k]] = (double)(long long)(t[k] - t[b->n]) * 1e-6;
  }
  return TG_OK;
}

void tg_batch_free(tg_batch* b) { delete b; }

}  // extern "C"
