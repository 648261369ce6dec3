// tet_render, tet_trace_paths, tet_optical_depth and the grid object's
// info / export / import / free entry points.
#include <cuda_fp16.h>

#include <mutex>

#include "walk_tet.cuh"

namespace tv {

thread_local cudaStream_t AllocScope::stream = nullptr;
thread_local cudaMemPool_t AllocScope::pool = nullptr;
thread_local bool AllocScope::active = false;

static std::mutex pool_mu;
static cudaMemPool_t build_pools[64] = {nullptr};

cudaMemPool_t build_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(pool_mu);
  if (!build_pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;                       // builds then allocate with cudaMalloc
    }
    unsigned long long keep = ~0ull;        // keep freed memory for the next build
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    build_pools[dev] = p;
  }
  return build_pools[dev];
}

GridImpl::~GridImpl() {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  void* ptrs[] = {rec, codes, verts, tag, count, qmin, qmax, sum, majorant, scratch, locator, chan, vmaj,
                  node_code, node_sum, node_cnt, node_mn, node_mx};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (prev >= 0) cudaSetDevice(prev);
}

static void normalize3(double v[3]) {
  const double l = std::sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
  v[0] /= l; v[1] /= l; v[2] /= l;
}

static void cross3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

CamF camera_setup(const tg_camera& c, const float box_min[3], double cube) {
  double f[3], up[3] = {c.up[0], c.up[1], c.up[2]}, r[3], u[3];
  for (int a = 0; a < 3; ++a) f[a] = (double)c.target[a] - (double)c.pos[a];
  normalize3(f);
  cross3(f, up, r);
  normalize3(r);
  cross3(r, f, u);
  normalize3(u);
  CamF o;
  for (int a = 0; a < 3; ++a) {
    o.eye[a] = ((double)c.pos[a] - (double)box_min[a]) / cube;
    o.fwd[a] = f[a];
    o.right[a] = r[a];
    o.up[a] = u[a];
  }
  o.tanF = std::tan((double)c.fov_y_deg * 0.0087266462599716478846);
  o.aspect = (double)c.width / (double)c.height;
  o.W = c.width;
  o.H = c.height;
  return o;
}

MedF medium_setup(const tg_medium& m, double cube) {
  MedF o;
  o.albedo = m.albedo;
  o.g = m.g;
  const double su = (double)m.sigma_scale * cube;
  o.sig_hi = (float)su;
  o.sig_lo = (float)(su - (double)o.sig_hi);
  o.E = m.sun_irradiance;
  o.Lenv = m.env_radiance;
  double w[3] = {-(double)m.sun_dir[0], -(double)m.sun_dir[1], -(double)m.sun_dir[2]};
  normalize3(w);
  for (int a = 0; a < 3; ++a) o.sun_w[a] = (float)w[a];
  o.max_bounces = m.max_bounces;
  return o;
}

bool camera_ok(const tg_camera* c) {
  return c && c->width > 0 && c->height > 0 && c->fov_y_deg > 0.f && c->fov_y_deg < 180.f &&
         (long long)c->width * c->height < (1ll << 31);
}

bool medium_ok(const tg_medium* m) { return m && m->max_bounces >= 1 && m->g > -1.f && m->g < 1.f; }

TetParams tet_params(const GridImpl& g) {
  TetParams p;
  p.rec = g.rec;
  p.codes = g.codes;
  p.n = g.n;
  p.K = g.K;
  p.depth = g.max_depth;
  for (int a = 0; a < 3; ++a) p.C[a] = g.C[a];
  p.scaleK = std::ldexp(1.0f, g.K);
  p.invK = std::ldexp(1.0f, -g.K);
  p.locator = g.locator;
  p.R = g.loc_R;
  return p;
}

__global__ void k_locator(TetParams P, int32_t* out, int nx, int ny, int nz) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nx * ny * nz) return;
  const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
  const float h = 1.0f / (float)P.R;
  const long long c = tet_locate(P, make_float3(((float)x + 0.5f) * h, ((float)y + 0.5f) * h, ((float)z + 0.5f) * h));
  out[i] = (int32_t)c;
}

void build_locator(GridImpl& G, cudaStream_t st) {
  if (G.n == 0) return;
  // about one locator cell per 4 tetrahedra, a power of two per cube edge in [8, 256]
  const double cubes = (double)G.C[0] * G.C[1] * G.C[2];
  int R = 8;
  while (R < 256 && (double)(2 * R) * (2 * R) * (2 * R) * cubes <= (double)G.n / 4.0) R *= 2;
  const long long nx = (long long)G.C[0] * R, ny = (long long)G.C[1] * R, nz = (long long)G.C[2] * R;
  DevBuf<int32_t> loc((size_t)(nx * ny * nz));
  TetParams p = tet_params(G);
  p.locator = nullptr;
  p.R = R;
  k_locator<<<(unsigned)((nx * ny * nz + 255) / 256), 256, 0, st>>>(p, loc.p, (int)nx, (int)ny, (int)nz);
  TV_LAUNCH();
  G.locator = loc.release();
  G.loc_R = R;
}

EstParams est_params(const GridImpl& g, const tg_camera& cam, const tg_medium& med, uint64_t seed) {
  EstParams ep;
  std::memset(&ep, 0, sizeof ep);
  ep.cam = camera_setup(cam, g.box_min, g.cube);
  ep.med = medium_setup(med, g.cube);
  ep.seed = seed;
  ep.regen_min = TV_REGEN_MIN;
  ep.ev_min = TV_EV_MIN;
  for (int a = 0; a < 3; ++a) ep.ext[a] = (float)g.C[a];
  return ep;
}

// ---------------------------------------------------------------------------
// Walk only: optical depth along grid-space rays.
// ---------------------------------------------------------------------------
template <int FMT>
__global__ void __launch_bounds__(EST_BLOCK) k_optical_depth(const TetParams P, long long n, const float* origin,
                                                            const float* dir, float sigma, float* tau,
                                                            int64_t* steps, int32_t* seq, int seq_cap,
                                                            int32_t* seq_len) {
  extern __shared__ __align__(16) double smem_d[];
  TetWalker<FMT> W(P, smem_d);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float3 o = make_float3(origin[3 * i], origin[3 * i + 1], origin[3 * i + 2]);
  float3 d = make_float3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
  const float inv = 1.0f / sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
  d = make_float3(d.x * inv, d.y * inv, d.z * inv);
  float od = 0.f, tin;
  long long k = 0;
  int len = 0;
  if (W.intersect(o, d, &tin)) {
    const ff3 e = {ff_add(ff_make(o.x), two_prod(tin, d.x)), ff_add(ff_make(o.y), two_prod(tin, d.y)),
                   ff_add(ff_make(o.z), two_prod(tin, d.z))};
    if (W.locate(make_float3(ff_float(e.x), ff_float(e.y), ff_float(e.z)))) {
      float tinv[TetWalker<FMT>::NDIR];
      W.dir_table(ff3{ff_make(d.x), ff_make(d.y), ff_make(d.z)}, tinv);
      W.begin(e, tinv);
      float t = 0.f;
      for (; k < SEG_STEP_LIMIT; ++k) {
        if (seq && len < seq_cap) seq[i * seq_cap + len] = W.cell();
        ++len;
        const Hop h = W.hop(t);
        if (!h.ok) break;
        od += sigma * h.rho * (h.texit - t);
        t = h.texit;
        if (!W.advance()) { ++k; break; }
      }
    }
  }
  tau[i] = od;
  if (steps) steps[i] = k;
  if (seq_len) seq_len[i] = len < seq_cap ? len : seq_cap;
}

}  // namespace tv

using namespace tv;

#define TV_API_BEGIN try {
#define TV_API_END                       \
  }                                      \
  catch (const tv::Error& e) {           \
    return e.code;                       \
  }                                      \
  catch (const std::bad_alloc&) {        \
    return TG_ENOMEM;                    \
  }                                      \
  catch (...) {                          \
    return TG_ECUDA;                     \
  }

extern "C" {

const char* tg_error_string(int s) {
  switch (s) {
    case TG_OK: return "ok";
    case TG_EINVAL: return "invalid argument";
    case TG_ENOMEM: return "out of device memory";
    case TG_ECUDA: return "CUDA error";
    case TG_ESTEPLIMIT: return "walk step limit exceeded";
    case TG_EROUNDLIMIT: return "grid build did not converge";
    case TG_EGRID: return "grid is not conforming";
    default: return "unknown status";
  }
}

int tg_grid_info(const tg_grid* g, int64_t* num_tets, int32_t* max_depth, int64_t* bytes, int32_t* K,
                 int32_t* rounds) {
  if (!g) return TG_EINVAL;
  const GridImpl& G = g->impl;
  if (num_tets) *num_tets = G.n;
  if (max_depth) *max_depth = G.max_depth;
  if (bytes) *bytes = G.n * (int64_t)(32 + 8);
  if (K) *K = G.K;
  if (rounds) *rounds = G.rounds;
  return TG_OK;
}

void tg_grid_free(tg_grid* g) { delete g; }

int tg_release_build_memory(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return TG_ECUDA;
  }
  cudaMemPool_t p = nullptr;
  {
    std::lock_guard<std::mutex> lk(pool_mu);
    p = build_pools[dev];
  }
  if (!p) return TG_OK;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(p, 0) != cudaSuccess) return TG_ECUDA;
  return TG_OK;
}

int tet_render(const tg_grid* g, const tg_camera* cam, const tg_medium* med, int32_t spp, uint64_t seed,
               int32_t sample_offset, float* accum_sum, float* accum_sumsq, tg_stats* stats, void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || !samples_ok(spp, sample_offset) || !accum_sum) return TG_EINVAL;
  TV_API_BEGIN
  const GridImpl& G = g->impl;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (spp == 0 || G.n == 0) return TG_OK;
  EstParams ep = est_params(G, *cam, *med, seed);
  ep.spp = spp;
  ep.sample_offset = sample_offset;
  ep.total = (long long)cam->width * cam->height * spp;
  CallCounter counter(st);
  ep.counter = counter.p;
  ep.sum = accum_sum;
  ep.sumsq = accum_sumsq;
  ep.stats = stats;
  run_tet<MODE_RENDER>(G, ep, st);
  return TG_OK;
  TV_API_END
}

int tet_trace_paths(const tg_grid* g, const tg_camera* cam, const tg_medium* med, uint64_t seed, int64_t n,
                    const int32_t* px, const int32_t* py, const int32_t* sample, float* L, int32_t* flags,
                    int32_t* collisions, int64_t* steps, int32_t* seq, int32_t seq_cap, int32_t* seq_len,
                    void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || n < 0 || (n > 0 && (!px || !py || !sample)) ||
      (seq && seq_cap <= 0))
    return TG_EINVAL;
  TV_API_BEGIN
  const GridImpl& G = g->impl;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n == 0) return TG_OK;
  EstParams ep = est_params(G, *cam, *med, seed);
  ep.spp = 1;
  ep.total = n;
  CallCounter counter(st);
  ep.counter = counter.p;
  ep.px = px; ep.py = py; ep.ps = sample;
  ep.outL = L; ep.outFlags = flags; ep.outColl = collisions; ep.outSteps = steps;
  ep.seq = seq; ep.seq_cap = seq ? seq_cap : 0; ep.seq_len = seq_len;
  run_tet<MODE_TRACE>(G, ep, st);
  return TG_OK;
  TV_API_END
}

int tet_optical_depth(const tg_grid* g, int64_t n, const float* origin, const float* dir, float sigma, float* tau,
                      int64_t* steps, int32_t* seq, int32_t seq_cap, int32_t* seq_len, void* cuda_stream) {
  if (!g || n < 0 || (n > 0 && (!origin || !dir || !tau)) || (seq && seq_cap <= 0)) return TG_EINVAL;
  TV_API_BEGIN
  const GridImpl& G = g->impl;
  if (n == 0 || G.n == 0) return TG_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const TetParams p = tet_params(G);
  const unsigned blocks = (unsigned)((n + EST_BLOCK - 1) / EST_BLOCK);
  const size_t shm = TetWalker<0>::smem_bytes();
  switch (G.fmt) {
    case TG_DENSITY_BF16:
      k_optical_depth<TG_DENSITY_BF16><<<blocks, EST_BLOCK, shm, st>>>(p, n, origin, dir, sigma, tau, steps, seq,
                                                                        seq_cap, seq_len);
      break;
    case TG_DENSITY_FP16:
      k_optical_depth<TG_DENSITY_FP16><<<blocks, EST_BLOCK, shm, st>>>(p, n, origin, dir, sigma, tau, steps, seq,
                                                                        seq_cap, seq_len);
      break;
    default:
      k_optical_depth<TG_DENSITY_FP32><<<blocks, EST_BLOCK, shm, st>>>(p, n, origin, dir, sigma, tau, steps, seq,
                                                                        seq_cap, seq_len);
  }
  TV_LAUNCH();
  return TG_OK;
  TV_API_END
}

}  // extern "C"
