// tet_render_noalloc: a frame render that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand
// all device memory out of their own pool or a fixed budget (a framework's
// caching allocator, a renderer embedded in a larger GPU program), and loops
// that cannot afford cudaMalloc's implicit device synchronisation.  This entry
// point serves them.  Its scratch -- the path-id counter of the persistent
// estimator and one 16-byte record per path (pixel, sample, estimate) -- is the
// file-scope array below, which every device that loads the library holds
// until the process exits.  The caller still passes the grid and the output
// image; the per-pixel sums are formed in a fixed sample order, so the result
// does not depend on thread scheduling.
#include <mutex>

#include "walk_tet.cuh"

namespace tv {

constexpr long long NOALLOC_MAX_PATHS = TG_NOALLOC_MAX_PATHS;
constexpr size_t NOALLOC_BYTES = 256 + (size_t)NOALLOC_MAX_PATHS * 16;

// scratch: [0, 256) counter, then px, py, sample (int32) and L (float) per path
static __device__ __align__(256) unsigned char noalloc_scratch[NOALLOC_BYTES];

// Device address of the scratch array on the current device: looked up once per
// device (with that device current) and cached.  A host-side symbol is not a
// device address, so kernels only ever receive this looked-up pointer.
static unsigned char* scratch_address(int* status) {
  static std::mutex mu;
  static unsigned char* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { *status = TG_ECUDA; return nullptr; }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) { *status = TG_ECUDA; return nullptr; }
    addr[dev] = static_cast<unsigned char*>(p);
  }
  *status = TG_OK;
  return addr[dev];
}

__global__ void k_noalloc_paths(int32_t* px, int32_t* py, int32_t* ps, long long n, int W, int spp, int offset) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long pix = i / spp;
  px[i] = (int32_t)(pix % W);
  py[i] = (int32_t)(pix / W);
  ps[i] = offset + (int32_t)(i - pix * spp);
}

__global__ void k_noalloc_sum(const float* L, long long npix, int spp, float* sum, float* sumsq) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  float s = 0.f, s2 = 0.f;
  for (int k = 0; k < spp; ++k) {
    const float v = L[p * spp + k];
    s += v;
    s2 += v * v;
  }
  sum[p] += s;
  if (sumsq) sumsq[p] += s2;
}

}  // namespace tv

using namespace tv;

extern "C" int tet_render_noalloc(const tg_grid* g, const tg_camera* cam, const tg_medium* med, int32_t spp,
                                  uint64_t seed, int32_t sample_offset, float* accum_sum, float* accum_sumsq,
                                  void* cuda_stream) {
  if (!g || !camera_ok(cam) || !medium_ok(med) || !samples_ok(spp, sample_offset) || !accum_sum) return TG_EINVAL;
  const long long npix = (long long)cam->width * cam->height;
  const long long n = npix * spp;
  if (n > NOALLOC_MAX_PATHS) return TG_EINVAL;          // more paths than the scratch array holds
  const GridImpl& G = g->impl;
  if (n == 0 || G.n == 0) return TG_OK;
  int status = TG_OK;
  unsigned char* base = scratch_address(&status);
  if (!base) return status;
  try {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(base);
    int32_t* px = reinterpret_cast<int32_t*>(base + 256);
    int32_t* py = px + NOALLOC_MAX_PATHS;
    int32_t* ps = py + NOALLOC_MAX_PATHS;
    float* L = reinterpret_cast<float*>(ps + NOALLOC_MAX_PATHS);
    // the counter must start at zero; the other arrays are fully written before they are read
    TV_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_noalloc_paths<<<blocks, 256, 0, st>>>(px, py, ps, n, cam->width, spp, sample_offset);
    TV_LAUNCH();
    // the renderer's own parameters for this grid, camera and medium; only the
    // per-path list, its length, the counter and the output differ
    EstParams ep = est_params(G, *cam, *med, seed);
    ep.spp = 1;
    ep.total = n;
    ep.counter = counter;
    ep.px = px; ep.py = py; ep.ps = ps;
    ep.outL = L;
    run_tet<MODE_TRACE>(G, ep, st);
    k_noalloc_sum<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(L, npix, spp, accum_sum, accum_sumsq);
    TV_LAUNCH();
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}
