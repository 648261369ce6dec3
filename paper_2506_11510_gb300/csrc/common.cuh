// Shared device/host pieces of libtetvol: error handling, the grid object,
// Philox4x32-10, Henyey-Greenstein sampling, camera set-up.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <new>
#include <utility>

#include "../../include/tetvol.h"

namespace tv {

struct Error {
  int code;
};

inline void check(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) throw Error{TG_ENOMEM};
  if (e != cudaSuccess) throw Error{TG_ECUDA};
}
#define TV_CUDA(x) ::tv::check(x)
#define TV_LAUNCH() ::tv::check(cudaGetLastError())

// Stream-ordered allocations of a build: while a build runs on a stream, the
// library's buffers come from a memory pool owned by the library (one per
// device) that keeps freed memory for the next build instead of returning it
// to the driver (a production build's temporaries are tens of GB, and
// allocating and freeing them took about 45 ms of a 267 ms build); elsewhere
// they use plain cudaMalloc / cudaFree.  tg_release_build_memory() hands the
// pool's unused memory back.
struct AllocScope {
  static thread_local cudaStream_t stream;
  static thread_local cudaMemPool_t pool;
  static thread_local bool active;
  cudaStream_t prev_stream;
  cudaMemPool_t prev_pool;
  bool prev_active;
  AllocScope(cudaStream_t st, cudaMemPool_t p) : prev_stream(stream), prev_pool(pool), prev_active(active) {
    stream = st; pool = p; active = p != nullptr;
  }
  ~AllocScope() { stream = prev_stream; pool = prev_pool; active = prev_active; }
};
cudaMemPool_t build_pool();      // the current device's pool (created on first use), or nullptr

inline void* dev_alloc(size_t bytes) {
  void* p = nullptr;
  if (AllocScope::active) check(cudaMallocFromPoolAsync(&p, bytes, AllocScope::pool, AllocScope::stream));
  else check(cudaMalloc(&p, bytes));
  return p;
}
inline void dev_free(void* p) {
  if (!p) return;
  if (AllocScope::active) cudaFreeAsync(p, AllocScope::stream);
  else cudaFree(p);
}

// Scratch of one call (a renderer's path counter, a cached frame's path
// records): taken from the library's stream-ordered pool on the call's stream
// and given back on that stream after the call's last kernel, so calls on
// other streams -- on the same grid or not -- never share it.
template <class T>
struct CallScratch {
  T* p = nullptr;
  cudaStream_t st;
  CallScratch(size_t count, cudaStream_t s) : st(s) {
    cudaMemPool_t pool = build_pool();
    void* q = nullptr;
    if (pool) check(cudaMallocFromPoolAsync(&q, count * sizeof(T), pool, s));
    else check(cudaMallocAsync(&q, count * sizeof(T), s));
    p = static_cast<T*>(q);
  }
  CallScratch(const CallScratch&) = delete;
  CallScratch& operator=(const CallScratch&) = delete;
  ~CallScratch() { if (p) cudaFreeAsync(p, st); }
};

// A zeroed path-id counter for one persistent-estimator launch on stream s.
struct CallCounter : CallScratch<unsigned long long> {
  explicit CallCounter(cudaStream_t s) : CallScratch<unsigned long long>(1, s) {
    check(cudaMemsetAsync(p, 0, sizeof(unsigned long long), s));
  }
};

// Device allocation owned by the library (RAII).
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept { std::swap(p, o.p); std::swap(n, o.n); return *this; }
  ~DevBuf() { if (p) dev_free(p); }
  void alloc(size_t count) {
    if (p) { dev_free(p); p = nullptr; n = 0; }
    if (count == 0) return;
    p = static_cast<T*>(dev_alloc(count * sizeof(T)));
    n = count;
  }
  // grow geometrically: scratch that follows a growing size is reallocated O(log) times
  void ensure(size_t count) { if (count > n) alloc(count > 2 * n ? count : 2 * n); }
  T* release() { T* r = p; p = nullptr; n = 0; return r; }
};

// ---------------------------------------------------------------------------
// Record layout of one tetrahedron (32 bytes, one DRAM sector):
//   word 0..3  link[f]  bits 0..26 index of the cell across face f (NO_NBR on
//                       the domain boundary), bits 27..31 face orientation
//                       p | s << 4 (outward normal (-1)^s P[p])
//   word 4..6  the four plane offsets P[p] . v in units of 2^-K cube, as
//              24-bit two's complement integers packed back to back
//   word 7     density: fp32 bits; bf16 bits in the high half with the low half
//              zero (the word is the density as a float); or fp16 bits in the low half
// ---------------------------------------------------------------------------
constexpr uint32_t NO_NBR = 0x7FFFFFFu;
constexpr int64_t MAX_TETS = 0x7FFFFFE;

struct GridImpl {
  int device = 0;
  int64_t n = 0;
  int K = 0, max_depth = 0, rounds = 0, fmt = 0;
  int C[3] = {1, 1, 1};
  int nvox[3] = {0, 0, 0};
  int n_per_cube = 1;
  float box_min[3] = {0, 0, 0};
  float voxel_size = 1;
  double cube = 1;                       // world size of a cube
  uint4* rec = nullptr;                  // 2 x uint4 per cell
  unsigned long long* codes = nullptr;
  int32_t* verts = nullptr;              // [n][12], absent for imported grids
  uint8_t* tag = nullptr;
  uint32_t *count = nullptr, *qmin = nullptr, *qmax = nullptr;
  unsigned long long* sum = nullptr;
  float* majorant = nullptr;
  unsigned long long* scratch = nullptr; // work counter of the persistent renderer
  int32_t* locator = nullptr;            // cell of each locator-grid cell centre (loc_R per cube edge)
  int loc_R = 0;
  float4* chan = nullptr;                // extra channels per cell: temperature, albedo, g, 0
  float* vmaj = nullptr;                 // voxel majorant per cell
  int chan_mask = 0;                     // 1 temperature, 2 albedo, 4 g, 8 majorants present
  // statistics of the interior nodes of the LEB tree, sorted by code (rebuilds)
  long long n_nodes = 0;
  unsigned long long *node_code = nullptr, *node_sum = nullptr;
  uint32_t *node_cnt = nullptr, *node_mn = nullptr, *node_mx = nullptr;
  ~GridImpl();
};

// Builds G.locator (point-location accelerator) for a finished grid.
void build_locator(GridImpl& G, cudaStream_t st);

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies
// with xor mixing; the key is bumped by the golden-ratio / sqrt(3) Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), hi1 = __umulhi(0xCD9E8D57u, c.z);
#else
    const uint32_t hi0 = (uint32_t)(((uint64_t)0xD2511F53u * c.x) >> 32);
    const uint32_t hi1 = (uint32_t)(((uint64_t)0xCD9E8D57u * c.z) >> 32);
#endif
    const uint32_t lo0 = 0xD2511F53u * c.x, lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// u in [0, 1): slot `slot` of stream `stream` of path (pixel, sample); key
// (seed lo, seed hi ^ pixel), counter (sample, slot / 4, stream, 0), 24 high bits
// of word slot % 4.  Stream 0 holds the fixed slots of a path (jitter, free paths,
// phase); other streams hold draws whose number varies (delta tracking).
__device__ __forceinline__ float rng_u(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t slot,
                                       uint32_t stream = 0u) {
  const uint4 o = philox10(make_uint4(sample, slot >> 2, stream, 0u), (uint32_t)seed, (uint32_t)(seed >> 32) ^ pixel);
  const uint32_t s = slot & 3u;
  const uint32_t w = s == 0 ? o.x : s == 1 ? o.y : s == 2 ? o.z : o.w;
  return (float)(w >> 8) * 0x1p-24f;      // exact: 24-bit integer times a power of two
}

// ---------------------------------------------------------------------------
// Henyey-Greenstein phase function (cos theta between the propagation
// directions before and after scattering; g > 0 forward).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float hg_eval(float g, float cos_t) {
  const float den = 1.0f + g * g - 2.0f * g * cos_t;
  return (1.0f - g * g) / (4.0f * 3.14159265358979f * den * sqrtf(den));
}

// Inverse-CDF sample of cos theta (uniform below |g| = 1e-3), azimuth 2 pi u2,
// rotated into the frame of d by the branch-free basis of Duff et al. (JCGT 2017).
// With s = (1 - g^2) / (1 - g + 2 g u) the inverse CDF is
// cos = (1 + g^2 - s^2) / 2g; its complements are evaluated in the
// cancellation-free products
//   1 - cos = (1 - g)(1 - u)(s + 1 - g) / (1 - g + 2 g u),
//   1 + cos = (1 + g) u (1 + g + s) / (1 - g + 2 g u),
// so sin = sqrt((1 - cos)(1 + cos)) keeps full relative precision near the
// forward and backward peaks.
__device__ __forceinline__ float3 hg_scatter(float g, float u1, float u2, float3 d) {
  float omc, opc;
  if (fabsf(g) < 1e-3f) {
    omc = 2.0f * u1;
    opc = 2.0f - 2.0f * u1;
  } else {
    const float den = 1.0f - g + 2.0f * g * u1;
    const float s = (1.0f - g * g) / den;
    omc = (1.0f - g) * (1.0f - u1) * (s + 1.0f - g) / den;
    opc = (1.0f + g) * u1 * (1.0f + g + s) / den;
  }
  const float ct = omc < opc ? 1.0f - omc : opc - 1.0f;
  const float st = sqrtf(fmaxf(0.0f, omc * opc));
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  const float sgn = copysignf(1.0f, d.z);
  const float a = -1.0f / (sgn + d.z);
  const float b = d.x * d.y * a;
  const float3 b1 = make_float3(1.0f + sgn * d.x * d.x * a, sgn * b, -sgn * d.x);
  const float3 b2 = make_float3(b, sgn + d.y * d.y * a, -d.y);
  float3 w = make_float3(st * cp * b1.x + st * sp * b2.x + ct * d.x,
                         st * cp * b1.y + st * sp * b2.y + ct * d.y,
                         st * cp * b1.z + st * sp * b2.z + ct * d.z);
  const float inv = 1.0f / sqrtf(w.x * w.x + w.y * w.y + w.z * w.z);
  return make_float3(w.x * inv, w.y * inv, w.z * inv);
}

// ---------------------------------------------------------------------------
// Float-float ("double-float") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2, about 44
// significant bits.  Error-free transformations: Knuth's two-sum and the
// fused-multiply-add two-product (Dekker's product with an FMA).
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return ff{a, 0.0f}; }

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  ff r = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(r.hi, __fadd_rn(r.lo, t.lo));
}

// cheaper sum for operands of equal sign (accumulating optical depths)
__device__ __forceinline__ ff ff_add_fast(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// a / b by one correction of the float quotient
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = ff_sub(a, ff_mul_f(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}

__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
__device__ __forceinline__ float ff_float(ff a) { return __fadd_rn(a.hi, a.lo); }

struct ff3 {
  ff x, y, z;
};

// ---------------------------------------------------------------------------
// Host set-up shared by the renderers: camera and medium in grid space.
// ---------------------------------------------------------------------------
struct CamF {
  double eye[3], fwd[3], right[3], up[3];   // camera rays are formed in fp64 (once per path)
  double tanF, aspect;
  int W, H;
};

struct MedF {
  float albedo, g, E, Lenv;
  float sig_hi, sig_lo;                 // extinction per grid unit at density 1, as float-float
  float sun_w[3];                       // unit direction towards the sun
  int max_bounces;
};

CamF camera_setup(const tg_camera& c, const float box_min[3], double cube);
MedF medium_setup(const tg_medium& m, double cube);
bool camera_ok(const tg_camera* c);
// A frame's sample indices [offset, offset + spp) must be non-negative int32
// values: beyond INT32_MAX they would wrap and repeat other samples' streams.
inline bool samples_ok(int32_t spp, int32_t offset) {
  return spp >= 0 && offset >= 0 && (int64_t)offset + spp <= (int64_t)INT32_MAX;
}
bool medium_ok(const tg_medium* m);

}  // namespace tv

struct tg_grid {
  tv::GridImpl impl;
};
