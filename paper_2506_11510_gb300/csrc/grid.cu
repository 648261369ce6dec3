// tg_grid_export / tg_grid_import: between the packed 32-byte records and the
// plain per-cell arrays of the C ABI.
#include <cuda_fp16.h>

#include "walk_tet.cuh"

namespace tv {

__device__ __forceinline__ int internal_to_nid(uint32_t id) { return (int)(id & 15u) + ((id >> 4) ? 9 : 0); }

__global__ void k_export(const uint4* __restrict__ rec, long long n, int K, int fmt, int32_t* nbr, uint8_t* nid,
                         float* plane, float* density) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 a = rec[2 * i], b = rec[2 * i + 1];
  const uint32_t link[4] = {a.x, a.y, a.z, a.w};
  const int c[4] = {sext24(b.x), sext24((b.x >> 24) | (b.y << 8)), sext24((b.y >> 16) | (b.z << 16)),
                    sext24(b.z >> 8)};
  const float s = ldexpf(1.0f, -K);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const uint32_t j = link[f] & NO_NBR;
    if (nbr) nbr[4 * i + f] = j == NO_NBR ? -1 : (int32_t)j;
    if (nid) nid[4 * i + f] = (uint8_t)internal_to_nid(link[f] >> 27);
    if (plane) plane[4 * i + f] = (float)c[f] * s;
  }
  if (density) {
    float r;
    if (fmt == TG_DENSITY_BF16) r = decode_density<TG_DENSITY_BF16>(b.w);
    else if (fmt == TG_DENSITY_FP16) r = decode_density<TG_DENSITY_FP16>(b.w);
    else r = decode_density<TG_DENSITY_FP32>(b.w);
    density[i] = r;
  }
}

__global__ void k_import(uint4* __restrict__ rec, long long n, int K, int fmt, const int32_t* nbr, const uint8_t* nid,
                         const float* plane, const float* density, int* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t link[4];
  int c[4];
  const float S = ldexpf(1.0f, K);
  for (int f = 0; f < 4; ++f) {
    const int j = nbr[4 * i + f];
    const int id = nid[4 * i + f];
    if (j < -1 || j >= n || id < 0 || id >= 18) { atomicExch(err, 1); return; }
    const uint32_t internal = id < 9 ? (uint32_t)id : (uint32_t)(id - 9) | 16u;
    link[f] = (j < 0 ? NO_NBR : (uint32_t)j) | (internal << 27);
    const float v = plane[4 * i + f] * S;
    c[f] = (int)v;
    if ((float)c[f] != v || c[f] >= (1 << 23) || c[f] < -(1 << 23)) { atomicExch(err, 1); return; }
  }
  uint32_t w;
  const float r = density[i];
  if (fmt == TG_DENSITY_BF16) {
    const uint32_t u = __float_as_uint(r);
    w = ((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16) << 16;
  } else if (fmt == TG_DENSITY_FP16) {
    w = (uint32_t)__half_as_ushort(__float2half_rn(r));
  } else {
    w = __float_as_uint(r);
  }
  const uint32_t m = 0xFFFFFFu;
  rec[2 * i] = make_uint4(link[0], link[1], link[2], link[3]);
  rec[2 * i + 1] = make_uint4(((uint32_t)c[0] & m) | ((uint32_t)c[1] << 24), (((uint32_t)c[1] & m) >> 8) | ((uint32_t)c[2] << 16),
                              (((uint32_t)c[2] & m) >> 16) | ((uint32_t)c[3] << 8), w);
}

__global__ void k_widen(const uint8_t* __restrict__ a, int32_t* __restrict__ b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

__global__ void k_max_depth(const unsigned long long* __restrict__ codes, long long n, int* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(out, (int)(codes[i] & 63ull));
}

}  // namespace tv

using namespace tv;

extern "C" {

int tg_grid_export(const tg_grid* g, uint64_t* codes, int32_t* verts, int32_t* tag, int32_t* nbr, uint8_t* nid,
                   float* plane, float* density, float* majorant, uint32_t* count, uint64_t* sum, uint32_t* qmin,
                   uint32_t* qmax, void* cuda_stream) {
  if (!g) return TG_EINVAL;
  const GridImpl& G = g->impl;
  if ((verts && !G.verts) || (tag && !G.tag) || (majorant && !G.majorant) || (count && !G.count) ||
      (sum && !G.sum) || (qmin && !G.qmin) || (qmax && !G.qmax))
    return TG_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t n = (size_t)G.n;
    if (n == 0) return TG_OK;
    if (codes) TV_CUDA(cudaMemcpyAsync(codes, G.codes, n * 8, cudaMemcpyDeviceToDevice, st));
    if (verts) TV_CUDA(cudaMemcpyAsync(verts, G.verts, n * 48, cudaMemcpyDeviceToDevice, st));
    if (majorant) TV_CUDA(cudaMemcpyAsync(majorant, G.majorant, n * 4, cudaMemcpyDeviceToDevice, st));
    if (count) TV_CUDA(cudaMemcpyAsync(count, G.count, n * 4, cudaMemcpyDeviceToDevice, st));
    if (sum) TV_CUDA(cudaMemcpyAsync(sum, G.sum, n * 8, cudaMemcpyDeviceToDevice, st));
    if (qmin) TV_CUDA(cudaMemcpyAsync(qmin, G.qmin, n * 4, cudaMemcpyDeviceToDevice, st));
    if (qmax) TV_CUDA(cudaMemcpyAsync(qmax, G.qmax, n * 4, cudaMemcpyDeviceToDevice, st));
    if (nbr || nid || plane || density) {
      const unsigned blocks = (unsigned)((n + 255) / 256);
      k_export<<<blocks, 256, 0, st>>>(G.rec, (long long)n, G.K, G.fmt, nbr, nid, plane, density);
      TV_LAUNCH();
    }
    if (tag) {
      k_widen<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G.tag, tag, (long long)n);
      TV_LAUNCH();
    }
  } catch (const Error& e) {
    return e.code;
  }
  return TG_OK;
}

int tg_grid_import(const tg_volume_desc* vol, int32_t K, int64_t num_tets, const uint64_t* codes, const int32_t* nbr,
                   const uint8_t* nid, const float* plane, const float* density, int32_t density_format,
                   void* cuda_stream, tg_grid** out) {
  if (!vol || !out || num_tets < 0 || num_tets > MAX_TETS || K < 1 || K > 20 || density_format < 0 ||
      density_format > 2 || (num_tets > 0 && (!codes || !nbr || !nid || !plane || !density)))
    return TG_EINVAL;
  if (vol->nx <= 0 || vol->ny <= 0 || vol->nz <= 0 || !(vol->voxel_size > 0)) return TG_EINVAL;
  tg_grid* g = new (std::nothrow) tg_grid();
  if (!g) return TG_ENOMEM;
  try {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GridImpl& G = g->impl;
    TV_CUDA(cudaGetDevice(&G.device));
    int n = 1;
    while (vol->nx % (2 * n) == 0 && vol->ny % (2 * n) == 0 && vol->nz % (2 * n) == 0 && n < (1 << 18)) n *= 2;
    G.n_per_cube = n;
    G.C[0] = vol->nx / n; G.C[1] = vol->ny / n; G.C[2] = vol->nz / n;
    G.nvox[0] = vol->nx; G.nvox[1] = vol->ny; G.nvox[2] = vol->nz;
    for (int a = 0; a < 3; ++a) G.box_min[a] = vol->box_min[a];
    G.voxel_size = vol->voxel_size;
    G.cube = (double)vol->voxel_size * (double)n;
    G.K = K;
    G.fmt = density_format;
    G.n = num_tets;
    DevBuf<uint4> rec(2 * (size_t)num_tets + 2);
    DevBuf<unsigned long long> cd((size_t)num_tets + 1), scratch(4);
    DevBuf<int> err(2);
    TV_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(int), st));
    TV_CUDA(cudaMemsetAsync(scratch.p, 0, 4 * sizeof(unsigned long long), st));
    if (num_tets > 0) {
      TV_CUDA(cudaMemcpyAsync(cd.p, codes, (size_t)num_tets * 8, cudaMemcpyDeviceToDevice, st));
      k_import<<<(unsigned)((num_tets + 255) / 256), 256, 0, st>>>(rec.p, num_tets, K, density_format, nbr, nid,
                                                                   plane, density, err.p);
      TV_LAUNCH();
      // the deepest level present bounds the point-location descent
      k_max_depth<<<(unsigned)((num_tets + 255) / 256), 256, 0, st>>>(cd.p, num_tets, err.p + 1);
      TV_LAUNCH();
    }
    int herr[2] = {0, 0};
    TV_CUDA(cudaMemcpyAsync(herr, err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    TV_CUDA(cudaStreamSynchronize(st));
    if (herr[0]) throw Error{TG_EINVAL};
    G.max_depth = herr[1];
    G.rec = rec.release();
    G.codes = cd.release();
    G.scratch = scratch.release();
    build_locator(G, st);
    TV_CUDA(cudaStreamSynchronize(st));
  } catch (const Error& e) {
    delete g;
    return e.code;
  }
  *out = g;
  return TG_OK;
}

}  // extern "C"
