// Cell walker over the regular voxel grid (the comparator of Sec. 4): a 3D DDA
// in the manner of Amanatides & Woo.  The exit parameter of a voxel along axis a
// is computed from the wall itself, ((i_a + [d_a > 0]) / n - o_a) / d_a, rather
// than by accumulating increments, so long walks do not drift.
#pragma once
#include "estimator.cuh"

namespace tv {

struct VoxParams {
  const float* rho;   // density[nz][ny][nx]
  int nx, ny, nz;
  float inv_n;        // voxel size in cubes (1 / voxels per cube edge)
  float n_f;          // voxels per cube edge
  int C[3];           // cubes per axis
};

struct VoxelWalker {
  using Params = VoxParams;
  static constexpr int NDIR = 4;            // direction-table entries: 1/d.x, 1/d.y, 1/d.z (NaN if 0), sign bits
  const VoxParams& P;
  double* tab;        // 8-byte slots: o.x, o.y, o.z as float-float pairs, then 1/d.x, 1/d.y, 1/d.z
  int ix, iy, iz;
  int axis;           // pending step axis
  int dir;            // bit a: d_a > 0, bit 3 + a: d_a < 0

  static size_t smem_bytes() { return sizeof(double) * 6 * EST_BLOCK; }

  __device__ VoxelWalker(const VoxParams& p, double* smem)
      : P(p), tab(smem + threadIdx.x), ix(0), iy(0), iz(0), axis(0), dir(0) {}

  __device__ __forceinline__ float& ftab(int q) { return *reinterpret_cast<float*>(tab + q * EST_BLOCK); }
  __device__ __forceinline__ float ftab(int q) const { return *reinterpret_cast<const float*>(tab + q * EST_BLOCK); }
  __device__ __forceinline__ float2& pair(int q) { return *reinterpret_cast<float2*>(tab + q * EST_BLOCK); }
  __device__ __forceinline__ float2 pair(int q) const { return *reinterpret_cast<const float2*>(tab + q * EST_BLOCK); }

  __device__ bool intersect(float3 o, float3 d, float* t_in) const { return box_intersect(P.C, o, d, t_in); }

  __device__ bool locate(float3 p) {
    const float q[3] = {p.x * P.n_f, p.y * P.n_f, p.z * P.n_f};
    const int lim[3] = {P.nx - 1, P.ny - 1, P.nz - 1};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int v = (int)floorf(q[a]);
      idx[a] = v < 0 ? 0 : (v > lim[a] ? lim[a] : v);
    }
    ix = idx[0]; iy = idx[1]; iz = idx[2];
    return true;
  }

  __device__ __forceinline__ void dir_table(const ff3& dd, float inv[4]) const {
    const float d[3] = {ff_float(dd.x), ff_float(dd.y), ff_float(dd.z)};
    uint32_t bits = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      inv[a] = d[a] != 0.f ? __frcp_rn(d[a]) : __int_as_float(0x7FFFFFFF);
      bits |= (d[a] > 0.f ? 1u : 0u) << a;
      bits |= (d[a] < 0.f ? 1u : 0u) << (3 + a);
    }
    inv[3] = __int_as_float((int)bits);
  }

  __device__ void begin(const ff3& o, const float* inv) {
    pair(0) = make_float2(o.x.hi, o.x.lo);
    pair(1) = make_float2(o.y.hi, o.y.lo);
    pair(2) = make_float2(o.z.hi, o.z.lo);
    ftab(3) = inv[0]; ftab(4) = inv[1]; ftab(5) = inv[2];
    dir = __float_as_int(inv[3]);
  }

  __device__ __forceinline__ float density() const {
    return __ldg(P.rho + ((size_t)iz * P.ny + iy) * P.nx + ix);
  }

  // exit parameter of axis a from the wall itself, ((i_a + [d_a > 0]) / n - o_a) / d_a,
  // with the origin as a float-float pair
  __device__ __forceinline__ float wall(int a, int i) const {
    const float w = (float)(i + ((dir >> a) & 1)) * P.inv_n;     // exact
    const float2 o = pair(a);
    return __fmul_rn(__fsub_rn(__fsub_rn(w, o.x), o.y), ftab(3 + a));   // NaN when d_a = 0
  }

  __device__ __forceinline__ Hop hop(float t) {
    const float tx = wall(0, ix), ty = wall(1, iy), tz = wall(2, iz);
    float best = INFINITY;
    int ax = 0;
    if (tx < best) { best = tx; ax = 0; }
    if (ty < best) { best = ty; ax = 1; }
    if (tz < best) { best = tz; ax = 2; }
    axis = ax;
    Hop h;
    h.ok = best < INFINITY;
    h.texit = fmaxf(best, t);
    h.rho = density();
    return h;
  }

  __device__ __forceinline__ bool advance() {
    const int s = ((dir >> axis) & 1) ? 1 : -1;
    if (axis == 0) { ix += s; return ix >= 0 && ix < P.nx; }
    if (axis == 1) { iy += s; return iy >= 0 && iy < P.ny; }
    iz += s;
    return iz >= 0 && iz < P.nz;
  }
  __device__ __forceinline__ int save() const { return (iz * P.ny + iy) * P.nx + ix; }
  __device__ __forceinline__ void restore(int c) { ix = c % P.nx; iy = (c / P.nx) % P.ny; iz = c / (P.nx * P.ny); }
  __device__ __forceinline__ int cell() const { return (iz * P.ny + iy) * P.nx + ix; }
};

}  // namespace tv
