// leb_build: the adaptive conforming grid of Sec. 2 on the GPU.
//
// Leaves live in structure-of-arrays form.  While many of them split, each
// round rebuilds them by a stable compaction in which a split leaf is replaced,
// in place, by its two children (bit 0 then bit 1); starting from the roots in
// code order this keeps them in depth-first order of their LEB codes.  Once few
// split (the closure's last rounds), the first child takes its parent's slot
// and the second is appended, so a round touches only what it splits; after
// the last round the appended run is sorted and merged with the ordered one.
//
// Round: (1) mark = criterion || hanging vertex (one of the six edge
// midpoints is a vertex of the grid, found in an open-addressing hash set of
// packed vertex coordinates, behind a Bloom filter that stays in L2); (2) exclusive scan of the marks gives
// every split leaf its rank; (3) split, inserting the new vertices; (4) the
// density statistics of the new leaves are gathered by warps over chunks of
// their voxel bounding boxes (exact integer inside tests against the four face
// planes), then the criterion is evaluated once per new leaf.
// Finalize: faces are matched by a radix sort of their vertex sums (verified
// against the full vertex triples), then the 32-byte records are packed.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace tv {

namespace {

constexpr unsigned long long EMPTY = ~0ull;
constexpr int TPB = 256;
constexpr int ROWS = 32;            // voxel-box rows per warp work item of the statistics pass (one per lane)

struct Geo {
  int nx, ny, nz, n, m, K, max_depth;
  int C[3];
  int h;                            // voxel i has its centre at (2i + 1) h, units of 2^-K cube
};

struct CamD {
  int on;
  double eye[3], f[3], r[3], u[3];
  double tanF, tanX, near_g, thr;
};

// The camera of criterion 2 rounded to float, with the magnitudes the error
// bounds of the float evaluation need (see camera_allows_f32).
struct CamF {
  float eye[3], f[3], r[3], u[3];
  float tanF, tanX, near_g, thr;
  float ef, er, eu;                 // sum_a |f_a| |eye_a|, and the same for r and u
};

struct Crit {
  Geo g;
  CamD cam;
  CamF camf;
  int var_on;
  unsigned long long theta_q16;
};

struct LeafPtrs {
  int4* v;                          // 3 int4 per leaf: x0 x1 x2 x3
  unsigned long long* code;
  uint8_t* tag;
  uint32_t *cnt, *mn, *mx;
  unsigned long long* sum;
  uint8_t* crit;
};

// Statistics of the interior nodes of the LEB tree (each leaf that is split
// leaves its code and statistics here), kept with the grid for rebuilds.
struct NodePtrs {
  unsigned long long* code;
  unsigned long long* sum;
  uint32_t *cnt, *mn, *mx;
};

struct Leaves {
  DevBuf<int4> v;
  DevBuf<unsigned long long> code, sum;
  DevBuf<uint8_t> tag, crit;
  DevBuf<uint32_t> cnt, mn, mx;
  size_t cap = 0;
  void ensure(size_t n) {
    if (n <= cap) return;
    size_t c = std::max<size_t>(2 * n, 1024);
    v.alloc(3 * c); code.alloc(c); sum.alloc(c); tag.alloc(c); crit.alloc(c); cnt.alloc(c); mn.alloc(c); mx.alloc(c);
    cap = c;
  }
  // room for n leaves, keeping the first `used` (geometric growth)
  void grow(size_t n, size_t used, cudaStream_t st) {
    if (n <= cap) return;
    Leaves g;
    g.ensure(n);
    if (used) {
      TV_CUDA(cudaMemcpyAsync(g.v.p, v.p, used * 3 * sizeof(int4), cudaMemcpyDeviceToDevice, st));
      TV_CUDA(cudaMemcpyAsync(g.code.p, code.p, used * 8, cudaMemcpyDeviceToDevice, st));
      TV_CUDA(cudaMemcpyAsync(g.sum.p, sum.p, used * 8, cudaMemcpyDeviceToDevice, st));
      TV_CUDA(cudaMemcpyAsync(g.tag.p, tag.p, used, cudaMemcpyDeviceToDevice, st));
      TV_CUDA(cudaMemcpyAsync(g.crit.p, crit.p, used, cudaMemcpyDeviceToDevice, st));
      TV_CUDA(cudaMemcpyAsync(g.cnt.p, cnt.p, used * 4, cudaMemcpyDeviceToDevice, st));
      TV_CUDA(cudaMemcpyAsync(g.mn.p, mn.p, used * 4, cudaMemcpyDeviceToDevice, st));
      TV_CUDA(cudaMemcpyAsync(g.mx.p, mx.p, used * 4, cudaMemcpyDeviceToDevice, st));
    }
    *this = std::move(g);            // the old arrays are given back on the stream, after the copies
  }
  LeafPtrs ptrs() { return LeafPtrs{v.p, code.p, tag.p, cnt.p, mn.p, mx.p, sum.p, crit.p}; }
};


__device__ __forceinline__ unsigned long long mix(unsigned long long k) {
  k ^= k >> 31; k *= 0x7FB5D329728EA185ull;
  k ^= k >> 27; k *= 0x81DADEF4BC2DD44Dull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ unsigned long long pack3(long long x, long long y, long long z) {
  return (unsigned long long)x | ((unsigned long long)y << 21) | ((unsigned long long)z << 42);
}

// Insert-if-absent into an open-addressing set; returns the slot, or -1 after
// probing every slot without success (a full table: the caller flags an error).
__device__ __forceinline__ long long hset_insert(unsigned long long* keys, unsigned long long mask,
                                                 unsigned long long key, unsigned long long* count) {
  unsigned long long s = mix(key) & mask;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev = atomicCAS(keys + s, EMPTY, key);
    if (prev == EMPTY) { if (count) atomicAdd(count, 1ull); return (long long)s; }
    if (prev == key) return (long long)s;
    s = (s + 1) & mask;
  }
  return -1;
}

// Slot of key, or -1 when absent (an empty slot, or every slot probed).
__device__ __forceinline__ long long hset_find(const unsigned long long* keys, unsigned long long mask,
                                               unsigned long long key) {
  unsigned long long s = mix(key) & mask;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    const unsigned long long k = keys[s];
    if (k == key) return (long long)s;
    if (k == EMPTY) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}

// A blocked Bloom filter over the vertex set (two bits of one 32-bit word per
// key, the word and bits from the key's hash): a clear bit proves a key absent
// with one read of a filter small enough to stay in L2; a set pair is confirmed
// in the hash set.
struct Bloom {
  uint32_t* w;
  unsigned long long mask;          // words - 1 (a power of two)
};
__device__ __forceinline__ void bloom_bits(const Bloom& b, unsigned long long key, unsigned long long* word,
                                           uint32_t* bits) {
  const unsigned long long h = mix(key ^ 0x9E3779B97F4A7C15ull);
  *word = h & b.mask;
  *bits = (1u << ((h >> 40) & 31u)) | (1u << ((h >> 45) & 31u));
}
__device__ __forceinline__ void bloom_add(const Bloom& b, unsigned long long key) {
  unsigned long long w;
  uint32_t m;
  bloom_bits(b, key, &w, &m);
  atomicOr(b.w + w, m);
}
__device__ __forceinline__ bool bloom_may_hold(const Bloom& b, unsigned long long key) {
  unsigned long long w;
  uint32_t m;
  bloom_bits(b, key, &w, &m);
  return (__ldg(b.w + w) & m) == m;
}

__device__ __forceinline__ void load_tet(const int4* v, long long i, int x[4][3]) {
  const int4 a = v[3 * i], b = v[3 * i + 1], c = v[3 * i + 2];
  x[0][0] = a.x; x[0][1] = a.y; x[0][2] = a.z; x[1][0] = a.w;
  x[1][1] = b.x; x[1][2] = b.y; x[2][0] = b.z; x[2][1] = b.w;
  x[2][2] = c.x; x[3][0] = c.y; x[3][1] = c.z; x[3][2] = c.w;
}

__device__ __forceinline__ void store_tet(int4* v, long long i, const int x[4][3]) {
  v[3 * i] = make_int4(x[0][0], x[0][1], x[0][2], x[1][0]);
  v[3 * i + 1] = make_int4(x[1][1], x[1][2], x[2][0], x[2][1]);
  v[3 * i + 2] = make_int4(x[2][2], x[3][0], x[3][1], x[3][2]);
}

// Outward face plane of face f (opposite vertex f) as n . p <= rhs with n in
// {0, +-1}^3: every LEB face is parallel to one of 9 planes.  Returns false if
// the face normal is not of that form.
__device__ __forceinline__ bool face_plane(const int x[4][3], int f, int nrm[3], long long* rhs) {
  const int a = (f + 1) & 3, b = (f + 2) & 3, c = (f + 3) & 3;
  long long u[3], v[3], w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    u[k] = (long long)x[b][k] - x[a][k];
    v[k] = (long long)x[c][k] - x[a][k];
    w[k] = (long long)x[f][k] - x[a][k];
  }
  long long n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  if (n[0] * w[0] + n[1] * w[1] + n[2] * w[2] > 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
  const long long m = max(max(llabs(n[0]), llabs(n[1])), llabs(n[2]));
  bool ok = m > 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    nrm[k] = (n[k] > 0) - (n[k] < 0);
    ok = ok && (n[k] == 0 || llabs(n[k]) == m);
  }
  *rhs = (long long)nrm[0] * x[a][0] + (long long)nrm[1] * x[a][1] + (long long)nrm[2] * x[a][2];
  return ok;
}

// orientation id (internal encoding p | s << 4) of a canonical outward normal
__device__ __forceinline__ int orient_id(const int n[3]) {
  // P = {x, y, z, x+y, x-y, y+z, y-z, x+z, x-z}
  const int P[9][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
                       {0, 1, 1}, {0, 1, -1}, {1, 0, 1}, {1, 0, -1}};
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    if (n[0] == P[p][0] && n[1] == P[p][1] && n[2] == P[p][2]) return p;
    if (n[0] == -P[p][0] && n[1] == -P[p][1] && n[2] == -P[p][2]) return p | 16;
  }
  return -1;
}

__device__ __forceinline__ int p9_dot(int p, const int v[3]) {
  switch (p) {
    case 0: return v[0];
    case 1: return v[1];
    case 2: return v[2];
    case 3: return v[0] + v[1];
    case 4: return v[0] - v[1];
    case 5: return v[1] + v[2];
    case 6: return v[1] - v[2];
    case 7: return v[0] + v[2];
    default: return v[0] - v[2];
  }
}

// ---------------------------------------------------------------------------
// A1: quantise density to q = round(rho 2^24) in [0, 2^24]
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t quantize1(float rho) {
  const float v = rho * 16777216.0f;
  if (!(v > 0.0f)) return 0u;
  if (v >= 16777216.0f) return 16777216u;
  return (uint32_t)rintf(v);
}

// rho may be device memory or page-locked host memory the device addresses
// directly (then each element crosses the host link exactly once, here): 16-byte
// loads when the volume is 16-byte aligned, one element at a time otherwise.
__global__ void k_quantize(const float* __restrict__ rho, uint32_t* __restrict__ q, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long done = 0;
  if ((reinterpret_cast<uintptr_t>(rho) & 15u) == 0 && (reinterpret_cast<uintptr_t>(q) & 15u) == 0) {
    const long long n4 = n / 4;
    const float4* r4 = reinterpret_cast<const float4*>(rho);
    uint4* q4 = reinterpret_cast<uint4*>(q);
    for (long long i = i0; i < n4; i += stride) {
      const float4 v = r4[i];
      q4[i] = make_uint4(quantize1(v.x), quantize1(v.y), quantize1(v.z), quantize1(v.w));
    }
    done = 4 * n4;
  }
  for (long long i = done + i0; i < n; i += stride) q[i] = quantize1(rho[i]);
}

// A2: six Kuhn tetrahedra per cube, tag 3, in root-id order
__global__ void k_roots(LeafPtrs L, Geo g, int nroots) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nroots) return;
  const int perm = r % 6, c = r / 6;
  const int cube[3] = {c % g.C[0], (c / g.C[0]) % g.C[1], c / (g.C[0] * g.C[1])};
  const int ax0 = perm < 2 ? 0 : (perm < 4 ? 1 : 2);
  const int ax1 = (perm == 0 || perm == 5) ? 1 : ((perm == 1 || perm == 3) ? 2 : 0);
  const int S = 1 << g.K;
  int x[4][3];
  for (int a = 0; a < 3; ++a) {
    x[0][a] = cube[a] * S;
    x[1][a] = x[0][a] + (a == ax0 ? S : 0);
    x[2][a] = x[1][a] + (a == ax1 ? S : 0);
    x[3][a] = x[0][a] + S;
  }
  store_tet(L.v, r, x);
  L.code[r] = (unsigned long long)r << 56;
  L.tag[r] = 3;
}

__global__ void k_insert_vertices(const int4* v, long long n, unsigned long long* keys, unsigned long long mask,
                                  Bloom bloom, unsigned long long* count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x[4][3];
  load_tet(v, i, x);
  for (int k = 0; k < 4; ++k) {
    const unsigned long long key = pack3(x[k][0], x[k][1], x[k][2]);
    if (hset_insert(keys, mask, key, count) < 0) atomicAdd(count + 3, 1ull);
    bloom_add(bloom, key);
  }
}

// the vertex set into a larger table, and its filter into a larger filter
__global__ void k_rehash(const unsigned long long* old, long long oldcap, unsigned long long* keys,
                         unsigned long long mask, Bloom bloom, unsigned long long* fail) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= oldcap) return;
  const unsigned long long k = old[i];
  if (k == EMPTY) return;
  if (hset_insert(keys, mask, k, nullptr) < 0) atomicAdd(fail, 1ull);
  bloom_add(bloom, k);
}

// voxel index range of the centres inside [lo, hi] (units of 2^-K) along one axis
__device__ __forceinline__ void voxel_range(int lo, int hi, int h, int dim, int* a, int* b) {
  // centre (2i + 1) h in [lo, hi]  <=>  ceil((lo - h) / 2h) <= i <= floor((hi - h) / 2h); 2h = 2^s, and
  // coordinates are below 2^20, so both are exact shifts of 32-bit values
  const int s = __ffs(h);                           // log2(2h)
  int ilo = -((h - lo) >> s);
  int ihi = (hi - h) >> s;
  if (ilo < 0) ilo = 0;
  if (ihi > dim - 1) ihi = dim - 1;
  *a = ilo;
  *b = ihi;
}

__device__ __forceinline__ void tet_box(const int x[4][3], const Geo& g, int lo[3], int hi[3]) {
  const int dims[3] = {g.nx, g.ny, g.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int mn = x[0][a], mx = x[0][a];
#pragma unroll
    for (int k = 1; k < 4; ++k) { mn = min(mn, x[k][a]); mx = max(mx, x[k][a]); }
    voxel_range(mn, mx, g.h, dims[a], &lo[a], &hi[a]);
  }
}

// Voxel box of a leaf: the voxels whose centres lie in the tet's bounding box,
// or (BOX) every voxel whose cell touches the bounding box.
template <bool BOX>
__device__ __forceinline__ void leaf_box(const int x[4][3], const Geo& g, int lo[3], int hi[3]) {
  if (!BOX) { tet_box(x, g, lo, hi); return; }
  const int dims[3] = {g.nx, g.ny, g.nz};
  const int w = 2 * g.h;                           // voxel edge in vertex units
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int mn = x[0][a], mx = x[0][a];
#pragma unroll
    for (int k = 1; k < 4; ++k) { mn = min(mn, x[k][a]); mx = max(mx, x[k][a]); }
    lo[a] = max(0, mn / w);                        // coordinates are non-negative
    hi[a] = min(dims[a] - 1, mx / w);
  }
}

// A box of at most 32 rows of at most 32 voxels: one thread scans it.
__device__ __forceinline__ bool small_box(const int lo[3], const int hi[3]) {
  return (long long)(hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1) <= 32 && hi[0] - lo[0] < 32;
}

// The voxel centres P = (2i+1, 2j+1, 2k+1) h of row (j, k) that lie in the closed
// tet form an interval [xa, xb] of i (xb < xa: none), found exactly from the four
// faces n . P <= rhs (n in {0, +-1}^3, h = 2^hs): with F = floor(B / h),
// B = rhs - n_y (2j+1) h - n_z (2k+1) h, a face with n_x = 1 gives
// i <= floor((F - 1) / 2), n_x = -1 gives i >= ceil((-F - 1) / 2), and n_x = 0
// keeps the row iff B >= 0.
// (Coordinates are at most 2^19 (the build refuses larger grids), so |rhs| < 2^21 and
// every term fits a 32-bit integer.)
__device__ __forceinline__ void row_interval(const int nrm[4][3], const int rhs[4], int hs, int jj, int kk,
                                             int x0, int x1, int* xa, int* xb) {
  const int Py = (2 * jj + 1) << hs, Pz = (2 * kk + 1) << hs;
  int a = x0, b = x1;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int B = rhs[f] - nrm[f][1] * Py - nrm[f][2] * Pz;
    const int F = B >> hs;                       // floor(B / h)
    if (nrm[f][0] > 0) b = min(b, (F - 1) >> 1);
    else if (nrm[f][0] < 0) a = max(a, -((F + 1) >> 1));
    else if (B < 0) b = a - 1;
  }
  *xa = a;
  *xb = max(b, a - 1);
}

// The four outward face planes of a tet as n . p <= rhs (32-bit rhs, see above).
__device__ __forceinline__ void face_planes32(const int x[4][3], int nrm[4][3], int rhs[4]) {
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    long long r = 0;
    face_plane(x, f, nrm[f], &r);
    rhs[f] = (int)r;
  }
}

// Statistics of a leaf whose box is small (small_box), by one thread (QUAD: rows
// start on 16-byte boundaries, and each row's voxels are read as aligned 16-byte quads).
template <bool BOX, bool QUAD>
__device__ __forceinline__ void small_box_stats(const int lo[3], const int hi[3], const int nrm[4][3],
                                                const int rhs[4], const uint32_t* __restrict__ q, const Geo& g,
                                                uint32_t& cnt, unsigned long long& sum, uint32_t& mn, uint32_t& mx) {
  const int hs = g.K - g.m - 1;
  cnt = 0; sum = 0; mn = 0xFFFFFFFFu; mx = 0;
  for (int kk = lo[2]; kk <= hi[2]; ++kk)
    for (int jj = lo[1]; jj <= hi[1]; ++jj) {
      int xa = lo[0], xb = hi[0];
      if (!BOX) row_interval(nrm, rhs, hs, jj, kk, lo[0], hi[0], &xa, &xb);
      const uint32_t* row = q + ((size_t)kk * g.ny + jj) * g.nx;
      if (QUAD) {
        for (int qd = xa >> 2; qd <= (xb >> 2) && xa <= xb; ++qd) {
          const uint4 v4 = __ldg(reinterpret_cast<const uint4*>(row) + qd);
          const uint32_t w[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int xx = 4 * qd + e;
            if (xx >= xa && xx <= xb) { ++cnt; sum += w[e]; mn = min(mn, w[e]); mx = max(mx, w[e]); }
          }
        }
      } else {
        for (int ii = xa; ii <= xb; ++ii) {
          const uint32_t v = __ldg(row + ii);
          ++cnt; sum += v; mn = min(mn, v); mx = max(mx, v);
        }
      }
    }
}

// What the work items of one leaf share (written once per leaf by pass 1, read
// by every work item of pass 2): its voxel box, its four face planes n . p <= rhs
// (n in {0, +-1}^3, two bits per component holding n + 1) and its index.
struct __align__(16) ScanDesc {
  int lo[3], hi[3];
  uint32_t nrm;
  int leaf;
  int rhs[4];
};

// A3 statistics, pass 1: the statistics of a new leaf with a small voxel box
// (by this thread), or the work items of a larger one (ROWS rows of its box
// each) and what they share, its statistics reset for pass 2
template <bool BOX, bool QUAD>
__global__ void k_stats_prep(LeafPtrs L, const long long* list, long long m, Geo g, unsigned long long* chunks,
                             ScanDesc* desc, const uint32_t* __restrict__ q) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const long long i = list ? list[j] : j;
  int x[4][3], lo[3], hi[3];
  load_tet(L.v, i, x);
  leaf_box<BOX>(x, g, lo, hi);
  const bool empty = !(hi[0] >= lo[0] && hi[1] >= lo[1] && hi[2] >= lo[2]);
  const bool small = !empty && small_box(lo, hi);
  int nrm[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, rhs[4] = {0, 0, 0, 0};
  if (!BOX && !empty) face_planes32(x, nrm, rhs);
  if (empty || small) {
    chunks[j] = 0;
    uint32_t cnt = 0, mn = 0xFFFFFFFFu, mx = 0;
    unsigned long long sum = 0;
    if (small) small_box_stats<BOX, QUAD>(lo, hi, nrm, rhs, q, g, cnt, sum, mn, mx);
    L.cnt[i] = cnt; L.sum[i] = sum; L.mn[i] = mn; L.mx[i] = mx;
    return;
  }
  const long long rows = (long long)(hi[1] - lo[1] + 1) * (long long)(hi[2] - lo[2] + 1);
  chunks[j] = (unsigned long long)((rows + ROWS - 1) / ROWS);
  L.cnt[i] = 0; L.sum[i] = 0; L.mn[i] = 0xFFFFFFFFu; L.mx[i] = 0;
  ScanDesc d;
#pragma unroll
  for (int a = 0; a < 3; ++a) { d.lo[a] = lo[a]; d.hi[a] = hi[a]; }
  d.nrm = 0;
  d.leaf = (int)i;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    d.rhs[f] = rhs[f];
#pragma unroll
    for (int a = 0; a < 3; ++a) d.nrm |= (uint32_t)(nrm[f][a] + 1) << (2 * (3 * f + a));
  }
  desc[j] = d;
}

// A3 statistics, between the passes: the leaf (position in the scan list) that
// owns each work item, so that a work item finds its leaf with one load.
__global__ void k_chunk_owner(const unsigned long long* __restrict__ chunk_off, long long m, int* __restrict__ owner) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const unsigned long long c1 = chunk_off[j + 1];
  for (unsigned long long c = chunk_off[j]; c < c1; ++c) owner[c] = (int)j;
}

// Accumulate the voxels [a + lane + 32 s, b] of one row (the warp reads them along x).
__device__ __forceinline__ void row_tail(const uint32_t* __restrict__ row, int a, int b, unsigned lane, uint32_t& cnt,
                                         unsigned long long& sum, uint32_t& mn, uint32_t& mx) {
  for (int ii = a + (int)lane; ii <= b; ii += 32) {
    const uint32_t v = __ldg(row + ii);
    ++cnt; sum += v; mn = min(mn, v); mx = max(mx, v);
  }
}

// A3 statistics, pass 2 (leaves with larger boxes): one warp per ROWS rows
// (along x) of a leaf's voxel box, one row interval per lane (row_interval), so
// only the voxels inside are read: by the whole warp along the rows when the box
// is at least 32 voxels wide (coalesced; the first 32 voxels of four rows are
// loaded together), else by each lane along its row.
template <bool BOX, bool QUAD>
__global__ void __launch_bounds__(TPB) k_stats_scan(LeafPtrs L, const ScanDesc* __restrict__ desc,
                                                    const unsigned long long* chunk_off, const int* __restrict__ owner,
                                                    unsigned long long total, const uint32_t* __restrict__ q, Geo g) {
  const unsigned lane = threadIdx.x & 31u;
  const long long warps = (long long)gridDim.x * (TPB / 32);
  const int hs = g.K - g.m - 1;                     // h = 2^hs
  for (long long c = (long long)blockIdx.x * (TPB / 32) + (threadIdx.x >> 5); c < (long long)total; c += warps) {
    const long long j = owner[c];                   // chunk_off[j] <= c < chunk_off[j + 1]
    const ScanDesc& D = desc[j];
    const long long i = D.leaf;
    const int lo[3] = {D.lo[0], D.lo[1], D.lo[2]}, hi[3] = {D.hi[0], D.hi[1], D.hi[2]};
    int nrm[4][3];
    int rhs[4];
    if (!BOX) {
      const uint32_t nb = D.nrm;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        rhs[f] = D.rhs[f];
#pragma unroll
        for (int a = 0; a < 3; ++a) nrm[f][a] = (int)((nb >> (2 * (3 * f + a))) & 3u) - 1;
      }
    }
    const long long wy = hi[1] - lo[1] + 1;
    const long long rows = wy * (hi[2] - lo[2] + 1);
    const long long r = ((long long)c - (long long)chunk_off[j]) * ROWS + lane;
    uint32_t cnt = 0, mn = 0xFFFFFFFFu, mx = 0;
    unsigned long long sum = 0;
    int xa = 0, xb = -1;
    long long rowoff = 0;
    if (r < rows) {
      const int jj = lo[1] + (int)(r % wy), kk = lo[2] + (int)(r / wy);
      if (BOX) { xa = lo[0]; xb = hi[0]; }
      else row_interval(nrm, rhs, hs, jj, kk, lo[0], hi[0], &xa, &xb);
      rowoff = ((long long)kk * g.ny + jj) * g.nx;
    }
    if (QUAD) {
      // (rows start on 16-byte boundaries) the chunk's voxels as aligned 16-byte quads, dealt
      // to the lanes in row order: neighbouring lanes read neighbouring quads of a row and
      // every lane has work however long or short the rows are
      const unsigned full = ~0u;
      const int qa = xa >> 2;
      const int nq = xb >= xa ? (xb >> 2) - qa + 1 : 0;
      int incl = nq;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(full, incl, o);
        if ((int)lane >= o) incl += t;
      }
      const int Q = __shfl_sync(full, incl, 31);
      const int start = incl - nq;
#pragma unroll 2
      for (int g0 = 0; g0 < Q; g0 += 32) {
        const int gq = g0 + (int)lane;
        // the row of quad gq: the last lane whose first quad is at or before it
        int rr = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1)
          if (__shfl_sync(full, start, rr + step) <= gq) rr += step;
        const int ra = __shfl_sync(full, xa, rr), rb = __shfl_sync(full, xb, rr);
        const long long ro = __shfl_sync(full, rowoff, rr);
        const int quad = (ra >> 2) + (gq - __shfl_sync(full, start, rr));
        if (gq < Q) {
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(q + ro) + quad);
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int xx = 4 * quad + e;
            if (xx >= ra && xx <= rb) { ++cnt; sum += w[e]; mn = min(mn, w[e]); mx = max(mx, w[e]); }
          }
        }
      }
    } else if (hi[0] - lo[0] >= 31) {
      // wide box: lanes along x (coalesced), four rows at a time
      for (int k = 0; k < 32; k += 4) {
        int a[4], b[4];
        long long ro[4];
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = __shfl_sync(~0u, xa, k + u);
          b[u] = __shfl_sync(~0u, xb, k + u);
          ro[u] = __shfl_sync(~0u, rowoff, k + u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = a[u] + (int)lane <= b[u] ? __ldg(q + ro[u] + a[u] + (int)lane) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (a[u] + (int)lane <= b[u]) { ++cnt; sum += v[u]; mn = min(mn, v[u]); mx = max(mx, v[u]); }
#pragma unroll
        for (int u = 0; u < 4; ++u) row_tail(q + ro[u], a[u] + 32, b[u], lane, cnt, sum, mn, mx);
      }
    } else {
      // narrow box: one row per lane
#pragma unroll 4
      for (int ii = xa; ii <= xb; ++ii) {
        const uint32_t v = __ldg(q + rowoff + ii);
        ++cnt; sum += v; mn = min(mn, v); mx = max(mx, v);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      cnt += __shfl_xor_sync(~0u, cnt, o);
      sum += __shfl_xor_sync(~0u, sum, o);
      mn = min(mn, __shfl_xor_sync(~0u, mn, o));
      mx = max(mx, __shfl_xor_sync(~0u, mx, o));
    }
    if (lane == 0 && cnt) {
      atomicAdd(L.cnt + i, cnt);
      atomicAdd(L.sum + i, sum);
      atomicMin(L.mn + i, mn);
      atomicMax(L.mx + i, mx);
    }
  }
}

__global__ void k_channel_store(LeafPtrs L, long long m, const uint32_t* __restrict__ q, Geo g, int c,
                                float* __restrict__ chan) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  unsigned long long sum = L.sum[i];
  uint32_t cnt = L.cnt[i];
  if (cnt == 0) {
    int x[4][3];
    load_tet(L.v, i, x);
    const int dims[3] = {g.nx, g.ny, g.nz};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long s4 = (long long)x[0][a] + x[1][a] + x[2][a] + x[3][a];
      const long long v = s4 >> (g.K + 2 - g.m);
      idx[a] = (int)(v < 0 ? 0 : (v > dims[a] - 1 ? dims[a] - 1 : v));
    }
    sum = q[((size_t)idx[2] * g.ny + idx[1]) * g.nx + idx[0]];
    cnt = 1;
  }
  float mean = (float)((double)sum / ((double)cnt * 16777216.0));
  if (c == 2) mean = (float)fmin(0.99, fmax(-0.99, 2.0 * (double)mean - 1.0));
  chan[4 * i + c] = mean;
}

// Voxel majorant of every final tet: (max q + 1) / 2^24 over the voxels touching its box
__global__ void k_vmaj_store(LeafPtrs L, long long m, float* __restrict__ vmaj) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  vmaj[i] = (float)(((double)L.mx[i] + 1.0) / 16777216.0);
}

// Rebuild: statistics of every node of a previous build of the same volume --
// its leaves and its interior nodes, each sorted by code.
struct PrevNodes {
  const unsigned long long *leaf_code, *leaf_sum, *node_code, *node_sum;
  const uint32_t *leaf_cnt, *leaf_mn, *leaf_mx, *node_cnt, *node_mn, *node_mx;
  long long nleaf, nnode;
};

__device__ __forceinline__ long long find_code(const unsigned long long* a, long long n, unsigned long long c) {
  long long lo = 0, hi = n;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (a[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo < n && a[lo] == c ? lo : -1;
}

// New leaves whose statistics a previous build already has take them from it;
// the others are listed as misses (miss[j] = 1) for the voxel scan.
__global__ void k_lookup(LeafPtrs L, const long long* list, long long m, PrevNodes P, uint8_t* known,
                         unsigned long long* miss) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const long long i = list ? list[j] : j;
  const unsigned long long c = L.code[i];
  long long k = find_code(P.leaf_code, P.nleaf, c);
  if (k >= 0) {
    L.cnt[i] = P.leaf_cnt[k]; L.sum[i] = P.leaf_sum[k]; L.mn[i] = P.leaf_mn[k]; L.mx[i] = P.leaf_mx[k];
  } else if ((k = find_code(P.node_code, P.nnode, c)) >= 0) {
    L.cnt[i] = P.node_cnt[k]; L.sum[i] = P.node_sum[k]; L.mn[i] = P.node_mn[k]; L.mx[i] = P.node_mx[k];
  }
  known[j] = k >= 0 ? 1 : 0;
  miss[j] = k >= 0 ? 0ull : 1ull;
}

__global__ void k_compact_misses(const long long* list, long long m, const unsigned long long* miss,
                                 const unsigned long long* pos, long long* out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m || !miss[j]) return;
  out[pos[j]] = list ? list[j] : j;
}

// Interior-node statistics sorted by code (perm from the key sort)
__global__ void k_iota(unsigned long long* a, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (unsigned long long)i;
}

__global__ void k_gather_nodes(NodePtrs src, const unsigned long long* perm, long long n, NodePtrs dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long k = (long long)perm[i];
  dst.sum[i] = src.sum[k]; dst.cnt[i] = src.cnt[k]; dst.mn[i] = src.mn[k]; dst.mx[i] = src.mx[k];
}

// Sec. 2 criterion 2 in fp64 with every product and sum rounded on its own.
__device__ bool camera_allows(const CamD& c, const Geo& g, const int x[4][3]) {
  if (!c.on) return true;
  const double s = ldexp(1.0, -g.K);
  double xc[4], yc[4], zc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double d0 = __dsub_rn(__dmul_rn((double)x[i][0], s), c.eye[0]);
    const double d1 = __dsub_rn(__dmul_rn((double)x[i][1], s), c.eye[1]);
    const double d2 = __dsub_rn(__dmul_rn((double)x[i][2], s), c.eye[2]);
    zc[i] = __dadd_rn(__dadd_rn(__dmul_rn(d0, c.f[0]), __dmul_rn(d1, c.f[1])), __dmul_rn(d2, c.f[2]));
    xc[i] = __dadd_rn(__dadd_rn(__dmul_rn(d0, c.r[0]), __dmul_rn(d1, c.r[1])), __dmul_rn(d2, c.r[2]));
    yc[i] = __dadd_rn(__dadd_rn(__dmul_rn(d0, c.u[0]), __dmul_rn(d1, c.u[1])), __dmul_rn(d2, c.u[2]));
  }
  bool near_ = true, right = true, left = true, top = true, bottom = true;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double ax = __dmul_rn(zc[i], c.tanX), ay = __dmul_rn(zc[i], c.tanF);
    near_ = near_ && zc[i] < c.near_g;
    right = right && xc[i] > ax;
    left = left && xc[i] < -ax;
    top = top && yc[i] > ay;
    bottom = bottom && yc[i] < -ay;
  }
  if (near_ || right || left || top || bottom) return false;
  double zmin = fmin(fmin(zc[0], zc[1]), fmin(zc[2], zc[3]));
  if (zmin < c.near_g) zmin = c.near_g;
  long long L2 = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) {
      long long e = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) { const long long t = (long long)x[i][a] - x[j][a]; e += t * t; }
      L2 = max(L2, e);
    }
  const double lmax2 = __dmul_rn(__dmul_rn((double)L2, s), s);
  const double pix = __dmul_rn(c.thr, zmin);
  return lmax2 > __dmul_rn(pix, pix);
}

// Criterion 2 in float with a bound on the error of every quantity it compares,
// relative to the exact value of the fp64 inputs: 1 or 0 when every comparison
// is decided by more than its bound (then the exact value, and so camera_allows,
// whose fp64 rounding is far inside the bound, decides the same way), -1 when
// one is too close to call (the caller then takes camera_allows).  Every float
// operation here is rounded once (relative error 2^-24), the inputs' conversion
// to float too; the bounds allow 2^-20, sixteen times that, on every term.
__device__ int camera_allows_f32(const CamF& c, const Geo& g, const int x[4][3]) {
  const float e = 9.5367431640625e-07f;           // 2^-20
  const float s = __int_as_float((127 - g.K) << 23);   // 2^-K (K < 127)
  float zc[4], xc[4], yc[4], ez[4], ex[4], ey[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float d[3], ad[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[a] = (float)x[i][a] * s - c.eye[a];       // x < 2^24: x s is exact
      ad[a] = fabsf(d[a]);
    }
    zc[i] = d[0] * c.f[0] + d[1] * c.f[1] + d[2] * c.f[2];
    xc[i] = d[0] * c.r[0] + d[1] * c.r[1] + d[2] * c.r[2];
    yc[i] = d[0] * c.u[0] + d[1] * c.u[1] + d[2] * c.u[2];
    ez[i] = e * (ad[0] * fabsf(c.f[0]) + ad[1] * fabsf(c.f[1]) + ad[2] * fabsf(c.f[2]) + c.ef);
    ex[i] = e * (ad[0] * fabsf(c.r[0]) + ad[1] * fabsf(c.r[1]) + ad[2] * fabsf(c.r[2]) + c.er);
    ey[i] = e * (ad[0] * fabsf(c.u[0]) + ad[1] * fabsf(c.u[1]) + ad[2] * fabsf(c.u[2]) + c.eu);
  }
  bool near_ = true, right = true, left = true, top = true, bottom = true;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float gz = zc[i] - c.near_g;
    if (fabsf(gz) <= ez[i] + e * c.near_g) return -1;
    near_ = near_ && gz < 0.f;
    const float ax = zc[i] * c.tanX, ay = zc[i] * c.tanF;
    const float bx = ex[i] + ez[i] * c.tanX + e * (fabsf(xc[i]) + fabsf(ax));
    const float by = ey[i] + ez[i] * c.tanF + e * (fabsf(yc[i]) + fabsf(ay));
    const float gr = xc[i] - ax, gl = xc[i] + ax, gt = yc[i] - ay, gb = yc[i] + ay;
    if (fabsf(gr) <= bx || fabsf(gl) <= bx || fabsf(gt) <= by || fabsf(gb) <= by) return -1;
    right = right && gr > 0.f;
    left = left && gl < 0.f;
    top = top && gt > 0.f;
    bottom = bottom && gb < 0.f;
  }
  if (near_ || right || left || top || bottom) return 0;
  float zmin = fminf(fminf(zc[0], zc[1]), fminf(zc[2], zc[3]));
  float ezm = fmaxf(fmaxf(ez[0], ez[1]), fmaxf(ez[2], ez[3]));
  if (fabsf(zmin - c.near_g) <= ezm + e * c.near_g) return -1;
  if (zmin < c.near_g) { zmin = c.near_g; ezm = 0.f; }
  long long L2 = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) {
      long long d2 = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) { const long long t = (long long)x[i][a] - x[j][a]; d2 += t * t; }
      L2 = max(L2, d2);
    }
  const float lm = (float)L2 * s * s;
  const float pix = c.thr * zmin, P = pix * pix;
  const float gf = lm - P;
  if (fabsf(gf) <= e * (lm + P) + 2.5f * pix * c.thr * ezm) return -1;
  return gf > 0.f ? 1 : 0;
}

// A3 statistics, pass 3 (empty D -> voxel of the centroid) and the criterion of every new leaf
__global__ void k_stats_finish(LeafPtrs L, const long long* list, long long m, const uint32_t* __restrict__ q,
                               Crit C, const uint8_t* known) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const long long i = list ? list[j] : j;
  int x[4][3];
  load_tet(L.v, i, x);
  const Geo& g = C.g;
  if (L.cnt[i] == 0) {
    const int dims[3] = {g.nx, g.ny, g.nz};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long s4 = (long long)x[0][a] + x[1][a] + x[2][a] + x[3][a];
      long long c = s4 >> (g.K + 2 - g.m);
      idx[a] = (int)(c < 0 ? 0 : (c > dims[a] - 1 ? dims[a] - 1 : c));
    }
    const uint32_t v = q[((size_t)idx[2] * g.ny + idx[1]) * g.nx + idx[0]];
    L.cnt[i] = 1; L.sum[i] = v; L.mn[i] = v; L.mx[i] = v;
  }
  const int depth = (int)(L.code[i] & 63ull);
  bool s = depth < g.max_depth;
  if (s && C.var_on) {
    const unsigned __int128 lhs = (unsigned __int128)(L.mx[i] - L.mn[i]) * L.cnt[i] * 65536u;
    const unsigned __int128 rhs = (unsigned __int128)C.theta_q16 * L.sum[i];
    s = lhs > rhs;
  }
  if (s && C.cam.on) {
    const int f = camera_allows_f32(C.camf, g, x);
    s = f < 0 ? camera_allows(C.cam, g, x) : f == 1;
  }
  L.crit[i] = s ? 1 : 0;
}

// A5: mark = criterion || a vertex of the grid at one of the six edge midpoints
// (the filter rules out most midpoints with one read from L2; the rest are
// looked up in the vertex set)
__global__ void k_mark(LeafPtrs L, long long n, const unsigned long long* keys, unsigned long long mask, Bloom bloom,
                       unsigned long long* marks, unsigned long long* nmark) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool mk = false;
  if (i < n) {
    mk = L.crit[i] != 0;
    if (!mk) {
      int x[4][3];
      load_tet(L.v, i, x);
      for (int a = 0; a < 4 && !mk; ++a)
        for (int b = a + 1; b < 4 && !mk; ++b) {
          const int s0 = x[a][0] + x[b][0], s1 = x[a][1] + x[b][1], s2 = x[a][2] + x[b][2];
          if ((s0 | s1 | s2) & 1) continue;        // off the lattice: not a vertex
          const unsigned long long key = pack3(s0 >> 1, s1 >> 1, s2 >> 1);
          mk = bloom_may_hold(bloom, key) && hset_find(keys, mask, key) >= 0;
        }
    }
    marks[i] = mk ? 1 : 0;
  }
  const unsigned b = __ballot_sync(~0u, mk);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(nmark, (unsigned long long)__popc(b));
}

// Child w of a tet with refinement edge x0 xk (Maubach bisection, z its
// midpoint): child 0 is the tet with xk replaced by z, child 1 drops x0, shifts
// x1..xk down by one and puts z at position k.  Written with static indices only
// (a select per vertex), so the vertices stay in registers.
__device__ __forceinline__ void bisect(const int x[4][3], int k, int w, int y[4][3]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int z = (x[0][a] + (k == 1 ? x[1][a] : (k == 2 ? x[2][a] : x[3][a]))) >> 1;
      const int up = i < 3 ? x[i + 1][a] : x[3][a];
      y[i][a] = i == k ? z : ((w == 1 && i < k) ? up : x[i][a]);
    }
}

// A4: Maubach bisection of the marked leaves.  While many leaves split, the
// leaves are rebuilt by a stable compaction in which a split leaf is replaced
// by its two children, which keeps them in depth-first order of their codes
// (APPEND false).  Once few do, the first child takes its parent's slot and the
// second is appended at n + its parent's rank among the split leaves, so a round
// touches only the leaves it splits (APPEND true; the appended leaves are put
// in order after the last round).  The new vertices go to the vertex set and
// its filter.
template <bool APPEND>
__global__ void k_split(LeafPtrs S, long long n, const unsigned long long* marks, const unsigned long long* pos,
                        LeafPtrs D, long long* newlist, unsigned long long* keys, unsigned long long mask,
                        Bloom bloom, unsigned long long* vcount, NodePtrs arch, long long abase) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (APPEND && !marks[i]) return;
  const long long before = (long long)pos[i];
  if (!marks[i]) {
    const long long j = i + before;
    D.v[3 * j] = S.v[3 * i]; D.v[3 * j + 1] = S.v[3 * i + 1]; D.v[3 * j + 2] = S.v[3 * i + 2];
    D.code[j] = S.code[i]; D.tag[j] = S.tag[i]; D.crit[j] = S.crit[i];
    D.cnt[j] = S.cnt[i]; D.sum[j] = S.sum[i]; D.mn[j] = S.mn[i]; D.mx[j] = S.mx[i];
    return;
  }
  const unsigned long long code = S.code[i];
  {
    const long long a = abase + before;
    arch.code[a] = code; arch.sum[a] = S.sum[i];
    arch.cnt[a] = S.cnt[i]; arch.mn[a] = S.mn[i]; arch.mx[a] = S.mx[i];
  }
  int x[4][3];
  load_tet(S.v, i, x);
  const int k = S.tag[i];
  const int depth = (int)(code & 63ull);
  const unsigned long long base = (code & ~63ull) | (unsigned long long)(depth + 1);
  const uint8_t nt = (uint8_t)(k > 1 ? k - 1 : 3);
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    int y[4][3];
    bisect(x, k, w, y);
    const long long j = APPEND ? (w == 0 ? i : n + before) : i + before + w;
    store_tet(D.v, j, y);
    D.code[j] = base | ((unsigned long long)w << (55 - depth));
    D.tag[j] = nt;
    newlist[2 * before + w] = j;
  }
  int z[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) z[a] = (x[0][a] + (k == 1 ? x[1][a] : (k == 2 ? x[2][a] : x[3][a]))) >> 1;
  const unsigned long long key = pack3(z[0], z[1], z[2]);
  if (hset_insert(keys, mask, key, vcount) < 0) atomicAdd(vcount + 3, 1ull);
  bloom_add(bloom, key);
}

// number of the n sorted codes a[] below c
__device__ __forceinline__ long long count_below(const unsigned long long* __restrict__ a, long long n,
                                                 unsigned long long c) {
  long long lo = 0, hi = n;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (a[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The leaves in code order, into the arrays the grid keeps: leaves [0, ns) are in
// order already, the nt appended after them are in order through tperm (their
// codes sorted: tcode), and each leaf's place is its rank in its own run plus the
// number of the other run's codes below its own.
__global__ void k_place_leaves(LeafPtrs S, long long ns, long long nt, const unsigned long long* __restrict__ tcode,
                               const uint32_t* __restrict__ tperm, LeafPtrs D) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns + nt) return;
  long long src, dst;
  unsigned long long code;
  if (t < ns) {
    src = t;
    code = S.code[t];
    dst = t + count_below(tcode, nt, code);
  } else {
    const long long r = t - ns;
    src = ns + tperm[r];
    code = tcode[r];
    dst = r + count_below(S.code, ns, code);
  }
  D.v[3 * dst] = S.v[3 * src]; D.v[3 * dst + 1] = S.v[3 * src + 1]; D.v[3 * dst + 2] = S.v[3 * src + 2];
  D.code[dst] = code; D.tag[dst] = S.tag[src];
  D.cnt[dst] = S.cnt[src]; D.sum[dst] = S.sum[src]; D.mn[dst] = S.mn[src]; D.mx[dst] = S.mx[src];
}

__global__ void k_iota32(uint32_t* a, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (uint32_t)i;
}

// A6: face matching
// Faces as (key, 4 i + f), the key the vertex sum of the face packed in 3 fields
// of fb bits; sorted by key, the two faces of a shared key are neighbours.
__global__ void k_face_keys(const int4* v, long long n, int fb, unsigned long long* keys, uint32_t* ids) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x[4][3];
  load_tet(v, i, x);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    unsigned long long s[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k != f)
#pragma unroll
        for (int a = 0; a < 3; ++a) s[a] += (unsigned long long)x[k][a];
    keys[4 * i + f] = s[0] | (s[1] << fb) | (s[2] << (2 * fb));
    ids[4 * i + f] = (uint32_t)(4 * i + f);
  }
}

// The face across each face (4 i' + f'), or NO_FACE for a face of one cell;
// three faces with one key flag the grid.
constexpr uint32_t NO_FACE = 0xFFFFFFFFu;
__global__ void k_face_pairs(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ ids,
                             long long nf, uint32_t* nbr, int* err) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nf) return;
  const unsigned long long k = keys[p];
  const bool prev = p > 0 && keys[p - 1] == k, next = p + 1 < nf && keys[p + 1] == k;
  if (prev && next) atomicOr(err, 8);
  nbr[ids[p]] = next ? ids[p + 1] : (prev ? ids[p - 1] : NO_FACE);
}

__device__ __forceinline__ bool same_face(const int x[4][3], int f, const int y[4][3], int g) {
  // the three vertices of face f of x are the three vertices of face g of y
  for (int a = 0; a < 4; ++a) {
    if (a == f) continue;
    bool found = false;
    for (int b = 0; b < 4; ++b)
      if (b != g && x[a][0] == y[b][0] && x[a][1] == y[b][1] && x[a][2] == y[b][2]) found = true;
    if (!found) return false;
  }
  return true;
}

__device__ __forceinline__ uint32_t encode_density(double mean, int fmt) {
  const float f = __double2float_rn(mean);
  if (fmt == TG_DENSITY_BF16) {
    const uint32_t u = __float_as_uint(f);
    return ((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16) << 16;   // the high half: the word reads as the float
  }
  if (fmt == TG_DENSITY_FP16) return (uint32_t)__half_as_ushort(__float2half_rn(f));
  return __float_as_uint(f);
}

__global__ void k_finalize(LeafPtrs L, long long n, Geo g, int fmt, const uint32_t* __restrict__ fnbr, uint4* rec,
                           float* majorant, int* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x[4][3];
  load_tet(L.v, i, x);
  uint32_t link[4];
  int cpl[4];
  for (int f = 0; f < 4; ++f) {
    uint32_t nb = NO_NBR;
    const uint32_t other = fnbr[4 * i + f];
    if (other != NO_FACE) {
      int y[4][3];
      load_tet(L.v, other >> 2, y);
      if (!same_face(x, f, y, (int)(other & 3))) { atomicOr(err, 2); return; }
      nb = other >> 2;
    } else {
      // a face of one cell must lie on the domain boundary
      bool bnd = false;
      const int a = (f + 1) & 3, b = (f + 2) & 3, cc = (f + 3) & 3;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const int lim = g.C[ax] << g.K;
        if (x[a][ax] == x[b][ax] && x[a][ax] == x[cc][ax] && (x[a][ax] == 0 || x[a][ax] == lim)) bnd = true;
      }
      if (!bnd) { atomicOr(err, 4); return; }
    }
    int nrm[3];
    long long rhs;
    if (!face_plane(x, f, nrm, &rhs)) { atomicOr(err, 16); return; }
    const int id = orient_id(nrm);
    if (id < 0) { atomicOr(err, 16); return; }
    const int v3[3] = {x[(f + 1) & 3][0], x[(f + 1) & 3][1], x[(f + 1) & 3][2]};
    cpl[f] = p9_dot(id & 15, v3);
    link[f] = nb | ((uint32_t)id << 27);
  }
  const double mean = __ddiv_rn((double)L.sum[i], __dmul_rn((double)L.cnt[i], 16777216.0));
  const uint32_t m24 = 0xFFFFFFu;
  rec[2 * i] = make_uint4(link[0], link[1], link[2], link[3]);
  rec[2 * i + 1] = make_uint4(((uint32_t)cpl[0] & m24) | ((uint32_t)cpl[1] << 24),
                              (((uint32_t)cpl[1] & m24) >> 8) | ((uint32_t)cpl[2] << 16),
                              (((uint32_t)cpl[2] & m24) >> 16) | ((uint32_t)cpl[3] << 8), encode_density(mean, fmt));
  majorant[i] = __double2float_rn(__ddiv_rn((double)L.mx[i], 16777216.0));
}

__global__ void k_code_depth(const unsigned long long* __restrict__ codes, long long n, int* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(out, (int)(codes[i] & 63ull));
}

unsigned long long next_pow2(unsigned long long v) {
  unsigned long long p = 1;
  while (p < v) p <<= 1;
  return p;
}

unsigned blocks_for(long long n, int tpb = TPB) { return (unsigned)std::max<long long>(1, (n + tpb - 1) / tpb); }

struct Scanner {
  DevBuf<char> tmp;
  void exclusive(const unsigned long long* in, unsigned long long* out, long long n, cudaStream_t st) {
    size_t bytes = 0;
    TV_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, st));
    tmp.ensure(bytes + 16);
    TV_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, bytes, in, out, n, st));
  }
};

// every row of the quantised volume starts on a 16-byte boundary
bool quad_rows(const Geo& g, const uint32_t* q) { return g.nx % 4 == 0 && reinterpret_cast<uintptr_t>(q) % 16 == 0; }

// Pass 2 of the statistics over `total` work items (offsets off[0..m]): the
// owner of every work item, then the scan.
template <bool BOX>
void stats_scan(LeafPtrs L, const ScanDesc* desc, long long m, const unsigned long long* off,
                unsigned long long total, DevBuf<int>& owner, const uint32_t* q, const Geo& g, int sms,
                cudaStream_t st) {
  owner.ensure(total);
  k_chunk_owner<<<blocks_for(m), TPB, 0, st>>>(off, m, owner.p);
  TV_LAUNCH();
  const long long wblocks = std::min<long long>((long long)(total + (TPB / 32) - 1) / (TPB / 32), (long long)sms * 64);
  // 16-byte loads along the rows when every row starts on a 16-byte boundary
  if (quad_rows(g, q))
    k_stats_scan<BOX, true><<<(unsigned)wblocks, TPB, 0, st>>>(L, desc, off, owner.p, total, q, g);
  else
    k_stats_scan<BOX, false><<<(unsigned)wblocks, TPB, 0, st>>>(L, desc, off, owner.p, total, q, g);
  TV_LAUNCH();
}

// Scratch of the rebuild's statistics lookup
struct LookupBufs {
  DevBuf<uint8_t> known;
  DevBuf<unsigned long long> miss, pos;
  DevBuf<long long> list;
};

// Statistics and criterion of m new leaves (list == nullptr: leaves 0..m-1).
// With a previous build (prev), leaves it already had take its statistics and
// only the others are scanned.
void stats_and_criterion(Leaves& Lv, const long long* list, long long m, const uint32_t* q, const Crit& C,
                         Scanner& scan, DevBuf<unsigned long long>& chunks, DevBuf<unsigned long long>& off,
                         DevBuf<int>& owner, DevBuf<ScanDesc>& desc, cudaStream_t st, int sms,
                         const PrevNodes* prev, LookupBufs& lk) {
  if (m == 0) return;
  LeafPtrs L = Lv.ptrs();
  const long long* slist = list;              // leaves to scan
  long long sm = m;
  const uint8_t* known = nullptr;
  if (prev) {
    lk.known.ensure(m);
    lk.miss.ensure(m + 1);
    lk.pos.ensure(m + 1);
    lk.list.ensure(m);
    k_lookup<<<blocks_for(m), TPB, 0, st>>>(L, list, m, *prev, lk.known.p, lk.miss.p);
    TV_LAUNCH();
    TV_CUDA(cudaMemsetAsync(lk.miss.p + m, 0, sizeof(unsigned long long), st));
    scan.exclusive(lk.miss.p, lk.pos.p, m + 1, st);
    k_compact_misses<<<blocks_for(m), TPB, 0, st>>>(list, m, lk.miss.p, lk.pos.p, lk.list.p);
    TV_LAUNCH();
    unsigned long long nm = 0;
    TV_CUDA(cudaMemcpyAsync(&nm, lk.pos.p + m, sizeof nm, cudaMemcpyDeviceToHost, st));
    TV_CUDA(cudaStreamSynchronize(st));
    slist = lk.list.p;
    sm = (long long)nm;
    known = lk.known.p;
  }
  if (sm > 0) {
    chunks.ensure(sm + 1);
    off.ensure(sm + 1);
    desc.ensure(sm);
    if (quad_rows(C.g, q))
      k_stats_prep<false, true><<<blocks_for(sm), TPB, 0, st>>>(L, slist, sm, C.g, chunks.p, desc.p, q);
    else
      k_stats_prep<false, false><<<blocks_for(sm), TPB, 0, st>>>(L, slist, sm, C.g, chunks.p, desc.p, q);
    TV_LAUNCH();
    TV_CUDA(cudaMemsetAsync(chunks.p + sm, 0, sizeof(unsigned long long), st));
    scan.exclusive(chunks.p, off.p, sm + 1, st);
    unsigned long long total = 0;
    TV_CUDA(cudaMemcpyAsync(&total, off.p + sm, sizeof total, cudaMemcpyDeviceToHost, st));
    TV_CUDA(cudaStreamSynchronize(st));
    if (total) stats_scan<false>(L, desc.p, sm, off.p, total, owner, q, C.g, sms, st);
  }
  k_stats_finish<<<blocks_for(m), TPB, 0, st>>>(L, list, m, q, C, known);
  TV_LAUNCH();
}

void normalize3(double v[3]) {
  const double l = std::sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
  v[0] /= l; v[1] /= l; v[2] /= l;
}

void cross3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

// Camera of criterion 2 in grid space (host, fp64, each operation rounded on its own).
CamD camera_for_criterion(const tg_camera* cam, float footprint_px, const float box_min[3], double cube) {
  CamD c;
  std::memset(&c, 0, sizeof c);
  c.on = cam != nullptr && footprint_px > 0.f;
  if (!c.on) return c;
  double up[3] = {cam->up[0], cam->up[1], cam->up[2]};
  for (int a = 0; a < 3; ++a) {
    c.eye[a] = ((double)cam->pos[a] - (double)box_min[a]) / cube;
    c.f[a] = (double)cam->target[a] - (double)cam->pos[a];
  }
  normalize3(c.f);
  cross3(c.f, up, c.r);
  normalize3(c.r);
  cross3(c.r, c.f, c.u);
  normalize3(c.u);
  c.tanF = std::tan((double)cam->fov_y_deg * 0.0087266462599716478846);
  c.tanX = c.tanF * ((double)cam->width / (double)cam->height);
  c.near_g = 1e-3 / cube;
  c.thr = (2.0 * c.tanF / (double)cam->height) * (double)footprint_px;
  return c;
}

CamF camera_f32(const CamD& c) {
  CamF f;
  std::memset(&f, 0, sizeof f);
  for (int a = 0; a < 3; ++a) {
    f.eye[a] = (float)c.eye[a]; f.f[a] = (float)c.f[a]; f.r[a] = (float)c.r[a]; f.u[a] = (float)c.u[a];
    f.ef += std::fabs(f.f[a]) * std::fabs(f.eye[a]);
    f.er += std::fabs(f.r[a]) * std::fabs(f.eye[a]);
    f.eu += std::fabs(f.u[a]) * std::fabs(f.eye[a]);
  }
  f.tanF = (float)c.tanF; f.tanX = (float)c.tanX; f.near_g = (float)c.near_g; f.thr = (float)c.thr;
  return f;
}

}  // namespace

int build_grid(const float* density, const tg_volume_desc* vol, const tg_camera* cam, float footprint_px,
               float theta, int32_t max_depth, int32_t fmt, cudaStream_t st, GridImpl& G, const GridImpl* prev) {
  Geo g;
  g.nx = vol->nx; g.ny = vol->ny; g.nz = vol->nz;
  int n = 1, m = 0;
  while (g.nx % (2 * n) == 0 && g.ny % (2 * n) == 0 && g.nz % (2 * n) == 0 && n < (1 << 18)) { n *= 2; ++m; }
  g.n = n; g.m = m;
  g.C[0] = g.nx / n; g.C[1] = g.ny / n; g.C[2] = g.nz / n;
  g.K = std::max((max_depth + 2) / 3 + 1, m + 1);
  g.max_depth = max_depth;
  for (int a = 0; a < 3; ++a)
    if (((long long)g.C[a] << g.K) > (1ll << 19)) return TG_EINVAL;
  const int nroots = 6 * g.C[0] * g.C[1] * g.C[2];
  if (nroots > 256) return TG_EINVAL;
  g.h = 1 << (g.K - m - 1);

  Crit C;
  C.g = g;
  const double cube = (double)vol->voxel_size * (double)n;
  C.cam = camera_for_criterion(cam, footprint_px, vol->box_min, cube);
  C.camf = camera_f32(C.cam);
  C.var_on = theta >= 0.f;
  C.theta_q16 = C.var_on ? (unsigned long long)std::llround((double)theta * 65536.0) : 0ull;

  int dev = 0, sms = 0;
  TV_CUDA(cudaGetDevice(&dev));
  TV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  const long long nvox = (long long)g.nx * g.ny * g.nz;
  DevBuf<uint32_t> q(nvox);
  k_quantize<<<(unsigned)std::min<long long>(blocks_for(nvox), (long long)sms * 32), TPB, 0, st>>>(density, q.p, nvox);
  TV_LAUNCH();

  Leaves A, B;
  A.ensure(nroots);
  k_roots<<<blocks_for(nroots), TPB, 0, st>>>(A.ptrs(), g, nroots);
  TV_LAUNCH();

  // vertex set
  unsigned long long hcap = next_pow2(std::max<long long>(4096, 8ll * nroots));
  DevBuf<unsigned long long> hkeys(hcap), counters(4);   // counters: vertices, marks
  DevBuf<uint32_t> bloomw(hcap / 8);                     // 4 filter bits per table slot
  TV_CUDA(cudaMemsetAsync(hkeys.p, 0xFF, hcap * 8, st));
  TV_CUDA(cudaMemsetAsync(bloomw.p, 0, hcap / 2, st));
  TV_CUDA(cudaMemsetAsync(counters.p, 0, 4 * 8, st));
  k_insert_vertices<<<blocks_for(nroots), TPB, 0, st>>>(A.v.p, nroots, hkeys.p, hcap - 1, Bloom{bloomw.p, hcap / 8 - 1},
                                                        counters.p);
  TV_LAUNCH();

  // a previous build of the same volume lends its node statistics
  PrevNodes pn;
  const PrevNodes* pp = nullptr;
  if (prev) {
    if (!prev->node_code || prev->K != g.K || prev->nvox[0] != g.nx || prev->nvox[1] != g.ny ||
        prev->nvox[2] != g.nz)
      return TG_EINVAL;
    pn.leaf_code = prev->codes; pn.leaf_sum = prev->sum; pn.leaf_cnt = prev->count; pn.leaf_mn = prev->qmin;
    pn.leaf_mx = prev->qmax; pn.nleaf = prev->n;
    pn.node_code = prev->node_code; pn.node_sum = prev->node_sum; pn.node_cnt = prev->node_cnt;
    pn.node_mn = prev->node_mn; pn.node_mx = prev->node_mx; pn.nnode = prev->n_nodes;
    pp = &pn;
  }
  LookupBufs lk;

  Scanner scan;
  DevBuf<unsigned long long> chunks, off, marks, pos;
  DevBuf<int> owner;
  DevBuf<ScanDesc> desc;
  DevBuf<long long> newlist;
  long long nsorted = -1;                          // leaves [0, nsorted) in code order once splits append
  // interior nodes, appended as leaves are split
  DevBuf<unsigned long long> acode, asum;
  DevBuf<uint32_t> acnt, amn, amx;
  long long nint = 0;
  stats_and_criterion(A, nullptr, nroots, q.p, C, scan, chunks, off, owner, desc, st, sms, pp, lk);

  long long N = nroots;
  const int max_rounds = 4 * max_depth + 16;
  int round = 0;
  for (;; ++round) {
    marks.ensure(N + 1);
    pos.ensure(N + 1);
    TV_CUDA(cudaMemsetAsync(counters.p + 1, 0, 8, st));
    k_mark<<<blocks_for(N), TPB, 0, st>>>(A.ptrs(), N, hkeys.p, hcap - 1, Bloom{bloomw.p, hcap / 8 - 1}, marks.p,
                                          counters.p + 1);
    TV_LAUNCH();
    unsigned long long hc[4];
    TV_CUDA(cudaMemcpyAsync(hc, counters.p, 32, cudaMemcpyDeviceToHost, st));
    TV_CUDA(cudaStreamSynchronize(st));
    if (hc[3]) return TG_ENOMEM;                 // the vertex set overflowed
    const long long M = (long long)hc[1];
    if (M == 0) break;
    if (round >= max_rounds) return TG_EROUNDLIMIT;
    if (N + M > MAX_TETS) return TG_ENOMEM;
    // grow the vertex set to keep its load under one half
    if (2 * (hc[0] + (unsigned long long)M) > hcap) {
      const unsigned long long ncap = next_pow2(4 * (hc[0] + (unsigned long long)M));
      DevBuf<unsigned long long> nk(ncap);
      DevBuf<uint32_t> nb(ncap / 8);
      TV_CUDA(cudaMemsetAsync(nk.p, 0xFF, ncap * 8, st));
      TV_CUDA(cudaMemsetAsync(nb.p, 0, ncap / 2, st));
      k_rehash<<<blocks_for((long long)hcap), TPB, 0, st>>>(hkeys.p, (long long)hcap, nk.p, ncap - 1,
                                                            Bloom{nb.p, ncap / 8 - 1}, counters.p + 3);
      TV_LAUNCH();
      TV_CUDA(cudaStreamSynchronize(st));
      hkeys = std::move(nk);
      bloomw = std::move(nb);
      hcap = ncap;
    }
    TV_CUDA(cudaMemsetAsync(marks.p + N, 0, 8, st));
    scan.exclusive(marks.p, pos.p, N + 1, st);
    // splits append once fewer than one leaf in eight splits (the compaction would copy every leaf)
    if (nsorted < 0 && 8 * M < N) {
      nsorted = N;
      B = Leaves();
    }
    if (nsorted >= 0) A.grow(N + M, N, st);
    else B.ensure(N + M);
    newlist.ensure(2 * M);
    if ((size_t)(nint + M) > acode.n) {
      // grow the interior-node arrays (keep what they hold)
      const size_t cap = std::max<size_t>(2 * (size_t)(nint + M), 1024);
      DevBuf<unsigned long long> c2(cap), s2(cap);
      DevBuf<uint32_t> n2(cap), m2(cap), x2(cap);
      if (nint) {
        TV_CUDA(cudaMemcpyAsync(c2.p, acode.p, nint * 8, cudaMemcpyDeviceToDevice, st));
        TV_CUDA(cudaMemcpyAsync(s2.p, asum.p, nint * 8, cudaMemcpyDeviceToDevice, st));
        TV_CUDA(cudaMemcpyAsync(n2.p, acnt.p, nint * 4, cudaMemcpyDeviceToDevice, st));
        TV_CUDA(cudaMemcpyAsync(m2.p, amn.p, nint * 4, cudaMemcpyDeviceToDevice, st));
        TV_CUDA(cudaMemcpyAsync(x2.p, amx.p, nint * 4, cudaMemcpyDeviceToDevice, st));
        TV_CUDA(cudaStreamSynchronize(st));
      }
      acode = std::move(c2); asum = std::move(s2); acnt = std::move(n2); amn = std::move(m2); amx = std::move(x2);
    }
    const NodePtrs arch{acode.p, asum.p, acnt.p, amn.p, amx.p};
    if (nsorted >= 0) {
      k_split<true><<<blocks_for(N), TPB, 0, st>>>(A.ptrs(), N, marks.p, pos.p, A.ptrs(), newlist.p, hkeys.p,
                                                   hcap - 1, Bloom{bloomw.p, hcap / 8 - 1}, counters.p, arch, nint);
      TV_LAUNCH();
    } else {
      k_split<false><<<blocks_for(N), TPB, 0, st>>>(A.ptrs(), N, marks.p, pos.p, B.ptrs(), newlist.p, hkeys.p,
                                                    hcap - 1, Bloom{bloomw.p, hcap / 8 - 1}, counters.p, arch, nint);
      TV_LAUNCH();
      std::swap(A, B);
    }
    N += M;
    nint += M;
    stats_and_criterion(A, newlist.p, 2 * M, q.p, C, scan, chunks, off, owner, desc, st, sms, pp, lk);
  }

  bloomw.alloc(0); marks.alloc(0); pos.alloc(0); newlist.alloc(0); chunks.alloc(0); off.alloc(0); owner.alloc(0);
  desc.alloc(0); B = Leaves();

  // ---- the leaves in code order, in exact-size arrays ----
  DevBuf<unsigned long long> codes(N), sum(N), scratch(4);
  DevBuf<int4> verts(3 * N);
  DevBuf<uint8_t> tag(N);
  DevBuf<uint32_t> cnt(N), mn(N), mx(N);
  {
    const long long ns = nsorted < 0 ? N : nsorted, nt = N - ns;
    DevBuf<unsigned long long> tcode(nt > 0 ? nt : 1);
    DevBuf<uint32_t> tiota(nt > 0 ? nt : 1), tperm(nt > 0 ? nt : 1);
    if (nt > 0) {
      k_iota32<<<blocks_for(nt), TPB, 0, st>>>(tiota.p, nt);
      TV_LAUNCH();
      size_t bytes = 0;
      TV_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, A.code.p + ns, tcode.p, tiota.p, tperm.p, nt, 0, 64, st));
      DevBuf<char> tmp(bytes + 16);
      TV_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, bytes, A.code.p + ns, tcode.p, tiota.p, tperm.p, nt, 0, 64, st));
    }
    const LeafPtrs D{verts.p, codes.p, tag.p, cnt.p, mn.p, mx.p, sum.p, nullptr};
    k_place_leaves<<<blocks_for(N), TPB, 0, st>>>(A.ptrs(), ns, nt, tcode.p, tperm.p, D);
    TV_LAUNCH();
  }
  A = Leaves();
  const LeafPtrs F{verts.p, codes.p, tag.p, cnt.p, mn.p, mx.p, sum.p, nullptr};

  // ---- interior-node statistics sorted by code (for rebuilds) ----
  DevBuf<unsigned long long> ncode(nint > 0 ? nint : 1), nsum(nint > 0 ? nint : 1);
  DevBuf<uint32_t> ncnt(nint > 0 ? nint : 1), nmn(nint > 0 ? nint : 1), nmx(nint > 0 ? nint : 1);
  if (nint > 0) {
    DevBuf<unsigned long long> iota(nint), perm(nint);
    k_iota<<<blocks_for(nint), TPB, 0, st>>>(iota.p, nint);
    TV_LAUNCH();
    size_t bytes = 0;
    TV_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, acode.p, ncode.p, iota.p, perm.p, nint, 0, 64, st));
    DevBuf<char> tmp(bytes + 16);
    TV_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, bytes, acode.p, ncode.p, iota.p, perm.p, nint, 0, 64, st));
    const NodePtrs src{acode.p, asum.p, acnt.p, amn.p, amx.p}, dst{ncode.p, nsum.p, ncnt.p, nmn.p, nmx.p};
    k_gather_nodes<<<blocks_for(nint), TPB, 0, st>>>(src, perm.p, nint, dst);
    TV_LAUNCH();
    TV_CUDA(cudaStreamSynchronize(st));
  }
  acode.alloc(0); asum.alloc(0); acnt.alloc(0); amn.alloc(0); amx.alloc(0);

  // ---- finalize: neighbours, orientations, planes, densities, records ----
  const long long NF = 4 * N;
  DevBuf<uint32_t> fnbr(NF);
  DevBuf<uint4> rec(2 * N);
  DevBuf<float> maj(N);
  DevBuf<int> err(2);
  TV_CUDA(cudaMemsetAsync(err.p, 0, 8, st));
  {
    // face keys: vertex sums below 3 C 2^K per axis
    int fb = 1;
    for (int a = 0; a < 3; ++a)
      while ((1ll << fb) <= 3ll * ((long long)g.C[a] << g.K)) ++fb;
    DevBuf<unsigned long long> fk(NF), fks(NF);
    DevBuf<uint32_t> fid(NF), fids(NF);
    k_face_keys<<<blocks_for(N), TPB, 0, st>>>(F.v, N, fb, fk.p, fid.p);
    TV_LAUNCH();
    size_t bytes = 0;
    TV_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, fk.p, fks.p, fid.p, fids.p, NF, 0, 3 * fb, st));
    DevBuf<char> tmp(bytes + 16);
    TV_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, bytes, fk.p, fks.p, fid.p, fids.p, NF, 0, 3 * fb, st));
    k_face_pairs<<<blocks_for(NF), TPB, 0, st>>>(fks.p, fids.p, NF, fnbr.p, err.p);
    TV_LAUNCH();
  }
  k_finalize<<<blocks_for(N), TPB, 0, st>>>(F, N, g, fmt, fnbr.p, rec.p, maj.p, err.p);
  TV_LAUNCH();
  int herr = 0;
  TV_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st));
  TV_CUDA(cudaStreamSynchronize(st));
  if (herr) return TG_EGRID;

  TV_CUDA(cudaMemsetAsync(scratch.p, 0, 32, st));
  int depth_reached = 0;
  TV_CUDA(cudaMemsetAsync(err.p + 1, 0, 4, st));
  k_code_depth<<<blocks_for(N), TPB, 0, st>>>(codes.p, N, err.p + 1);
  TV_LAUNCH();
  TV_CUDA(cudaMemcpyAsync(&depth_reached, err.p + 1, 4, cudaMemcpyDeviceToHost, st));
  TV_CUDA(cudaStreamSynchronize(st));

  G.device = dev;
  G.n = N;
  G.K = g.K;
  G.max_depth = depth_reached;
  G.rounds = round;
  G.fmt = fmt;
  for (int a = 0; a < 3; ++a) { G.C[a] = g.C[a]; G.box_min[a] = vol->box_min[a]; }
  G.nvox[0] = g.nx; G.nvox[1] = g.ny; G.nvox[2] = g.nz;
  G.n_per_cube = n;
  G.voxel_size = vol->voxel_size;
  G.cube = cube;
  G.rec = rec.release();
  G.majorant = maj.release();
  G.codes = codes.release();
  G.sum = sum.release();
  G.verts = reinterpret_cast<int32_t*>(verts.release());
  G.tag = tag.release();
  G.count = cnt.release();
  G.qmin = mn.release();
  G.qmax = mx.release();
  G.scratch = scratch.release();
  G.n_nodes = nint;
  G.node_code = ncode.release();
  G.node_sum = nsum.release();
  G.node_cnt = ncnt.release();
  G.node_mn = nmn.release();
  G.node_mx = nmx.release();
  build_locator(G, st);
  TV_CUDA(cudaStreamSynchronize(st));
  return TG_OK;
}

// Per-tet channels and voxel majorants of a built grid (see tg_grid_channels).
int grid_channels(GridImpl& G, const float* density, const float* temperature, const float* albedo,
                  const float* aniso, cudaStream_t st) {
  if (!G.verts || G.n == 0) return TG_EINVAL;
  Geo g;
  g.nx = G.nvox[0]; g.ny = G.nvox[1]; g.nz = G.nvox[2];
  g.n = G.n_per_cube;
  int m = 0;
  while ((1 << m) < g.n) ++m;
  g.m = m;
  g.K = G.K;
  g.max_depth = G.max_depth;
  for (int a = 0; a < 3; ++a) g.C[a] = G.C[a];
  g.h = 1 << (g.K - m - 1);
  int dev = 0, sms = 0;
  TV_CUDA(cudaGetDevice(&dev));
  TV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long N = G.n;
  const long long nvox = (long long)g.nx * g.ny * g.nz;
  DevBuf<uint32_t> q(nvox), cnt(N), mn(N), mx(N);
  DevBuf<unsigned long long> sum(N), chunks, off;
  DevBuf<int> owner;
  DevBuf<ScanDesc> desc;
  DevBuf<float> chan((size_t)N * 4), vmaj(N);
  TV_CUDA(cudaMemsetAsync(chan.p, 0, (size_t)N * 16, st));
  LeafPtrs L{reinterpret_cast<int4*>(G.verts), G.codes, nullptr, cnt.p, mn.p, mx.p, sum.p, nullptr};
  Scanner scan;
  const unsigned qblocks = (unsigned)std::min<long long>(blocks_for(nvox), (long long)sms * 32);
  auto leaf_stats = [&](bool box) {
    chunks.ensure(N + 1);
    off.ensure(N + 1);
    desc.ensure(N);
    const bool qr = quad_rows(g, q.p);
    if (box && qr) k_stats_prep<true, true><<<blocks_for(N), TPB, 0, st>>>(L, nullptr, N, g, chunks.p, desc.p, q.p);
    else if (box) k_stats_prep<true, false><<<blocks_for(N), TPB, 0, st>>>(L, nullptr, N, g, chunks.p, desc.p, q.p);
    else if (qr) k_stats_prep<false, true><<<blocks_for(N), TPB, 0, st>>>(L, nullptr, N, g, chunks.p, desc.p, q.p);
    else k_stats_prep<false, false><<<blocks_for(N), TPB, 0, st>>>(L, nullptr, N, g, chunks.p, desc.p, q.p);
    TV_LAUNCH();
    TV_CUDA(cudaMemsetAsync(chunks.p + N, 0, sizeof(unsigned long long), st));
    scan.exclusive(chunks.p, off.p, N + 1, st);
    unsigned long long total = 0;
    TV_CUDA(cudaMemcpyAsync(&total, off.p + N, sizeof total, cudaMemcpyDeviceToHost, st));
    TV_CUDA(cudaStreamSynchronize(st));
    if (total) {
      if (box) stats_scan<true>(L, desc.p, N, off.p, total, owner, q.p, g, sms, st);
      else stats_scan<false>(L, desc.p, N, off.p, total, owner, q.p, g, sms, st);
    }
  };
  const float* vols[3] = {temperature, albedo, aniso};
  int mask = 8;
  for (int c = 0; c < 3; ++c) {
    if (!vols[c]) continue;
    k_quantize<<<qblocks, TPB, 0, st>>>(vols[c], q.p, nvox);
    TV_LAUNCH();
    leaf_stats(false);
    k_channel_store<<<blocks_for(N), TPB, 0, st>>>(L, N, q.p, g, c, chan.p);
    TV_LAUNCH();
    mask |= 1 << c;
  }
  k_quantize<<<qblocks, TPB, 0, st>>>(density, q.p, nvox);
  TV_LAUNCH();
  leaf_stats(true);
  k_vmaj_store<<<blocks_for(N), TPB, 0, st>>>(L, N, vmaj.p);
  TV_LAUNCH();
  TV_CUDA(cudaStreamSynchronize(st));
  if (G.chan) cudaFree(G.chan);
  if (G.vmaj) cudaFree(G.vmaj);
  G.chan = reinterpret_cast<float4*>(chan.release());
  G.vmaj = vmaj.release();
  G.chan_mask = mask;
  return TG_OK;
}

}  // namespace tv

extern "C" int tg_grid_channels(tg_grid* g, const float* density, const float* temperature, const float* albedo,
                                const float* aniso, void* cuda_stream) {
  if (!g || !density) return TG_EINVAL;
  try {
    tv::AllocScope scope((cudaStream_t)cuda_stream, tv::build_pool());
    return tv::grid_channels(g->impl, density, temperature, albedo, aniso, (cudaStream_t)cuda_stream);
  } catch (const tv::Error& e) {
    return e.code;
  } catch (const std::bad_alloc&) {
    return TG_ENOMEM;
  }
}

extern "C" int tg_grid_export_channels(const tg_grid* g, float* chan, float* vmaj, void* cuda_stream) {
  if (!g) return TG_EINVAL;
  const tv::GridImpl& G = g->impl;
  if (!G.chan_mask) return TG_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (chan && cudaMemcpyAsync(chan, G.chan, (size_t)G.n * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TG_ECUDA;
  if (vmaj && cudaMemcpyAsync(vmaj, G.vmaj, (size_t)G.n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return TG_ECUDA;
  return TG_OK;
}

// The volume a build reads: device memory, or page-locked (pinned) host memory
// that the device addresses directly -- read once, by the quantisation kernel.
// Pageable host memory is refused before any kernel could touch it.
static int build_volume_pointer(const float* p, const float** dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return TG_ECUDA;
  }
  if (a.type == cudaMemoryTypeUnregistered) return TG_EINVAL;
  *dev = a.devicePointer ? static_cast<const float*>(a.devicePointer) : p;
  return TG_OK;
}

extern "C" int leb_build(const float* density, const tg_volume_desc* vol, const tg_camera* cam,
                         float target_footprint_px, float variation_threshold, int32_t max_depth,
                         int32_t density_format, void* cuda_stream, tg_grid** out) {
  if (!density || !vol || !out || vol->nx <= 0 || vol->ny <= 0 || vol->nz <= 0 || !(vol->voxel_size > 0) ||
      max_depth < 0 || max_depth > 50 || density_format < 0 || density_format > 2)
    return TG_EINVAL;
  if ((long long)vol->nx * vol->ny * vol->nz >= (1ll << 34)) return TG_EINVAL;
  if (cam && !tv::camera_ok(cam)) return TG_EINVAL;
  const int vs = build_volume_pointer(density, &density);
  if (vs != TG_OK) return vs;
  tg_grid* g = new (std::nothrow) tg_grid();
  if (!g) return TG_ENOMEM;
  int st;
  try {
    tv::AllocScope scope((cudaStream_t)cuda_stream, tv::build_pool());
    st = tv::build_grid(density, vol, cam, target_footprint_px, variation_threshold, max_depth, density_format,
                        (cudaStream_t)cuda_stream, g->impl, nullptr);
  } catch (const tv::Error& e) {
    st = e.code;
  } catch (const std::bad_alloc&) {
    st = TG_ENOMEM;
  }
  if (st != TG_OK) {
    delete g;
    return st;
  }
  *out = g;
  return TG_OK;
}

extern "C" int leb_rebuild(const tg_grid* prev, const float* density, const tg_volume_desc* vol,
                           const tg_camera* cam, float target_footprint_px, float variation_threshold,
                           int32_t max_depth, int32_t density_format, void* cuda_stream, tg_grid** out) {
  if (!prev || !density || !vol || !out || vol->nx <= 0 || vol->ny <= 0 || vol->nz <= 0 ||
      !(vol->voxel_size > 0) || max_depth < 0 || max_depth > 50 || density_format < 0 || density_format > 2)
    return TG_EINVAL;
  if ((long long)vol->nx * vol->ny * vol->nz >= (1ll << 34)) return TG_EINVAL;
  if (cam && !tv::camera_ok(cam)) return TG_EINVAL;
  const int vs = build_volume_pointer(density, &density);
  if (vs != TG_OK) return vs;
  tg_grid* g = new (std::nothrow) tg_grid();
  if (!g) return TG_ENOMEM;
  int st;
  try {
    tv::AllocScope scope((cudaStream_t)cuda_stream, tv::build_pool());
    st = tv::build_grid(density, vol, cam, target_footprint_px, variation_threshold, max_depth, density_format,
                        (cudaStream_t)cuda_stream, g->impl, &prev->impl);
  } catch (const tv::Error& e) {
    st = e.code;
  } catch (const std::bad_alloc&) {
    st = TG_ENOMEM;
  }
  if (st != TG_OK) {
    delete g;
    return st;
  }
  *out = g;
  return TG_OK;
}
