// CPU oracle of the adaptive tetrahedral-grid volumetric path tracer of
// Benyoub & Dupuy, "Adaptive Tetrahedral Grids for Volumetric Path-Tracing"
// (SIGGRAPH Talks 2025).
//
// TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
// benchmark's CPU-baseline leg, never by the product path.  Plain and slow on
// purpose; shares nothing with the CUDA library.  fp64 throughout, compiled
// with -ffp-contract=off so every product and sum is rounded on its own.
//
// Where the paper leaves a choice open the readings below are used (each is
// restated where it is implemented):
//  * roots: six Kuhn tetrahedra per unit cube (depth 2 of this hierarchy is the
//    paper's 24 "one per halfedge" tetrahedra of the control cube, Sec. 2);
//  * bisection: Maubach's tagged rule (Sec. 2 cites Maubach 1995);
//  * propagation: a leaf with a vertex at the midpoint of one of its edges is
//    bisected, until no such leaf remains (the "deterministic rule" of Sec. 2);
//  * D = voxel centres inside the closed tetrahedron; if none, the voxel that
//    holds the centroid;
//  * free paths are optical depths consumed across cells (regular tracking),
//    exact for the per-tetrahedron constant density of Sec. 3;
//  * Henyey-Greenstein phase function, sun next-event estimation, constant
//    environment on escape, Philox4x32-10 random numbers (not in the paper).
//
// Pins (tests/test_oracle_*.py) tie each part to something other than this
// file: Philox to cuRAND's generator; roots, bisection, closure and statistics
// to the paper's control cube (tests/golden), exact volumes, conformity,
// brute-force voxel sums and a random-order closure; the walk to clipping the
// ray with every tetrahedron; free flights to the exponential law (KS);
// transmittance, single scattering and the throughput rule to closed forms; HG
// sampling to its density; the camera model to an absorbing-block image.
// Partly pinned: the camera criterion's footprint threshold (bounds and
// monotonicity only).  Parity unpinned: multiple scattering in a heterogeneous
// medium as a whole has no closed form; beyond its pinned steps it is checked
// only by the white furnace and by agreement with the DDA tracker.

#include "oracle.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef __int128 i128;
typedef unsigned __int128 u128;

const int OK = 0, EINVAL_ = -1, ENOMEM_ = -2, ESTEPLIMIT_ = -4, EROUNDLIMIT_ = -5, EGRID_ = -6;
const int64_t STEP_LIMIT = 1 << 20;   // cells per segment before a walk gives up
const double PI = 3.14159265358979323846;

// ============================================================================
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor S-box on a 4x32-bit counter, key bumped by the Weyl constants
// between rounds.
// ============================================================================
void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Random number of a path: key = (seed lo, seed hi ^ pixel), counter =
// (sample, slot / 4, stream, 0), word slot % 4; u = (word >> 8) * 2^-24 in [0, 1).
// Stream 0: 0, 1 pixel jitter; 2 + 3b free path of bounce b; 3 + 3b, 4 + 3b phase.
// Streams 1 + 2b and 2 + 2b: the k-th delta-tracking draw of the free flight and
// of the shadow ray of bounce b (slot k).
double uniform(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t slot, uint32_t stream = 0) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ pixel};
  uint32_t ctr[4] = {sample, slot / 4, stream, 0};
  uint32_t out[4];
  philox(ctr, key, out);
  return (double)(out[slot % 4] >> 8) * (1.0 / 16777216.0);
}

// ============================================================================
// Vectors
// ============================================================================
struct V3 { double x, y, z; };
V3 v3(double x, double y, double z) { V3 r = {x, y, z}; return r; }
V3 add(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
V3 sub(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
V3 mul(V3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
double dot(V3 a, V3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
V3 cross(V3 a, V3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
V3 normalize(V3 a) { double l = std::sqrt(dot(a, a)); return v3(a.x / l, a.y / l, a.z / l); }
V3 from_f(const float* p) { return v3((double)p[0], (double)p[1], (double)p[2]); }

// ============================================================================
// Domain: the volume box is tiled by unit cubes of n^3 voxels (n the largest
// power of two dividing all three voxel counts).  Grid space measures lengths
// in cubes; vertex coordinates are integers in units of 2^-K cube.
// ============================================================================
struct Domain {
  int nx, ny, nz, n, m, C[3], K, max_depth;
  V3 box_min;
  double voxel_size, cube;   // world size of a voxel and of a cube
};

int make_domain(int nx, int ny, int nz, const float box_min[3], float voxel_size, int max_depth, Domain* d) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || !(voxel_size > 0) || max_depth < 0 || max_depth > 50) return EINVAL_;
  int n = 1, m = 0;
  while (nx % (2 * n) == 0 && ny % (2 * n) == 0 && nz % (2 * n) == 0 && n < (1 << 18)) { n *= 2; ++m; }
  d->nx = nx; d->ny = ny; d->nz = nz; d->n = n; d->m = m;
  d->C[0] = nx / n; d->C[1] = ny / n; d->C[2] = nz / n;
  int kd = (max_depth + 2) / 3 + 1;            // ceil(max_depth/3) + 1: every edge midpoint is a lattice point
  d->K = std::max(kd, m + 1);                  // and every voxel centre too
  for (int a = 0; a < 3; ++a)
    if (((int64_t)d->C[a] << d->K) >= (1 << 20)) return EINVAL_;
  if ((int64_t)d->C[0] * d->C[1] * d->C[2] * 6 > 256) return EINVAL_;   // root id fits 8 bits of the code
  d->max_depth = max_depth;
  d->box_min = from_f(box_min);
  d->voxel_size = (double)voxel_size;
  d->cube = d->voxel_size * (double)n;
  return OK;
}

// ============================================================================
// Sec. 2, LEB.  A tetrahedron is (x0, x1, x2, x3) with tag k in {1,2,3}.
// Maubach's bisection cuts the edge x0-xk at its midpoint z; the children are
// (x0..x_{k-1}, z, x_{k+1}..x3) and (x1..xk, z, x_{k+1}..x3), both with tag
// k-1 (or 3 when k = 1).  Its code is (root, depth, path of child bits).
// ============================================================================
struct Tet {
  int32_t x[4][3];
  int32_t tag, depth;
  uint32_t root;
  uint64_t path;                 // `depth` bits, the first bisection most significant
};

uint64_t code_of(const Tet& t) {
  // root above the path bits left-aligned below it (depth-first pre-order), depth in the low 6 bits
  uint64_t p = t.depth ? (t.path << (56 - t.depth)) & ((1ull << 56) - 1) : 0;
  return ((uint64_t)t.root << 56) | p | (uint64_t)t.depth;
}

Tet child(const Tet& T, int which) {
  int k = T.tag;
  int32_t z[3];
  for (int a = 0; a < 3; ++a) z[a] = (T.x[0][a] + T.x[k][a]) / 2;   // exact: the sum is even by choice of K
  Tet C;
  int i = 0;
  if (which == 0) for (int j = 0; j < k; ++j) std::memcpy(C.x[i++], T.x[j], sizeof z);
  else            for (int j = 1; j <= k; ++j) std::memcpy(C.x[i++], T.x[j], sizeof z);
  std::memcpy(C.x[i++], z, sizeof z);
  for (int j = k + 1; j < 4; ++j) std::memcpy(C.x[i++], T.x[j], sizeof z);
  C.tag = k > 1 ? k - 1 : 3;
  C.depth = T.depth + 1;
  C.root = T.root;
  C.path = (T.path << 1) | (uint64_t)which;
  return C;
}

// Six Kuhn tetrahedra of cube (cx, cy, cz): x0 the low corner, x3 the high corner,
// x1 and x2 reached by stepping along the axes in the order of a permutation;
// permutations in lexicographic order.  Root id = 6 * cube index + permutation.
const int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

Tet root_tet(const Domain& D, int cx, int cy, int cz, int perm) {
  Tet T;
  int32_t s = 1 << D.K;
  int32_t v[3] = {cx * s, cy * s, cz * s};
  std::memcpy(T.x[0], v, sizeof v);
  for (int j = 0; j < 3; ++j) { v[PERMS[perm][j]] += s; std::memcpy(T.x[j + 1], v, sizeof v); }
  T.tag = 3; T.depth = 0; T.path = 0;
  T.root = (uint32_t)(((cz * D.C[1] + cy) * D.C[0] + cx) * 6 + perm);
  return T;
}

// exact orientation determinant det(b - a, c - a, d - a)
i128 orient(const int64_t a[3], const int64_t b[3], const int64_t c[3], const int64_t d[3]) {
  i128 b0 = b[0] - a[0], b1 = b[1] - a[1], b2 = b[2] - a[2];
  i128 c0 = c[0] - a[0], c1 = c[1] - a[1], c2 = c[2] - a[2];
  i128 d0 = d[0] - a[0], d1 = d[1] - a[1], d2 = d[2] - a[2];
  return b0 * (c1 * d2 - c2 * d1) - b1 * (c0 * d2 - c2 * d0) + b2 * (c0 * d1 - c1 * d0);
}
int sgn(i128 v) { return (v > 0) - (v < 0); }

// Point-in-tetrahedron test for the closed tetrahedron: p is inside when, for
// every face, it lies on the same side of the face plane as the opposite vertex,
// or on the plane.
struct TetTest {
  int64_t q[4][3][3];   // the three vertices of face f
  int sref[4];          // side of the opposite vertex
  explicit TetTest(const Tet& T) {
    int64_t X[4][3];
    for (int i = 0; i < 4; ++i) for (int a = 0; a < 3; ++a) X[i][a] = T.x[i][a];
    for (int f = 0; f < 4; ++f) {
      int j = 0;
      for (int i = 0; i < 4; ++i) if (i != f) { for (int a = 0; a < 3; ++a) q[f][j][a] = X[i][a]; ++j; }
      sref[f] = sgn(orient(q[f][0], q[f][1], q[f][2], X[f]));
    }
  }
  bool inside(const int64_t p[3]) const {
    for (int f = 0; f < 4; ++f) {
      int sp = sgn(orient(q[f][0], q[f][1], q[f][2], p));
      if (sp != 0 && sp != sref[f]) return false;
    }
    return true;
  }
};

int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

// ============================================================================
// Sec. 2, subdivision criteria.
// ============================================================================
struct Volume {
  const Domain* D;
  std::vector<uint32_t> q;    // round(rho * 2^24), clamped to [0, 2^24]
};

void quantise(const float* density, const Domain& D, Volume* V) {
  size_t N = (size_t)D.nx * D.ny * D.nz;
  V->D = &D;
  V->q.resize(N);
  for (size_t i = 0; i < N; ++i) {
    double r = (double)density[i];
    double s = std::nearbyint(r * 16777216.0);
    if (!(s > 0)) s = 0;                      // negatives and NaN become empty space
    if (s > 16777216.0) s = 16777216.0;
    V->q[i] = (uint32_t)s;
  }
}

struct Stats { uint32_t count, qmin, qmax; uint64_t sum; };

// D = the voxels whose centres lie in the closed tetrahedron; if there are none,
// the voxel holding the centroid.
Stats density_stats(const Volume& V, const Tet& T) {
  const Domain& D = *V.D;
  int64_t h = (int64_t)1 << (D.K - D.m - 1);     // voxel i has centre (2i + 1) h
  int dims[3] = {D.nx, D.ny, D.nz};
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    int64_t mn = T.x[0][a], mx = T.x[0][a];
    for (int i = 1; i < 4; ++i) { mn = std::min<int64_t>(mn, T.x[i][a]); mx = std::max<int64_t>(mx, T.x[i][a]); }
    lo[a] = std::max<int64_t>(0, ceil_div(mn - h, 2 * h));
    hi[a] = std::min<int64_t>(dims[a] - 1, floor_div(mx - h, 2 * h));
  }
  Stats s = {0, 0xFFFFFFFFu, 0, 0};
  TetTest inside(T);
  for (int64_t k = lo[2]; k <= hi[2]; ++k)
    for (int64_t j = lo[1]; j <= hi[1]; ++j)
      for (int64_t i = lo[0]; i <= hi[0]; ++i) {
        int64_t p[3] = {(2 * i + 1) * h, (2 * j + 1) * h, (2 * k + 1) * h};
        if (!inside.inside(p)) continue;
        uint32_t v = V.q[((size_t)k * D.ny + j) * D.nx + i];
        s.count++; s.sum += v; s.qmin = std::min(s.qmin, v); s.qmax = std::max(s.qmax, v);
      }
  if (s.count == 0) {
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
      int64_t sx = (int64_t)T.x[0][a] + T.x[1][a] + T.x[2][a] + T.x[3][a];  // 4 * centroid
      int64_t c = sx >> (D.K + 2 - D.m);                                    // floor(centroid * n)
      idx[a] = std::min<int64_t>(std::max<int64_t>(c, 0), dims[a] - 1);
    }
    uint32_t v = V.q[((size_t)idx[2] * D.ny + idx[1]) * D.nx + idx[0]];
    s.count = 1; s.sum = v; s.qmin = v; s.qmax = v;
  }
  return s;
}

// Camera of the criterion, everything in grid space and fp64.
struct CamCrit {
  bool on;
  V3 eye, f, r, u;
  double tanF, tanX, near_g, thr;
};

const double HALF_DEG = 0.0087266462599716478846;   // pi / 360

CamCrit camera_criterion(const orc_camera* cam, float footprint_px, const Domain& D) {
  CamCrit c;
  std::memset(&c, 0, sizeof c);
  c.on = cam != nullptr && footprint_px > 0;
  if (!c.on) return c;
  V3 E = from_f(cam->pos), T = from_f(cam->target), U = from_f(cam->up);
  V3 eg = sub(E, D.box_min);
  c.eye = v3(eg.x / D.cube, eg.y / D.cube, eg.z / D.cube);
  c.f = normalize(sub(T, E));
  c.r = normalize(cross(c.f, U));
  c.u = normalize(cross(c.r, c.f));
  c.tanF = std::tan((double)cam->fov_y_deg * HALF_DEG);
  c.tanX = c.tanF * ((double)cam->width / (double)cam->height);
  c.near_g = 1e-3 / D.cube;                       // near plane 1e-3 world units ahead of the eye
  c.thr = (2.0 * c.tanF / (double)cam->height) * (double)footprint_px;   // world length of F pixels at unit depth
  return c;
}

// "prevent subdivision for tetrahedrons that either lie outside of the view
// frustum, or project into less than one pixel" (Sec. 2, criterion 2):
// outside = all four vertices strictly beyond one frustum plane (near or side);
// projected size = longest edge / (pixel length at the nearest vertex depth).
bool camera_allows_split(const CamCrit& c, const Domain& D, const Tet& T) {
  if (!c.on) return true;
  const double s = std::ldexp(1.0, -D.K);
  double xc[4], yc[4], zc[4];
  for (int i = 0; i < 4; ++i) {
    V3 p = v3((double)T.x[i][0] * s, (double)T.x[i][1] * s, (double)T.x[i][2] * s);
    V3 d = sub(p, c.eye);
    zc[i] = dot(d, c.f); xc[i] = dot(d, c.r); yc[i] = dot(d, c.u);
  }
  bool all_near = true, all_r = true, all_l = true, all_t = true, all_b = true;
  for (int i = 0; i < 4; ++i) {
    double ax = zc[i] * c.tanX, ay = zc[i] * c.tanF;
    all_near = all_near && zc[i] < c.near_g;
    all_r = all_r && xc[i] > ax;
    all_l = all_l && xc[i] < -ax;
    all_t = all_t && yc[i] > ay;
    all_b = all_b && yc[i] < -ay;
  }
  if (all_near || all_r || all_l || all_t || all_b) return false;
  double zmin = std::min(std::min(zc[0], zc[1]), std::min(zc[2], zc[3]));
  if (zmin < c.near_g) zmin = c.near_g;
  int64_t L2 = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) {
      int64_t e = 0;
      for (int a = 0; a < 3; ++a) { int64_t t = (int64_t)T.x[i][a] - T.x[j][a]; e += t * t; }
      L2 = std::max(L2, e);
    }
  double lmax2 = (double)L2 * s * s;
  double pix = c.thr * zmin;
  return lmax2 > pix * pix;
}

struct Criterion {
  const Domain* D;
  const Volume* V;
  CamCrit cam;
  bool var_on;
  int64_t theta_q16;     // theta as a multiple of 2^-16
};

// "(max(D) - min(D)) / mean(D)" above the threshold (Sec. 2, criterion 1),
// evaluated exactly as (max - min) * |D| * 2^16 > theta_q16 * sum(D); a mean of
// zero gives no split.
bool variation_allows_split(const Criterion& C, const Stats& s) {
  if (!C.var_on) return true;
  u128 lhs = (u128)(s.qmax - s.qmin) * (u128)s.count * (u128)65536;
  u128 rhs = (u128)(uint64_t)C.theta_q16 * (u128)s.sum;
  return lhs > rhs;
}

bool split(const Criterion& C, const Tet& T, const Stats& s) {
  if (T.depth >= C.D->max_depth) return false;
  if (!variation_allows_split(C, s)) return false;
  return camera_allows_split(C.cam, *C.D, T);
}

// ============================================================================
// Storage of the per-tetrahedron density (Sec. 3: one density value per cell):
// the mean of D rounded once to fp32, then to bf16 or fp16 (round to nearest even).
// ============================================================================
float to_bf16(float x) {
  uint32_t b; std::memcpy(&b, &x, 4);
  if ((b & 0x7F800000u) == 0x7F800000u) return x;
  uint32_t lsb = (b >> 16) & 1u;
  b = (b + 0x7FFFu + lsb) & 0xFFFF0000u;
  float y; std::memcpy(&y, &b, 4); return y;
}

float to_fp16(float x) {
  // round x (>= 0, <= 1 here) to the nearest binary16 value, ties to even, via exact fp64 steps
  double v = (double)x;
  if (v == 0) return 0.0f;
  int e; std::frexp(v, &e);                 // v = f * 2^e, f in [0.5, 1)
  int exp_unbiased = e - 1;                 // v in [2^eu, 2^(eu+1))
  int q = std::max(exp_unbiased, -14) - 10; // spacing of binary16 values at v
  double scaled = std::ldexp(v, -q);
  double r = std::nearbyint(scaled);        // ties to even in the default rounding mode
  return (float)std::ldexp(r, q);
}

float stored_density(const Stats& s, int fmt) {
  double mean = (double)s.sum / ((double)s.count * 16777216.0);
  float f = (float)mean;
  if (fmt == 1) return to_bf16(f);
  if (fmt == 2) return to_fp16(f);
  return f;
}

// ============================================================================
// Face normals (Sec. 3: 18 orientations).  The 9 unsigned plane normals; a face
// id is p + 9 * (outward normal = -P[p]).
// ============================================================================
const int P9[9][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
                      {0, 1, 1}, {0, 1, -1}, {1, 0, 1}, {1, 0, -1}};

int face_normal_id(const Tet& T, int f) {
  int64_t q[3][3]; int j = 0;
  for (int i = 0; i < 4; ++i) if (i != f) { for (int a = 0; a < 3; ++a) q[j][a] = T.x[i][a]; ++j; }
  int64_t u[3], v[3], w[3];
  for (int a = 0; a < 3; ++a) { u[a] = q[1][a] - q[0][a]; v[a] = q[2][a] - q[0][a]; w[a] = T.x[f][a] - q[0][a]; }
  int64_t nrm[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  if (nrm[0] * w[0] + nrm[1] * w[1] + nrm[2] * w[2] > 0) for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
  int64_t mx = std::max(std::llabs(nrm[0]), std::max(std::llabs(nrm[1]), std::llabs(nrm[2])));
  if (mx == 0) return -1;
  int c[3];
  for (int a = 0; a < 3; ++a) {
    if (nrm[a] == 0) c[a] = 0;
    else if (std::llabs(nrm[a]) == mx) c[a] = nrm[a] > 0 ? 1 : -1;
    else return -1;                                  // not one of the 18 orientations
  }
  for (int p = 0; p < 9; ++p) {
    if (c[0] == P9[p][0] && c[1] == P9[p][1] && c[2] == P9[p][2]) return p;
    if (c[0] == -P9[p][0] && c[1] == -P9[p][1] && c[2] == -P9[p][2]) return p + 9;
  }
  return -1;
}

// ============================================================================
// The built grid.
// ============================================================================
uint64_t vkey(const int32_t v[3]) {
  return (uint64_t)v[0] | ((uint64_t)v[1] << 21) | ((uint64_t)v[2] << 42);
}

}  // namespace

struct orc_grid {
  Domain D;
  int density_format;
  int rounds, depth_reached;
  std::vector<Tet> tets;          // sorted by code
  std::vector<uint64_t> codes;
  std::vector<Stats> stats;
  std::vector<std::array<int32_t, 4>> nbr;
  std::vector<std::array<uint8_t, 4>> nid;
  std::vector<std::array<float, 4>> plane;
  std::vector<float> rho, rho_max;
  std::unordered_map<uint64_t, int32_t> index_of_code;
  // extra per-tet channels (orc_grid_channels): temperature, albedo, g; the voxel majorant
  int channel_mask = 0;
  std::vector<std::array<float, 3>> chan;
  std::vector<float> vmaj;
};

namespace {

int set_threads(int n) {
#ifdef _OPENMP
  return n > 0 ? n : omp_get_max_threads();
#else
  (void)n; return 1;
#endif
}

// Sec. 2: bisect every leaf that the criterion selects or that has a vertex of
// the current grid at the midpoint of one of its edges (a hanging vertex),
// until no leaf is selected.  The fixed point does not depend on the order in
// which leaves are split: it is the coarsest conforming grid in which no leaf
// satisfies the criterion.
int build_grid(const Volume& V, const Criterion& C, int max_rounds, int nthreads, orc_grid* G) {
  const Domain& D = *V.D;
  std::vector<Tet> leaves;
  for (int cz = 0; cz < D.C[2]; ++cz)
    for (int cy = 0; cy < D.C[1]; ++cy)
      for (int cx = 0; cx < D.C[0]; ++cx)
        for (int p = 0; p < 6; ++p) leaves.push_back(root_tet(D, cx, cy, cz, p));
  std::vector<Stats> st(leaves.size());
  std::vector<char> crit(leaves.size());
  {
    // one root at a time per thread: each root's statistics scan a whole cube of voxels
    int nt0 = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt0)
    for (int64_t i = 0; i < (int64_t)leaves.size(); ++i) {
      st[i] = density_stats(V, leaves[i]);
      crit[i] = split(C, leaves[i], st[i]);
    }
  }
  std::unordered_set<uint64_t> verts;
  for (const Tet& t : leaves) for (int i = 0; i < 4; ++i) verts.insert(vkey(t.x[i]));

  int round = 0;
  for (;; ++round) {
    std::vector<char> mark(leaves.size());
    int64_t nmark = 0;
    int nt = set_threads(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt) reduction(+ : nmark)
    for (int64_t i = 0; i < (int64_t)leaves.size(); ++i) {
      bool m = crit[i] != 0;
      for (int a = 0; a < 4 && !m; ++a)
        for (int b = a + 1; b < 4 && !m; ++b) {
          int32_t s[3]; bool even = true;
          for (int c = 0; c < 3; ++c) { s[c] = leaves[i].x[a][c] + leaves[i].x[b][c]; even = even && (s[c] % 2 == 0); }
          if (!even) continue;                 // a midpoint off the lattice cannot be a vertex
          int32_t mid[3] = {s[0] / 2, s[1] / 2, s[2] / 2};
          m = verts.count(vkey(mid)) != 0;
        }
      mark[i] = m; nmark += m;
    }
    if (nmark == 0) break;
    if (round >= max_rounds) return EROUNDLIMIT_;
    std::vector<Tet> next;
    std::vector<Stats> nst;
    std::vector<char> ncrit;
    next.reserve(leaves.size() + nmark);
    for (size_t i = 0; i < leaves.size(); ++i) {
      if (!mark[i]) { next.push_back(leaves[i]); nst.push_back(st[i]); ncrit.push_back(crit[i]); continue; }
      if (leaves[i].depth >= 50) return EROUNDLIMIT_;
      for (int w = 0; w < 2; ++w) { next.push_back(child(leaves[i], w)); nst.push_back(Stats()); ncrit.push_back(2); }
      verts.insert(vkey(next.back().x[leaves[i].tag]));     // z sits at position k of both children
    }
    // chunks small enough that the few, large cells of the first rounds spread over the threads
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(64, (int64_t)next.size() / (16 * nt)));
#pragma omp parallel for schedule(dynamic, chunk) num_threads(nt)
    for (int64_t i = 0; i < (int64_t)next.size(); ++i)
      if (ncrit[i] == 2) { nst[i] = density_stats(V, next[i]); ncrit[i] = split(C, next[i], nst[i]); }
    leaves.swap(next); st.swap(nst); crit.swap(ncrit);
  }

  // canonical order: sort by code (depth-first pre-order of the LEB forest)
  size_t N = leaves.size();
  std::vector<size_t> order(N);
  for (size_t i = 0; i < N; ++i) order[i] = i;
  std::vector<uint64_t> codes(N);
  for (size_t i = 0; i < N; ++i) codes[i] = code_of(leaves[i]);
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return codes[a] < codes[b]; });
  G->tets.resize(N); G->codes.resize(N); G->stats.resize(N);
  G->depth_reached = 0;
  for (size_t i = 0; i < N; ++i) {
    G->tets[i] = leaves[order[i]]; G->codes[i] = codes[order[i]]; G->stats[i] = st[order[i]];
    G->depth_reached = std::max(G->depth_reached, G->tets[i].depth);
  }
  G->rounds = round;

  // neighbours: faces are matched by their sorted vertex triples; every face must be
  // shared by exactly two leaves, or lie on the domain boundary and belong to one
  struct TripleHash {
    size_t operator()(const std::array<int32_t, 9>& k) const {
      uint64_t h = 1469598103934665603ull;
      for (int32_t v : k) { h ^= (uint32_t)v; h *= 1099511628211ull; }
      return (size_t)h;
    }
  };
  std::unordered_map<std::array<int32_t, 9>, std::vector<std::pair<int32_t, int32_t>>, TripleHash> faces;
  faces.reserve(N * 3);
  for (size_t i = 0; i < N; ++i)
    for (int f = 0; f < 4; ++f) {
      std::array<std::array<int32_t, 3>, 3> tri; int j = 0;
      for (int v = 0; v < 4; ++v) if (v != f) { tri[j] = {G->tets[i].x[v][0], G->tets[i].x[v][1], G->tets[i].x[v][2]}; ++j; }
      std::sort(tri.begin(), tri.end());
      std::array<int32_t, 9> key;
      for (int a = 0; a < 3; ++a) for (int c = 0; c < 3; ++c) key[3 * a + c] = tri[a][c];
      faces[key].push_back({(int32_t)i, f});
    }
  G->nbr.assign(N, {-1, -1, -1, -1});
  for (auto& kv : faces) {
    const auto& v = kv.second;
    if (v.size() == 2) {
      G->nbr[v[0].first][v[0].second] = v[1].first;
      G->nbr[v[1].first][v[1].second] = v[0].first;
    } else if (v.size() == 1) {
      const auto& k = kv.first;
      bool on_boundary = false;
      for (int a = 0; a < 3; ++a) {
        int32_t lim = D.C[a] << D.K;
        if (k[a] == k[3 + a] && k[a] == k[6 + a] && (k[a] == 0 || k[a] == lim)) on_boundary = true;
      }
      if (!on_boundary) return EGRID_;
    } else {
      return EGRID_;
    }
  }
  G->nid.resize(N); G->plane.resize(N); G->rho.resize(N); G->rho_max.resize(N);
  const double s = std::ldexp(1.0, -D.K);
  for (size_t i = 0; i < N; ++i) {
    const Tet& T = G->tets[i];
    for (int f = 0; f < 4; ++f) {
      int id = face_normal_id(T, f);
      if (id < 0) return EGRID_;
      G->nid[i][f] = (uint8_t)id;
      int p = id % 9;
      const int32_t* a = T.x[(f + 1) % 4];       // any vertex of face f
      int64_t c = (int64_t)P9[p][0] * a[0] + (int64_t)P9[p][1] * a[1] + (int64_t)P9[p][2] * a[2];
      G->plane[i][f] = (float)((double)c * s);
    }
    G->rho[i] = stored_density(G->stats[i], G->density_format);
    G->rho_max[i] = (float)((double)G->stats[i].qmax / 16777216.0);
  }
  G->index_of_code.reserve(N * 2);
  for (size_t i = 0; i < N; ++i) G->index_of_code[G->codes[i]] = (int32_t)i;
  return OK;
}

// ============================================================================
// Sec. 3: point location.  Descend from the Kuhn root that holds the point,
// taking at every bisection the child on the point's side of the cutting plane
// (the child holding x0 when the point is on it), until the node is a leaf.
// ============================================================================
int root_of_point(const Domain& D, V3 p, Tet* out) {
  double pc[3] = {p.x, p.y, p.z};
  int c[3]; double fr[3];
  for (int a = 0; a < 3; ++a) {
    double fl = std::floor(pc[a]);
    int ci = (int)std::max(0.0, std::min(fl, (double)(D.C[a] - 1)));
    c[a] = ci; fr[a] = pc[a] - ci;
  }
  // Kuhn tetrahedron of permutation (a, b, c) holds the points with fr[a] >= fr[b] >= fr[c]
  int best = 0;
  for (int perm = 0; perm < 6; ++perm) {
    const int* P = PERMS[perm];
    if (fr[P[0]] >= fr[P[1]] && fr[P[1]] >= fr[P[2]]) { best = perm; break; }
  }
  *out = root_tet(D, c[0], c[1], c[2], best);
  return OK;
}

// side of p relative to the plane through z and the two vertices other than x0 and xk,
// as seen from x0: >= 0 means the child holding x0
int descend_side(const Domain& D, const Tet& T, V3 p) {
  int k = T.tag;
  const double s = std::ldexp(1.0, -D.K);
  auto P = [&](const int32_t* v) { return v3(v[0] * s, v[1] * s, v[2] * s); };
  V3 z = mul(add(P(T.x[0]), P(T.x[k])), 0.5);
  V3 q[2]; int j = 0;
  for (int i = 1; i < 4; ++i) if (i != k) q[j++] = P(T.x[i]);
  V3 n = cross(sub(q[0], z), sub(q[1], z));
  double s0 = dot(n, sub(P(T.x[0]), z));
  double sp = dot(n, sub(p, z));
  return (s0 > 0) == (sp > 0) || sp == 0 ? 0 : 1;
}

int locate(const orc_grid* G, V3 p) {
  Tet T;
  root_of_point(G->D, p, &T);
  for (;;) {
    auto it = G->index_of_code.find(code_of(T));
    if (it != G->index_of_code.end()) return it->second;
    if (T.depth >= G->depth_reached) return -1;
    T = child(T, descend_side(G->D, T, p));
  }
}

// ============================================================================
// Sec. 3: the cells a ray walks through.  Both cell kinds answer one question:
// from parameter t inside cell c, where does the ray o + t d leave it and into
// which cell (-1 outside the domain).  `near_tie` reports a second exit
// candidate within 1e-5 (1 + |t|) of the first (an edge or vertex crossing).
// ============================================================================
struct Exit { double t; int32_t next; bool near_tie; int tested; };

struct TetCells {
  const orc_grid* G;
  double sigma_unit;      // extinction per grid unit at density 1
  double density(int32_t c) const { return (double)G->rho[c]; }
  // "we only need to test at most 3 faces by using the direction of the ray" (Sec. 3):
  // faces whose outward normal points against d cannot be exits and are skipped
  Exit exit(int32_t c, V3 o, V3 d, double t) const {
    double best = INFINITY, second = INFINITY; int bf = -1, tested = 0;
    for (int f = 0; f < 4; ++f) {
      int id = G->nid[c][f], p = id % 9;
      V3 n = v3(P9[p][0], P9[p][1], P9[p][2]);
      double nd = dot(n, d);
      double outward = id < 9 ? nd : -nd;
      if (!(outward > 0)) continue;
      ++tested;
      double tf = ((double)G->plane[c][f] - dot(n, o)) / nd;
      if (tf < best) { second = best; best = tf; bf = f; }
      else if (tf < second) second = tf;
    }
    Exit e;
    e.tested = tested;
    if (bf < 0) { e.t = t; e.next = -2; e.near_tie = true; return e; }
    e.t = std::max(best, t);
    e.next = G->nbr[c][bf];
    e.near_tie = (second - best) < 1e-5 * (1.0 + std::fabs(best));
    return e;
  }
};

struct VoxelCells {
  const float* rho;
  int nx, ny, nz, n;
  double sigma_unit;
  double density(int32_t c) const { return (double)rho[c]; }
  Exit exit(int32_t c, V3 o, V3 d, double t) const {
    int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    int idx[3] = {i, j, k}, dim[3] = {nx, ny, nz};
    double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    double best = INFINITY, second = INFINITY; int ba = -1;
    for (int a = 0; a < 3; ++a) {
      if (dd[a] == 0) continue;
      double wall = (double)(idx[a] + (dd[a] > 0 ? 1 : 0)) / (double)n;
      double ta = (wall - oo[a]) / dd[a];
      if (ta < best) { second = best; best = ta; ba = a; }
      else if (ta < second) second = ta;
    }
    Exit e; e.tested = 3;
    e.t = std::max(best, t);
    e.near_tie = (second - best) < 1e-5 * (1.0 + std::fabs(best));
    idx[ba] += dd[ba] > 0 ? 1 : -1;
    if (idx[ba] < 0 || idx[ba] >= dim[ba]) e.next = -1;
    else e.next = (idx[2] * ny + idx[1]) * nx + idx[0];
    return e;
  }
};

struct Ray { V3 o, d; };

struct PathLog {
  int32_t* seq; int32_t cap, len;
  bool degenerate;
  int64_t steps;
  int max_tested;
  void visit(int32_t c) { if (len < cap) seq[len] = c; ++len; }
};

// Sec. 3, "IntersectGrid": slab test against the domain box [0, C] in grid space.
bool intersect_grid(const Domain& D, const Ray& r, double* t_in) {
  double o[3] = {r.o.x, r.o.y, r.o.z}, d[3] = {r.d.x, r.d.y, r.d.z};
  double tn = 0, tf = INFINITY;
  for (int a = 0; a < 3; ++a) {
    double hi = (double)D.C[a];
    if (d[a] == 0) { if (o[a] < 0 || o[a] > hi) return false; continue; }
    double t1 = (0 - o[a]) / d[a], t2 = (hi - o[a]) / d[a];
    tn = std::max(tn, std::min(t1, t2));
    tf = std::min(tf, std::max(t1, t2));
  }
  *t_in = tn;
  return tn < tf;
}

// Sec. 3, "GridIntersectionPoint"
V3 grid_intersection_point(const Ray& r, double t_in) { return add(r.o, mul(r.d, t_in)); }

// Sec. 3, "SampleFreePath": the free path is an optical depth, -ln(1 - u).
double sample_free_path(double u) { return -std::log(1.0 - u); }

// Sec. 3, "MarchThroughCells": consume the optical depth tau across the cells
// from `cell`, starting at the segment origin.  Returns true and the collision
// point when tau is used up inside the domain, false when the ray leaves it.
template <class Cells>
int march_through_cells(const Cells& cells, const Ray& r, int32_t* cell, double tau, V3* x, PathLog* log) {
  double t = 0;
  for (int64_t step = 0;; ++step) {
    if (step >= STEP_LIMIT) return ESTEPLIMIT_;
    int32_t c = *cell;
    log->visit(c); log->steps++;
    double lambda = cells.sigma_unit * cells.density(c);    // "ReadDensity"
    Exit e = cells.exit(c, r.o, r.d, t);
    log->max_tested = std::max(log->max_tested, e.tested);
    if (e.next == -2) return EGRID_;
    if (e.near_tie || e.t - t < 1e-5 * (1.0 + std::fabs(t))) log->degenerate = true;
    double dtau = lambda * (e.t - t);
    if (lambda > 0 && dtau >= tau) {
      double tc = t + tau / lambda;
      if (e.t - tc < 1e-5 * (1.0 + std::fabs(tc))) log->degenerate = true;   // collision next to a face
      *x = add(r.o, mul(r.d, tc));
      return 1;
    }
    tau -= dtau;
    t = e.t;
    if (e.next < 0) return 0;
    *cell = e.next;
  }
}

// Transmittance exp(-sum sigma l) from x to the domain boundary (shadow ray).
template <class Cells>
int transmittance(const Cells& cells, const Ray& r, int32_t cell, double* T, PathLog* log) {
  double t = 0, od = 0;
  for (int64_t step = 0;; ++step) {
    if (step >= STEP_LIMIT) return ESTEPLIMIT_;
    log->visit(cell); log->steps++;
    Exit e = cells.exit(cell, r.o, r.d, t);
    if (e.next == -2) return EGRID_;
    if (e.near_tie) log->degenerate = true;
    od += cells.sigma_unit * cells.density(cell) * (e.t - t);
    t = e.t;
    if (e.next < 0) break;
    cell = e.next;
  }
  *T = std::exp(-od);
  return OK;
}

// Henyey-Greenstein phase function, theta between the propagation directions
// before and after the event; g > 0 scatters forward.
double hg_pdf(double g, double cos_theta) {
  double den = 1.0 + g * g - 2.0 * g * cos_theta;
  return (1.0 - g * g) / (4.0 * PI * den * std::sqrt(den));
}

// Inverse-CDF sample of cos(theta) (uniform for |g| < 1e-3), azimuth 2 pi u2,
// around d in the orthonormal frame of Duff et al. (JCGT 2017).
V3 sample_phase_function(double g, double u1, double u2, V3 d) {
  double ct;
  if (std::fabs(g) < 1e-3) ct = 1.0 - 2.0 * u1;
  else {
    double s = (1.0 - g * g) / (1.0 - g + 2.0 * g * u1);
    ct = (1.0 + g * g - s * s) / (2.0 * g);
  }
  ct = std::max(-1.0, std::min(1.0, ct));
  double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
  double phi = 2.0 * PI * u2;
  double sign = std::copysign(1.0, d.z);
  double a = -1.0 / (sign + d.z);
  double b = d.x * d.y * a;
  V3 b1 = v3(1.0 + sign * d.x * d.x * a, sign * b, -sign * d.x);
  V3 b2 = v3(b, sign + d.y * d.y * a, -d.y);
  return normalize(add(add(mul(b1, st * std::cos(phi)), mul(b2, st * std::sin(phi))), mul(d, ct)));
}

struct CamRay {
  V3 eye_g, f, r, u;
  double tanF, aspect;
  int W, H;
};

CamRay camera_rays(const orc_camera* cam, const Domain& D) {
  CamRay c;
  V3 E = from_f(cam->pos), T = from_f(cam->target), U = from_f(cam->up);
  V3 eg = sub(E, D.box_min);
  c.eye_g = v3(eg.x / D.cube, eg.y / D.cube, eg.z / D.cube);
  c.f = normalize(sub(T, E));
  c.r = normalize(cross(c.f, U));
  c.u = normalize(cross(c.r, c.f));
  c.tanF = std::tan((double)cam->fov_y_deg * HALF_DEG);
  c.aspect = (double)cam->width / (double)cam->height;
  c.W = cam->width; c.H = cam->height;
  return c;
}

// pinhole ray through film point ((px + u0) / W, (py + u1) / H), y pointing down
Ray camera_ray(const CamRay& c, int px, int py, double u0, double u1) {
  double x = ((double)px + u0) / c.W, y = ((double)py + u1) / c.H;
  V3 d = add(c.f, sub(mul(c.r, (2 * x - 1) * c.tanF * c.aspect), mul(c.u, (2 * y - 1) * c.tanF)));
  Ray r = {c.eye_g, normalize(d)};
  return r;
}

struct PathOut { double L; int32_t flags, collisions; int64_t steps; int32_t seq_len; };

// Learned radiance cache (the cached estimator): a path may end into the cache
// at its depth-th collision, after that collision's next-event estimate; the
// cache then stands for the rest of the path, the radiance that the scattered
// continuation from x brings back along -d, weighted by the path throughput
// after the albedo at x.  Training samples are a full path's own collision
// vertices: position x (grid space divided by the domain extent, in [0,1]^3),
// the direction d the path arrived with, and as target the rest of that path's
// estimate, (L_final - L after vertex j's NEE) / beta_j.  Both use 8 doubles.
struct CacheIO {
  int depth = 0;               // > 0: end the path into the cache at this collision
  double* query = nullptr;     // [8]: x (3), beta, d (3), L so far; beta = 0 when the path ended before
  int vcap = 0;                // vertices recorded per path
  double* vtx = nullptr;       // [vcap][8]: x (3), target, d (3), valid
  float survive = 0.0f;        // in (0, 1): Russian roulette once all vcap vertices are recorded
  int roulette_from = 0;       // ... and only at collisions b >= roulette_from (0-based)
};

// Russian roulette on a training path after its last training vertex: before
// each further scattering the path goes on with probability q and its
// throughput is divided by q, so the expected rest of the path -- and with it
// every target -- is unchanged, while the path ends after about 1 / (1 - q)
// more collisions instead of running to the bounce limit.  The decision after
// collision b is slot b of its own Philox stream, so it shifts no other draw.
// With a start collision r, only collisions b >= r play it: paths shorter than
// r are untouched and only the long tail is cut.
const uint32_t ROULETTE_STREAM = 0x10000u;

// Sec. 3, Algorithm 1 "Trace", with the estimator around it: throughput beta
// is multiplied by the albedo at every collision; every collision adds the sun
// seen through the shadow ray (next-event estimation); a path that leaves the
// grid adds the environment; at most max_bounces collisions.
template <class Cells, class Locate>
PathOut trace(const Cells& cells, const Domain& D, const Locate& locate_fn, const CamRay& cr,
              const orc_medium* med, uint64_t seed, int px, int py, int sample,
              int32_t* seq, int32_t seq_cap, CacheIO* cache = nullptr) {
  PathOut out = {0, 0, 0, 0, 0};
  int nv = 0;                              // cache: vertices recorded
  double vbeta[64], vL[64];                // their throughput and the estimate after their NEE
  if (cache && cache->vcap > 64) cache->vcap = 64;
  auto finish_cache = [&](double Lf) {
    if (!cache) return;
    if (cache->query) {
      if (cache->query[3] == 0) for (int k = 0; k < 7; ++k) cache->query[k] = 0;
      cache->query[7] = Lf;
    }
    for (int j = 0; j < cache->vcap; ++j) {
      double* v = cache->vtx + 8 * j;
      if (j < nv && vbeta[j] > 0) {
        v[3] = (Lf - vL[j]) / vbeta[j];
        v[7] = 1;
      } else {
        for (int k = 0; k < 8; ++k) v[k] = 0;
      }
    }
  };
  if (cache && cache->query) cache->query[3] = 0;
  PathLog log = {seq, seq_cap, 0, false, 0, 0};
  uint32_t pixel = (uint32_t)(py * cr.W + px);
  double u0 = uniform(seed, pixel, (uint32_t)sample, 0), u1 = uniform(seed, pixel, (uint32_t)sample, 1);
  Ray ray = camera_ray(cr, px, py, u0, u1);
  double L = 0, beta = 1;
  V3 w_sun = normalize(mul(from_f(med->sun_dir), -1.0));
  double t_in;
  if (!intersect_grid(D, ray, &t_in)) {                      // "IntersectGrid"
    out.L = med->env_radiance; out.flags = 4; finish_cache(out.L); return out;
  }
  ray.o = grid_intersection_point(ray, t_in);                // "GridIntersectionPoint"
  int32_t cell = locate_fn(ray.o);
  if (cell < 0) { out.flags = 16; finish_cache(0); return out; }
  for (int b = 0;; ++b) {                                     // "while InsideGrid(ray)"
    double tau = sample_free_path(uniform(seed, pixel, sample, 2 + 3 * b));   // "SampleFreePath"
    V3 x;
    int hit = march_through_cells(cells, ray, &cell, tau, &x, &log);         // "MarchThroughCells"
    if (hit < 0) { out.flags |= hit == ESTEPLIMIT_ ? 8 : 16; break; }
    if (hit == 0) { L += beta * med->env_radiance; break; }
    out.collisions++;
    beta *= med->albedo;
    if (log.len < seq_cap) seq[log.len] = -1;
    log.len++;
    double T;
    Ray shadow = {x, w_sun};
    int st = transmittance(cells, shadow, cell, &T, &log);
    if (st < 0) { out.flags |= st == ESTEPLIMIT_ ? 8 : 16; break; }
    if (log.len < seq_cap) seq[log.len] = -1;
    log.len++;
    L += beta * hg_pdf(med->g, dot(ray.d, w_sun)) * med->sun_irradiance * T;
    if (cache && nv < cache->vcap) {
      double* v = cache->vtx + 8 * nv;
      v[0] = x.x / D.C[0]; v[1] = x.y / D.C[1]; v[2] = x.z / D.C[2];
      v[4] = ray.d.x; v[5] = ray.d.y; v[6] = ray.d.z;
      vbeta[nv] = beta; vL[nv] = L;
      ++nv;
    }
    if (b + 1 >= med->max_bounces) { out.flags |= 2; break; }
    if (cache && cache->depth > 0 && b + 1 == cache->depth) {
      // the path ends into the cache: it stands for everything after this vertex
      double* q = cache->query;
      if (q) {
        q[0] = x.x / D.C[0]; q[1] = x.y / D.C[1]; q[2] = x.z / D.C[2]; q[3] = beta;
        q[4] = ray.d.x; q[5] = ray.d.y; q[6] = ray.d.z;
      }
      break;
    }
    if (cache && cache->vcap > 0 && nv >= cache->vcap && b >= cache->roulette_from && cache->survive > 0.0f &&
        cache->survive < 1.0f) {
      const double q = (double)cache->survive;
      if (uniform(seed, pixel, (uint32_t)sample, (uint32_t)b, ROULETTE_STREAM) >= q) { out.flags |= 32; break; }
      beta /= q;
    }
    ray.d = sample_phase_function(med->g, uniform(seed, pixel, sample, 3 + 3 * b),
                                  uniform(seed, pixel, sample, 4 + 3 * b), ray.d);   // "SamplePhaseFunction"
    ray.o = x;
  }
  out.L = L;
  finish_cache(L);
  if (log.degenerate) out.flags |= 1;
  out.steps = log.steps;
  out.seq_len = std::min(log.len, seq_cap);
  return out;
}

// ============================================================================
// Extra channels (Sec. 3: "extra channels for, e.g., temperature, albedo, phase
// function parameters").  Per tet, the mean of each channel volume over D (the
// same voxel set as the density), quantised like the density; g = 2 a - 1 from
// an anisotropy volume a in [0, 1], clamped to [-0.99, 0.99].  The voxel
// majorant of a tet bounds the voxel density anywhere in it: (max q + 1) / 2^24
// over the voxels whose cells touch the tet's bounding box.
// ============================================================================
float channel_mean(const Stats& st) {
  return (float)((double)st.sum / ((double)st.count * 16777216.0));
}

float voxel_majorant(const Volume& V, const Tet& T) {
  const Domain& D = *V.D;
  int64_t w = (int64_t)1 << (D.K - D.m);          // voxel edge in vertex units
  int dims[3] = {D.nx, D.ny, D.nz};
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    int64_t mn = T.x[0][a], mx = T.x[0][a];
    for (int i = 1; i < 4; ++i) { mn = std::min<int64_t>(mn, T.x[i][a]); mx = std::max<int64_t>(mx, T.x[i][a]); }
    lo[a] = std::max<int64_t>(0, floor_div(mn, w));
    hi[a] = std::min<int64_t>(dims[a] - 1, floor_div(mx, w));
  }
  uint32_t m = 0;
  for (int64_t k = lo[2]; k <= hi[2]; ++k)
    for (int64_t j = lo[1]; j <= hi[1]; ++j)
      for (int64_t i = lo[0]; i <= hi[0]; ++i) m = std::max(m, V.q[((size_t)k * D.ny + j) * D.nx + i]);
  return (float)(((double)m + 1.0) / 16777216.0);
}

// The extended estimator.  flags: emission (1), per-tet albedo (2), per-tet g
// (4), voxel medium with delta tracking (8).
//  * emission: at every real collision the collision estimator of the emitted
//    radiance, beta (1 - albedo) Le with Le = emission_scale * temperature;
//  * voxel medium: the density at x is the voxel value of the voxel holding x
//    (the regular-grid comparator's medium); free flights are tracked against
//    the tet majorant (regular tracking in the majorant medium, then a tentative
//    collision is real with probability rho(x) / majorant, decided in fp32 as
//    u * majorant < rho(x)), shadow rays use ratio tracking, prod (1 - rho / majorant).
//    Delta-tracking random numbers (acceptance, then the next free path, per
//    tentative collision; free paths of a shadow ray): slot k of stream 1 + 2b
//    (free flight of bounce b) or 2 + 2b (its shadow ray), k counted per segment.
struct ExtSpec { int flags; double emission_scale; const float* voxel; };

struct MajorantCells {
  const orc_grid* G;
  double sigma_unit;
  double density(int32_t c) const { return (double)G->vmaj[c]; }
  Exit exit(int32_t c, V3 o, V3 d, double t) const { TetCells tc = {G, sigma_unit}; return tc.exit(c, o, d, t); }
};

float voxel_density_at(const orc_grid* G, const float* vox, V3 x) {
  const Domain& D = G->D;
  double p[3] = {x.x, x.y, x.z};
  int dims[3] = {D.nx, D.ny, D.nz};
  int64_t idx[3];
  for (int a = 0; a < 3; ++a) {
    int64_t i = (int64_t)std::floor(p[a] * (double)D.n);
    idx[a] = std::min<int64_t>(std::max<int64_t>(i, 0), dims[a] - 1);
  }
  return vox[((size_t)idx[2] * D.ny + idx[1]) * D.nx + idx[0]];
}

template <class Locate>
PathOut trace_ext(const orc_grid* G, const ExtSpec& X, const Locate& locate_fn, const CamRay& cr,
                  const orc_medium* med, uint64_t seed, int px, int py, int sample) {
  const double sigma_unit = (double)med->sigma_scale * G->D.cube;
  TetCells cells = {G, sigma_unit};
  MajorantCells mcells = {G, sigma_unit};
  const bool voxel = (X.flags & 8) != 0;
  PathOut out = {0, 0, 0, 0, 0};
  PathLog log = {nullptr, 0, 0, false, 0, 0};
  uint32_t pixel = (uint32_t)(py * cr.W + px);
  uint32_t kseg = 0;                                  // draws of the current segment
  auto draw = [&](uint32_t stream) { return uniform(seed, pixel, (uint32_t)sample, kseg++, stream); };
  double u0 = uniform(seed, pixel, (uint32_t)sample, 0), u1 = uniform(seed, pixel, (uint32_t)sample, 1);
  Ray ray = camera_ray(cr, px, py, u0, u1);
  double L = 0, beta = 1;
  V3 w_sun = normalize(mul(from_f(med->sun_dir), -1.0));
  double t_in;
  if (!intersect_grid(G->D, ray, &t_in)) { out.L = med->env_radiance; out.flags = 4; return out; }
  ray.o = grid_intersection_point(ray, t_in);
  int32_t cell = locate_fn(ray.o);
  if (cell < 0) { out.flags = 16; return out; }
  for (int b = 0;; ++b) {
    double tau = sample_free_path(uniform(seed, pixel, sample, 2 + 3 * b));
    V3 x;
    int hit;
    kseg = 0;
    if (!voxel) {
      hit = march_through_cells(cells, ray, &cell, tau, &x, &log);
    } else {
      for (;;) {
        hit = march_through_cells(mcells, ray, &cell, tau, &x, &log);
        if (hit != 1) break;
        const float rx = voxel_density_at(G, X.voxel, x);
        const float mj = G->vmaj[cell];
        const float u = (float)draw(1u + 2u * b);
        if (u * mj < rx) break;                              // a real collision
        ray.o = x;                                           // a null collision: fly on from x
        tau = sample_free_path(draw(1u + 2u * b));
      }
    }
    if (hit < 0) { out.flags |= hit == ESTEPLIMIT_ ? 8 : 16; break; }
    if (hit == 0) { L += beta * med->env_radiance; break; }
    out.collisions++;
    const std::array<float, 3>& ch = G->chan[cell];
    const double albedo = (X.flags & 2) ? (double)ch[1] : (double)med->albedo;
    const double g = (X.flags & 4) ? (double)ch[2] : (double)med->g;
    if (X.flags & 1) L += beta * (1.0 - albedo) * X.emission_scale * (double)ch[0];
    beta *= albedo;
    double T;
    Ray shadow = {x, w_sun};
    if (!voxel) {
      int st = transmittance(cells, shadow, cell, &T, &log);
      if (st < 0) { out.flags |= st == ESTEPLIMIT_ ? 8 : 16; break; }
    } else {
      // ratio tracking towards the sun
      T = 1.0;
      int32_t sc = cell;
      int st = 0;
      kseg = 0;
      for (;;) {
        V3 xs;
        st = march_through_cells(mcells, shadow, &sc, sample_free_path(draw(2u + 2u * b)), &xs, &log);
        if (st != 1) break;
        T *= 1.0 - (double)voxel_density_at(G, X.voxel, xs) / (double)G->vmaj[sc];
        shadow.o = xs;
      }
      if (st < 0) { out.flags |= st == ESTEPLIMIT_ ? 8 : 16; break; }
    }
    L += beta * hg_pdf(g, dot(ray.d, w_sun)) * med->sun_irradiance * T;
    if (b + 1 >= med->max_bounces) { out.flags |= 2; break; }
    ray.d = sample_phase_function(g, uniform(seed, pixel, sample, 3 + 3 * b),
                                  uniform(seed, pixel, sample, 4 + 3 * b), ray.d);
    ray.o = x;
  }
  out.L = L;
  if (log.degenerate) out.flags |= 1;
  out.steps = log.steps;
  return out;
}

bool valid_camera(const orc_camera* c) {
  return c && c->width > 0 && c->height > 0 && c->fov_y_deg > 0 && c->fov_y_deg < 180;
}
bool valid_medium(const orc_medium* m) { return m && m->max_bounces >= 1 && m->g > -1 && m->g < 1; }

}  // namespace

// ============================================================================
// C API
// ============================================================================
extern "C" {

int orc_build(const float* density, int32_t nx, int32_t ny, int32_t nz, const float box_min[3],
              float voxel_size, const orc_camera* cam, float footprint_px, float theta,
              int32_t max_depth, int32_t density_format, int32_t max_rounds, int32_t nthreads,
              orc_grid** out) {
  if (!density || !out || density_format < 0 || density_format > 2) return EINVAL_;
  if (cam && !valid_camera(cam)) return EINVAL_;
  orc_grid* G = new (std::nothrow) orc_grid();
  if (!G) return ENOMEM_;
  int st = make_domain(nx, ny, nz, box_min, voxel_size, max_depth, &G->D);
  if (st) { delete G; return st; }
  G->density_format = density_format;
  Volume V;
  quantise(density, G->D, &V);
  Criterion C;
  C.D = &G->D; C.V = &V;
  C.cam = camera_criterion(cam, footprint_px, G->D);
  C.var_on = theta >= 0;
  C.theta_q16 = C.var_on ? std::llround((double)theta * 65536.0) : 0;
  if (max_rounds <= 0) max_rounds = 4 * max_depth + 16;
  st = build_grid(V, C, max_rounds, nthreads, G);
  if (st) { delete G; return st; }
  *out = G;
  return OK;
}

void orc_grid_free(orc_grid* g) { delete g; }

int orc_grid_info(const orc_grid* g, int64_t* num_tets, int32_t* max_depth_reached, int32_t* K,
                  int32_t* rounds, int32_t* cubes, int32_t* voxels_per_cube) {
  if (!g) return EINVAL_;
  if (num_tets) *num_tets = (int64_t)g->tets.size();
  if (max_depth_reached) *max_depth_reached = g->depth_reached;
  if (K) *K = g->D.K;
  if (rounds) *rounds = g->rounds;
  if (cubes) for (int a = 0; a < 3; ++a) cubes[a] = g->D.C[a];
  if (voxels_per_cube) *voxels_per_cube = g->D.n;
  return OK;
}

int orc_grid_export(const orc_grid* g, uint64_t* codes, int32_t* verts, int32_t* tag, int32_t* nbr,
                    uint8_t* nid, float* plane, float* density, float* majorant, uint32_t* count,
                    uint64_t* sum, uint32_t* qmin, uint32_t* qmax) {
  if (!g) return EINVAL_;
  size_t N = g->tets.size();
  for (size_t i = 0; i < N; ++i) {
    if (codes) codes[i] = g->codes[i];
    if (verts) for (int v = 0; v < 4; ++v) for (int a = 0; a < 3; ++a) verts[(i * 4 + v) * 3 + a] = g->tets[i].x[v][a];
    if (tag) tag[i] = g->tets[i].tag;
    for (int f = 0; f < 4; ++f) {
      if (nbr) nbr[i * 4 + f] = g->nbr[i][f];
      if (nid) nid[i * 4 + f] = g->nid[i][f];
      if (plane) plane[i * 4 + f] = g->plane[i][f];
    }
    if (density) density[i] = g->rho[i];
    if (majorant) majorant[i] = g->rho_max[i];
    if (count) count[i] = g->stats[i].count;
    if (sum) sum[i] = g->stats[i].sum;
    if (qmin) qmin[i] = g->stats[i].qmin;
    if (qmax) qmax[i] = g->stats[i].qmax;
  }
  return OK;
}

int orc_render_paths(const orc_grid* g, const orc_camera* cam, const orc_medium* med, uint64_t seed,
                     int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                     double* L, int32_t* flags, int32_t* collisions, int64_t* steps,
                     int32_t* seq, int32_t seq_cap, int32_t* seq_len, int32_t nthreads) {
  if (!g || !valid_camera(cam) || !valid_medium(med) || n < 0) return EINVAL_;
  TetCells cells = {g, (double)med->sigma_scale * g->D.cube};
  CamRay cr = camera_rays(cam, g->D);
  auto loc = [&](V3 p) { return locate(g, p); };
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    int32_t* s = seq && seq_cap > 0 ? seq + i * (int64_t)seq_cap : nullptr;
    PathOut o = trace(cells, g->D, loc, cr, med, seed, px[i], py[i], sample[i], s, s ? seq_cap : 0);
    if (L) L[i] = o.L;
    if (flags) flags[i] = o.flags;
    if (collisions) collisions[i] = o.collisions;
    if (steps) steps[i] = o.steps;
    if (seq_len) seq_len[i] = o.seq_len;
  }
  return OK;
}

int orc_cache_paths(const orc_grid* g, const orc_camera* cam, const orc_medium* med, uint64_t seed, int64_t n,
                    const int32_t* px, const int32_t* py, const int32_t* sample, int32_t cache_depth,
                    double* query, int32_t max_vertices, double* vertices, double* L, int32_t* flags,
                    float survive, int32_t roulette_from, int32_t nthreads) {
  if (!g || !valid_camera(cam) || !valid_medium(med) || n < 0 || cache_depth < 0 || max_vertices < 0 ||
      max_vertices > 64 || (max_vertices > 0 && !vertices) || (cache_depth > 0 && !query) ||
      !(survive >= 0.0f && survive <= 1.0f) || roulette_from < 0)
    return EINVAL_;
  TetCells cells = {g, (double)med->sigma_scale * g->D.cube};
  CamRay cr = camera_rays(cam, g->D);
  auto loc = [&](V3 p) { return locate(g, p); };
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    CacheIO io;
    io.depth = cache_depth;
    io.query = cache_depth > 0 ? query + 8 * i : nullptr;
    io.vcap = max_vertices;
    io.vtx = max_vertices > 0 ? vertices + 8 * max_vertices * i : nullptr;
    io.survive = survive;
    io.roulette_from = roulette_from;
    PathOut o = trace(cells, g->D, loc, cr, med, seed, px[i], py[i], sample[i], nullptr, 0, &io);
    if (L) L[i] = o.L;
    if (flags) flags[i] = o.flags;
  }
  return OK;
}

int orc_grid_channels(orc_grid* g, const float* density, const float* temperature, const float* albedo,
                      const float* aniso, int32_t nthreads) {
  if (!g || !density) return EINVAL_;
  const Domain& D = g->D;
  size_t N = g->tets.size();
  g->chan.assign(N, {0.0f, 0.0f, 0.0f});
  g->vmaj.assign(N, 0.0f);
  const float* vols[3] = {temperature, albedo, aniso};
  int nt = set_threads(nthreads);
  for (int c = 0; c < 3; ++c) {
    if (!vols[c]) continue;
    Volume V;
    quantise(vols[c], D, &V);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t i = 0; i < (int64_t)N; ++i) {
      float m = channel_mean(density_stats(V, g->tets[i]));
      if (c == 2) m = (float)std::min(0.99, std::max(-0.99, 2.0 * (double)m - 1.0));
      g->chan[i][c] = m;
    }
  }
  Volume V;
  quantise(density, D, &V);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
  for (int64_t i = 0; i < (int64_t)N; ++i) g->vmaj[i] = voxel_majorant(V, g->tets[i]);
  g->channel_mask = (temperature ? 1 : 0) | (albedo ? 2 : 0) | (aniso ? 4 : 0) | 8;
  return OK;
}

int orc_grid_export_channels(const orc_grid* g, float* chan, float* vmaj) {
  if (!g || !g->channel_mask) return EINVAL_;
  for (size_t i = 0; i < g->tets.size(); ++i) {
    if (chan) for (int c = 0; c < 3; ++c) chan[3 * i + c] = g->chan[i][c];
    if (vmaj) vmaj[i] = g->vmaj[i];
  }
  return OK;
}

int orc_render_ext_paths(const orc_grid* g, const orc_camera* cam, const orc_medium* med, const orc_ext* ext,
                         uint64_t seed, int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                         double* L, int32_t* flags, int32_t* collisions, int64_t* steps, int32_t nthreads) {
  if (!g || !valid_camera(cam) || !valid_medium(med) || !ext || n < 0) return EINVAL_;
  int need = ext->flags & 15;
  if ((need & ~g->channel_mask) || ((ext->flags & 8) && !ext->density)) return EINVAL_;
  ExtSpec X = {ext->flags, (double)ext->emission_scale, ext->density};
  CamRay cr = camera_rays(cam, g->D);
  auto loc = [&](V3 p) { return locate(g, p); };
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    PathOut o = trace_ext(g, X, loc, cr, med, seed, px[i], py[i], sample[i]);
    if (L) L[i] = o.L;
    if (flags) flags[i] = o.flags;
    if (collisions) collisions[i] = o.collisions;
    if (steps) steps[i] = o.steps;
  }
  return OK;
}

int orc_render(const orc_grid* g, const orc_camera* cam, const orc_medium* med, int32_t spp, uint64_t seed,
               int32_t sample_offset, double* sum, double* sumsq, int64_t* steps, int32_t nthreads) {
  if (!g || !valid_camera(cam) || !valid_medium(med) || spp < 0 || !sum) return EINVAL_;
  TetCells cells = {g, (double)med->sigma_scale * g->D.cube};
  CamRay cr = camera_rays(cam, g->D);
  auto loc = [&](V3 p) { return locate(g, p); };
  int64_t total = 0;
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(+ : total)
  for (int py = 0; py < cam->height; ++py)
    for (int px = 0; px < cam->width; ++px)
      for (int s = 0; s < spp; ++s) {
        PathOut o = trace(cells, g->D, loc, cr, med, seed, px, py, sample_offset + s, nullptr, 0);
        sum[py * cam->width + px] += o.L;
        if (sumsq) sumsq[py * cam->width + px] += o.L * o.L;
        total += o.steps;
      }
  if (steps) *steps = total;
  return OK;
}

static int dda_setup(int32_t nx, int32_t ny, int32_t nz, const float box_min[3], float voxel_size,
                     Domain* D) {
  return make_domain(nx, ny, nz, box_min, voxel_size, 0, D);
}

// entry voxel: the voxel holding the entry point (floor, clamped to the grid)
static int32_t voxel_of(const Domain& D, V3 p) {
  double pc[3] = {p.x, p.y, p.z};
  int dims[3] = {D.nx, D.ny, D.nz};
  int idx[3];
  for (int a = 0; a < 3; ++a) {
    double v = std::floor(pc[a] * D.n);
    idx[a] = (int)std::max(0.0, std::min(v, (double)(dims[a] - 1)));
  }
  return (idx[2] * D.ny + idx[1]) * D.nx + idx[0];
}

int orc_dda_paths(const float* density, int32_t nx, int32_t ny, int32_t nz, const float box_min[3],
                  float voxel_size, const orc_camera* cam, const orc_medium* med, uint64_t seed, int64_t n,
                  const int32_t* px, const int32_t* py, const int32_t* sample, double* L, int32_t* flags,
                  int32_t* collisions, int64_t* steps, int32_t nthreads) {
  Domain D;
  if (!density || !valid_camera(cam) || !valid_medium(med) || dda_setup(nx, ny, nz, box_min, voxel_size, &D))
    return EINVAL_;
  VoxelCells cells = {density, nx, ny, nz, D.n, (double)med->sigma_scale * D.cube};
  CamRay cr = camera_rays(cam, D);
  auto loc = [&](V3 p) { return voxel_of(D, p); };
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    PathOut o = trace(cells, D, loc, cr, med, seed, px[i], py[i], sample[i], nullptr, 0);
    if (L) L[i] = o.L;
    if (flags) flags[i] = o.flags;
    if (collisions) collisions[i] = o.collisions;
    if (steps) steps[i] = o.steps;
  }
  return OK;
}

int orc_dda_render(const float* density, int32_t nx, int32_t ny, int32_t nz, const float box_min[3],
                   float voxel_size, const orc_camera* cam, const orc_medium* med, int32_t spp, uint64_t seed,
                   int32_t sample_offset, double* sum, double* sumsq, int64_t* steps, int32_t nthreads) {
  Domain D;
  if (!density || !sum || !valid_camera(cam) || !valid_medium(med) ||
      dda_setup(nx, ny, nz, box_min, voxel_size, &D))
    return EINVAL_;
  VoxelCells cells = {density, nx, ny, nz, D.n, (double)med->sigma_scale * D.cube};
  CamRay cr = camera_rays(cam, D);
  auto loc = [&](V3 p) { return voxel_of(D, p); };
  int64_t total = 0;
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(+ : total)
  for (int py = 0; py < cam->height; ++py)
    for (int px = 0; px < cam->width; ++px)
      for (int s = 0; s < spp; ++s) {
        PathOut o = trace(cells, D, loc, cr, med, seed, px, py, sample_offset + s, nullptr, 0);
        sum[py * cam->width + px] += o.L;
        if (sumsq) sumsq[py * cam->width + px] += o.L * o.L;
        total += o.steps;
      }
  if (steps) *steps = total;
  return OK;
}

int orc_optical_depth(const orc_grid* g, int64_t n, const double* origin, const double* dir, double sigma,
                      double* tau, int64_t* steps, int32_t* max_faces_tested, int32_t* flags, int32_t* seq,
                      int32_t seq_cap, int32_t* seq_len) {
  if (!g || n < 0) return EINVAL_;
  TetCells cells = {g, sigma};
  for (int64_t i = 0; i < n; ++i) {
    Ray r = {v3(origin[3 * i], origin[3 * i + 1], origin[3 * i + 2]),
             normalize(v3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]))};
    int32_t* s = seq && seq_cap > 0 ? seq + i * (int64_t)seq_cap : nullptr;
    PathLog log = {s, s ? seq_cap : 0, 0, false, 0, 0};
    double t_in, T = 1;
    int32_t fl = 0;
    if (intersect_grid(g->D, r, &t_in)) {
      r.o = grid_intersection_point(r, t_in);
      int32_t c = locate(g, r.o);
      if (c < 0) fl |= 16;
      else {
        int st = transmittance(cells, r, c, &T, &log);
        if (st < 0) fl |= st == ESTEPLIMIT_ ? 8 : 16;
      }
    } else {
      fl |= 4;
    }
    if (log.degenerate) fl |= 1;
    tau[i] = -std::log(T);
    if (T == 0) tau[i] = INFINITY;
    if (steps) steps[i] = log.steps;
    if (max_faces_tested) max_faces_tested[i] = log.max_tested;
    if (flags) flags[i] = fl;
    if (seq_len) seq_len[i] = std::min(log.len, s ? seq_cap : 0);
  }
  return OK;
}

int orc_path_profile(const float* density, int32_t nx, int32_t ny, int32_t nz, const float box_min[3],
                     float voxel_size, const orc_camera* cam, float footprint_px, float theta,
                     int32_t max_depth, int32_t density_format, int64_t n, const double* points,
                     uint64_t* codes, uint32_t* count, uint64_t* sum, uint32_t* qmin, uint32_t* qmax,
                     float* density_out, uint8_t* split_out, int32_t nthreads) {
  Domain D;
  if (!density || make_domain(nx, ny, nz, box_min, voxel_size, max_depth, &D)) return EINVAL_;
  Volume V;
  quantise(density, D, &V);
  Criterion C;
  C.D = &D; C.V = &V;
  C.cam = camera_criterion(cam, footprint_px, D);
  C.var_on = theta >= 0;
  C.theta_q16 = C.var_on ? std::llround((double)theta * 65536.0) : 0;
  int levels = max_depth + 1;
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    V3 p = v3(points[3 * i], points[3 * i + 1], points[3 * i + 2]);
    Tet T;
    root_of_point(D, p, &T);
    for (int d = 0; d < levels; ++d) {
      Stats s = density_stats(V, T);
      int64_t o = i * levels + d;
      codes[o] = code_of(T);
      if (count) count[o] = s.count;
      if (sum) sum[o] = s.sum;
      if (qmin) qmin[o] = s.qmin;
      if (qmax) qmax[o] = s.qmax;
      if (density_out) density_out[o] = stored_density(s, density_format);
      if (split_out) split_out[o] = split(C, T, s) ? 1 : 0;
      if (d + 1 < levels) T = child(T, descend_side(D, T, p));
    }
  }
  return OK;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox(ctr, key, out); }
double orc_uniform(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t slot) {
  return uniform(seed, pixel, sample, slot);
}
void orc_hg_sample(double g, double u1, double u2, const double dir_in[3], double dir_out[3]) {
  V3 o = sample_phase_function(g, u1, u2, v3(dir_in[0], dir_in[1], dir_in[2]));
  dir_out[0] = o.x; dir_out[1] = o.y; dir_out[2] = o.z;
}
double orc_hg_pdf(double g, double cos_theta) { return hg_pdf(g, cos_theta); }
int orc_locate(const orc_grid* g, int64_t n, const double* points, int32_t* leaf) {
  if (!g) return EINVAL_;
  for (int64_t i = 0; i < n; ++i) leaf[i] = locate(g, v3(points[3 * i], points[3 * i + 1], points[3 * i + 2]));
  return OK;
}

}  // extern "C"
