// Cell walker over the tetrahedral grid (Sec. 3, "Path Tracing within
// Tetrahedral Grids"): the exit face of the current cell is found among the
// faces whose stored orientation faces along the ray (at most three), and the
// ray moves to the neighbour across it.
//
// Face planes only take the 9 orientations P = {x, y, z, x+y, x-y, y+z, y-z,
// x+z, x-z}, so per segment the walker keeps, for each orientation p, one
// 16-byte entry in shared memory (one column per thread: conflict-free):
// nO[p] = (P[p] . o) 2^K as a float-float pair (hi, lo), and 2^-K / (P[p] . d)
// for the outward normals +P[p] and -P[p] -- NaN for the one that does not point
// along d (a face that cannot be an exit).  The exit parameter of a face with
// integer plane offset c (units of 2^-K) is then (c - nO.hi - nO.lo) times the
// reciprocal of its normal's sign: one 16-byte load per face.  The float-float
// nO keeps c - nO accurate to the distance walked rather than to |o|.
//
// The walk is a chain of dependent record loads.  To shorten each link the
// walker loads the record of the cell it moves to as soon as the exit face is
// known -- before the caller's optical-depth work and before any warp-wide
// event round -- into the same registers that held the current record.  A
// segment start (begin) loads the record of the cell it starts in.
#pragma once
#include "estimator.cuh"

namespace tv {

struct TetParams {
  const uint4* rec;
  const unsigned long long* codes;
  long long n;
  int K, depth;                 // vertex scale exponent; deepest level present
  int C[3];                     // cubes per axis
  float scaleK, invK;           // 2^K, 2^-K
  const int32_t* locator;       // cell holding the centre of each locator-grid cell (may be null)
  int R;                        // locator cells per cube edge
};

__device__ __forceinline__ int sext24(uint32_t v) { return ((int)(v << 8)) >> 8; }

// Signed 24-bit plane offset held in three consecutive bytes of the 8-byte pair
// (lo, hi): one byte permute whose fourth selector replicates the sign of the
// third byte (prmt: a selector with its top bit set copies the selected byte's sign).
__device__ __forceinline__ int prmt_s24(uint32_t lo, uint32_t hi, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(lo), "r"(hi), "r"(sel));
  return (int)r;
}

template <int FMT>
__device__ __forceinline__ float decode_density(uint32_t w) {
  if (FMT == TG_DENSITY_BF16) return __uint_as_float(w);          // bf16 in the high half, low half zero
  if (FMT == TG_DENSITY_FP16) return __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu)));
  return __uint_as_float(w);
}

// Point location by descent of the LEB hierarchy: from the Kuhn root holding
// p, take at every bisection the child on p's side of the cutting plane (the
// child holding x0 when p lies on it) down to the deepest level of the grid;
// the cell is then the last code <= the point's code (depth-first order).
inline __device__ long long tet_locate(const TetParams& P, float3 p) {
  const float pc[3] = {p.x, p.y, p.z};
  int cube[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int c = (int)floorf(pc[a]);
    c = c < 0 ? 0 : (c > P.C[a] - 1 ? P.C[a] - 1 : c);
    cube[a] = c;
    fr[a] = pc[a] - (float)c;
  }
  // Kuhn permutation (a, b, c) holds fr[a] >= fr[b] >= fr[c]; permutations in lexicographic order
  int perm;
  if (fr[0] >= fr[1] && fr[1] >= fr[2]) perm = 0;
  else if (fr[0] >= fr[2] && fr[2] >= fr[1]) perm = 1;
  else if (fr[1] >= fr[0] && fr[0] >= fr[2]) perm = 2;
  else if (fr[1] >= fr[2] && fr[2] >= fr[0]) perm = 3;
  else if (fr[2] >= fr[0] && fr[0] >= fr[1]) perm = 4;
  else perm = 5;
  const int ax0 = (perm < 2) ? 0 : (perm < 4 ? 1 : 2);
  const int ax1 = (perm == 0 || perm == 5) ? 1 : ((perm == 1 || perm == 3) ? 2 : 0);
  const int S = 1 << P.K;
  int x[4][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[0][a] = cube[a] * S;
    x[1][a] = x[0][a] + (a == ax0 ? S : 0);
    x[2][a] = x[1][a] + (a == ax1 ? S : 0);
    x[3][a] = x[0][a] + S;
  }
  const unsigned long long root = (unsigned long long)(((cube[2] * P.C[1] + cube[1]) * P.C[0] + cube[0]) * 6 + perm);
  int k = 3;
  unsigned long long path = 0;
  for (int lev = 0; lev < P.depth; ++lev) {
    int z2[3], u[3], v[3];
    const int ia = k == 1 ? 2 : 1;       // the two vertices other than x0 and xk
    const int ib = k == 3 ? 2 : 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      z2[a] = x[0][a] + x[k][a];
      u[a] = 2 * x[ia][a] - z2[a];
      v[a] = 2 * x[ib][a] - z2[a];
    }
    const long long n0 = (long long)u[1] * v[2] - (long long)u[2] * v[1];
    const long long n1 = (long long)u[2] * v[0] - (long long)u[0] * v[2];
    const long long n2 = (long long)u[0] * v[1] - (long long)u[1] * v[0];
    const int c0 = (n0 > 0) - (n0 < 0), c1 = (n1 > 0) - (n1 < 0), c2 = (n2 > 0) - (n2 < 0);
    const long long s0 = (long long)c0 * (2 * x[0][0] - z2[0]) + (long long)c1 * (2 * x[0][1] - z2[1]) +
                         (long long)c2 * (2 * x[0][2] - z2[2]);
    const float cp = (float)c0 * p.x + (float)c1 * p.y + (float)c2 * p.z;
    const float cz = (float)(c0 * z2[0] + c1 * z2[1] + c2 * z2[2]) * (0.5f * P.invK);
    const int side = (cp == cz || ((cp > cz) == (s0 > 0))) ? 0 : 1;
    path = (path << 1) | (unsigned long long)side;
    int y[4][3];
    int j = 0;
    if (side == 0) {
      for (int i = 0; i < k; ++i, ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) y[j][a] = x[i][a];
    } else {
      for (int i = 1; i <= k; ++i, ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) y[j][a] = x[i][a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) y[j][a] = z2[a] >> 1;
    ++j;
    for (int i = k + 1; i < 4; ++i, ++j)
#pragma unroll
      for (int a = 0; a < 3; ++a) y[j][a] = x[i][a];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int a = 0; a < 3; ++a) x[i][a] = y[i][a];
    k = k > 1 ? k - 1 : 3;
  }
  const unsigned long long bits = P.depth ? ((path << (56 - P.depth)) & ((1ull << 56) - 1)) : 0ull;
  const unsigned long long key = (root << 56) | bits | (unsigned long long)P.depth;
  // last code <= key
  long long lo = 0, hi = P.n;          // invariant: codes[lo-1] <= key < codes[hi]
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (P.codes[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// Orientation table of a direction, indexed by the orientation id p | s << 4:
// 2^-K / (P[p] . d) (correctly rounded reciprocal, exact scaling) when the
// outward normal (-1)^s P[p] points along d, NaN otherwise -- a NaN exit
// parameter never compares smaller, so masked faces need no test.
constexpr int TET_NID = 25;

__device__ __forceinline__ void tet_dir_table(const ff3& d, float invK, float inv[TET_NID]) {
  const float nd[9] = {ff_float(d.x), ff_float(d.y), ff_float(d.z), ff_float(ff_add(d.x, d.y)),
                       ff_float(ff_sub(d.x, d.y)), ff_float(ff_add(d.y, d.z)), ff_float(ff_sub(d.y, d.z)),
                       ff_float(ff_add(d.x, d.z)), ff_float(ff_sub(d.x, d.z))};
#pragma unroll
  for (int q = 0; q < TET_NID; ++q) inv[q] = __int_as_float(0x7FFFFFFF);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const float r = __frcp_rn(nd[p]) * invK;
    if (nd[p] > 0.f) inv[p] = r;
    if (nd[p] < 0.f) inv[p | 16] = r;
  }
}

// BATCH: the walker of a batch of grids -- the grid (and so its parameters)
// changes from path to path and from lane to lane; set_job points it at one.
template <int FMT, bool BATCH = false>
struct TetWalker {
  using Params = TetParams;
  static constexpr int NDIR = TET_NID;      // direction-table entries (tet_dir_table's layout)
  const TetParams& P0;                      // the grid's parameters (uniform)
  const TetParams* Pj = nullptr;            // BATCH: the current path's grid
  const uint4* brec = nullptr;              // BATCH: its records
  float4* tab;         // the block's segment table; entry p of this thread at tab[p * EST_BLOCK + threadIdx.x]
  int cur, nxt;
  uint4 ra, rb;        // the record of the cell the walk is in (loaded ahead, see above)

  static size_t smem_bytes() { return sizeof(float4) * 9 * EST_BLOCK; }

  __device__ TetWalker(const TetParams& p, double* smem)
      : P0(p), tab(reinterpret_cast<float4*>(smem)), cur(0), nxt(0) {
    ra = rb = make_uint4(NO_NBR, NO_NBR, NO_NBR, NO_NBR);
  }

  __device__ __forceinline__ const TetParams& prm() const {
    if constexpr (BATCH) return *Pj;
    else return P0;
  }
  __device__ __forceinline__ const uint4* recs() const {
    if constexpr (BATCH) return brec;
    else return P0.rec;
  }
  __device__ __forceinline__ void set_job(const TetParams* p) {
    Pj = p;
    brec = p->rec;
  }

  // (the address is formed from the block's base and threadIdx.x each time: no per-thread
  // pointer stays live through the cell loop)
  __device__ __forceinline__ float4& entry(int p) { return tab[p * EST_BLOCK + threadIdx.x]; }

  __device__ bool intersect(float3 o, float3 d, float* t_in) const { return box_intersect(prm().C, o, d, t_in); }

  // Point location: start from the cell that holds the centre of p's locator-grid
  // cell and walk the straight segment from that centre to p; where the segment
  // ends, the current cell holds p.  Near the domain boundary (camera-ray entry
  // points) cells are coarse and this takes a step or two.  Falls back to the
  // exact descent of the LEB hierarchy.
  __device__ bool locate(float3 p) {
    const TetParams& P = prm();
    long long c = -1;
    if (P.locator) {
      const float pc[3] = {p.x, p.y, p.z};
      int idx[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int lim = P.C[a] * P.R - 1;
        const int v = (int)floorf(pc[a] * (float)P.R);
        idx[a] = v < 0 ? 0 : (v > lim ? lim : v);
      }
      const int start = P.locator[((size_t)idx[2] * (P.C[1] * P.R) + idx[1]) * (P.C[0] * P.R) + idx[0]];
      if (start >= 0) {
        const float h = 1.0f / (float)P.R;
        const float3 ctr = make_float3(((float)idx[0] + 0.5f) * h, ((float)idx[1] + 0.5f) * h,
                                       ((float)idx[2] + 0.5f) * h);
        const float3 v = make_float3(p.x - ctr.x, p.y - ctr.y, p.z - ctr.z);
        const float len = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
        cur = start;
        c = start;
        if (len > 0.f) {
          const float inv = 1.0f / len;
          float tinv[TET_NID];
          dir_table(ff3{ff_make(v.x * inv), ff_make(v.y * inv), ff_make(v.z * inv)}, tinv);
          begin(ff3{ff_make(ctr.x), ff_make(ctr.y), ff_make(ctr.z)}, tinv);
          float t = 0.f;
          int k = 0;
          for (; k < 64; ++k) {
            const Hop hp = hop(t);
            if (!hp.ok || hp.texit >= len || !advance()) break;
            t = hp.texit;
          }
          c = k == 64 ? -1 : cur;
        }
      }
    }
    if (c < 0) c = tet_locate(P, p);
    cur = (int)c;                  // the segment that starts here loads its record (begin)
    return c >= 0;
  }

  __device__ __forceinline__ void dir_table(const ff3& d, float inv[TET_NID]) const { tet_dir_table(d, prm().invK, inv); }

  // the 32-byte record of cell i (one DRAM sector) with one 256-bit load
  __device__ __forceinline__ void load(int i, uint4& a, uint4& b) const {
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(recs() + 2 * (size_t)i));
  }

  // Per-segment table for the ray o + t d (direction table inv from dir_table):
  // nO[p] as a float-float pair and the two reciprocals of normal p; then the
  // record of the current cell, where the segment starts.
  __device__ void begin(const ff3& o, const float* inv) {
    const ff no[9] = {o.x, o.y, o.z, ff_add(o.x, o.y), ff_sub(o.x, o.y), ff_add(o.y, o.z), ff_sub(o.y, o.z),
                      ff_add(o.x, o.z), ff_sub(o.x, o.z)};
    const float scaleK = prm().scaleK;
#pragma unroll
    for (int p = 0; p < 9; ++p) entry(p) = make_float4(no[p].hi * scaleK, no[p].lo * scaleK, inv[p], inv[p | 16]);
    load(cur, ra, rb);
  }

  // Exit of the current cell from parameter t.  All four faces are evaluated; the
  // ones whose outward normal does not face the ray get a NaN parameter from the
  // table and never win, so the lanes of a warp run one instruction stream.  The
  // record of the exit neighbour is requested before returning.
  __device__ __forceinline__ Hop hop(float t) {
    const uint4 a = ra, b = rb;
    const uint32_t link[4] = {a.x, a.y, a.z, a.w};
    // the four planes: bytes 0-2, 3-5, 6-8 and 9-11 of (b.x, b.y, b.z), sign-extended
    const int c[4] = {prmt_s24(b.x, b.y, 0xA210u), prmt_s24(b.x, b.y, 0xD543u), prmt_s24(b.y, b.z, 0xC432u),
                      prmt_s24(b.z, 0u, 0xB321u)};
    const float rho = decode_density<FMT>(b.w);
    float best = INFINITY;
    uint32_t blink = NO_NBR;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      // orientation id p | s << 4 in the link's top five bits: p selects the entry, s (bit 31) the sign
      const float4 e = entry((int)((link[f] >> 27) & 15u));
      const float tf = __fmul_rn(__fsub_rn(__fsub_rn((float)c[f], e.x), e.y), (int)link[f] < 0 ? e.w : e.z);
      const bool better = tf < best;
      best = better ? tf : best;
      blink = better ? link[f] : blink;
    }
    nxt = (int)(blink & NO_NBR);
    if ((uint32_t)nxt != NO_NBR) load(nxt, ra, rb);
    Hop h;
    h.ok = best < INFINITY;
    h.texit = fmaxf(best, t);
    h.rho = rho;
    return h;
  }

  __device__ __forceinline__ bool advance() {
    if ((uint32_t)nxt == NO_NBR) return false;
    cur = nxt;                     // its record is already in ra, rb
    return true;
  }
  __device__ __forceinline__ int save() const { return cur; }
  __device__ __forceinline__ void restore(int c) { cur = c; }   // the next begin loads its record
  __device__ __forceinline__ int cell() const { return cur; }
};

// Walker parameters of a built grid, and the estimator's launch parameters for
// a camera and medium on it (render.cu).
TetParams tet_params(const GridImpl& g);
EstParams est_params(const GridImpl& g, const tg_camera& cam, const tg_medium& med, uint64_t seed);

// The persistent estimator over a grid, instantiated for the grid's density format.
template <int MODE, bool EXT = false>
void run_tet(const GridImpl& g, const EstParams& ep, cudaStream_t st) {
  const TetParams p = tet_params(g);
  switch (g.fmt) {
    case TG_DENSITY_BF16: launch_estimate<TetWalker<TG_DENSITY_BF16>, MODE, EXT>(p, ep, st); break;
    case TG_DENSITY_FP16: launch_estimate<TetWalker<TG_DENSITY_FP16>, MODE, EXT>(p, ep, st); break;
    default: launch_estimate<TetWalker<TG_DENSITY_FP32>, MODE, EXT>(p, ep, st); break;
  }
}

}  // namespace tv
