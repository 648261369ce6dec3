// The path estimator of Sec. 3 (Algorithm 1 plus sun next-event estimation) as
// one persistent kernel over a cell walker.  Every warp keeps 32 paths in
// flight; a lane whose path ends takes a new path id from a global counter
// (one atomic per warp, ballot + popc to hand out the ids), so lanes keep
// walking while the warp's other paths finish (warp-level regeneration).
//
// Precision.  Where a free flight ends depends on the optical depth consumed
// along it; a flight that starts in dense medium and ends in thin medium turns
// an error dx at its start into sigma_start / sigma_end * dx at its end, and
// these ratios multiply over the bounces of a path.  So the quantities that
// place the collisions are kept above fp32 precision, cheaply:
//  * camera rays are formed in fp64 once per path (the eye is far from the
//    medium, so a direction error becomes a large transverse offset) and kept
//    as float-float pairs;
//  * segment origins (collision points) are float-float (about 44 bits, on the
//    FP32 pipe), and the collision point inside its cell is placed in
//    float-float from the optical depth left;
//  * the per-segment plane terms P[p] . o are float-float, so exit parameters
//    carry an error relative to the distance walked, not to |o|.
// The optical depth along a segment is summed in fp32 with Kahan compensation
// (the running sum and the negated low part it lost): per-path parity with the
// fp64 oracle is the same as with a float-float sum, and the sum is three
// additions per cell.  Exit parameters, directions after scattering, densities
// and shadow walks are fp32: their errors are not amplified.  GB300's FP64 rate
// is far too low for the per-cell loop; shadow walks are the majority of all
// cell steps.
//
// SIMD efficiency.  A warp keeps 32 paths in flight, each in one of four
// states: idle (waiting for a path id), walking, event (waiting for the warp
// to process a collision, an escape or the end of a shadow walk) and done.
// Free flights and shadow walks share one step: a segment walks cells from
// parameter 0, accumulating optical depth until a limit (the sampled free path,
// or the shadow cut-off) or the boundary, with all four faces evaluated under
// predication.  Events and new paths are batched: a warp handles them when at
// least regen_min / ev_min lanes wait (or nothing else can run), so the long,
// branchy event code runs with many lanes at once.  Once the launch has no
// path ids left, a warp handles every event as soon as it comes: what remains
// is the tail of the longest paths, whose walks would otherwise wait for the
// other lanes' segments to end; a launch with no more paths than lanes does so
// from the start (a training trace of 2^17 paths: 14 ms before, 10 ms after).
//
// Walker interface (tetrahedra: walk_tet.cuh, voxels: walk_voxel.cuh):
//   bool intersect(o, d, &t_in)   slab test with the domain box (fp32)
//   bool locate(p)                current cell := the cell that holds p
//   void dir_table(d, inv)        direction table of a segment (NDIR floats)
//   void begin(o, inv)            per-thread segment table for the ray o + t d
//   Hop  hop(t)                   exit parameter of the current cell from t
//   bool advance()                move to the pending cell (false: boundary)
//   int  save() / restore(c)      remember / return to a cell
//   int  cell()                   current cell id (for traces)
#pragma once
#include "common.cuh"

namespace tv {

constexpr int EST_BLOCK = 256;
#ifndef TV_EST_MIN_BLOCKS
#define TV_EST_MIN_BLOCKS 4             // resident blocks per SM the register budget is sized for
#endif
#ifndef TV_REGEN_MIN
#define TV_REGEN_MIN 8                  // idle lanes before a warp fetches new paths
#endif
#ifndef TV_EV_MIN
#define TV_EV_MIN 12                    // waiting lanes before a warp handles events
#endif
#ifndef TV_TILE
#define TV_TILE 64                      // pixels are handed out in TV_TILE x TV_TILE tiles (when they divide the image)
#endif
#ifndef TV_STEPS_PER_ROUND
#define TV_STEPS_PER_ROUND 16           // cell steps between two warp-wide regeneration / event rounds
#endif
constexpr int SEG_STEP_LIMIT = 1 << 20;      // cells per segment before a walk gives up
// A shadow walk whose optical depth passes this value contributes at most
// E * beta * p * e^-40 < 1e-16 and is stopped early (not in trace mode).
constexpr float SHADOW_TAU_CUTOFF = 40.0f;

// What the kernel does with a finished path: add it to the image (render),
// write per-path outputs for a list of paths (trace), or write a per-path
// record for the radiance cache to complete (cached render).
enum : int { MODE_RENDER = 0, MODE_TRACE = 1, MODE_CACHED = 2 };
enum : int { S_IDLE = 0, S_WALK = 1, S_EVENT = 2, S_DONE = 3 };
enum : int { M_FREE = 0, M_SHADOW = 1 };
enum : int { EV_LIMIT = 1, EV_BOUNDARY = 2 };

struct Hop {
  float texit;
  float rho;
  bool ok;
};

struct EstParams {
  CamF cam;
  MedF med;
  uint64_t seed;
  int spp, sample_offset;
  long long total;                          // number of paths
  unsigned long long* counter;              // path-id counter, zero at launch
  float* sum;
  float* sumsq;
  tg_stats* stats;
  int regen_min;                            // idle lanes needed before a warp refills
  int ev_min;                               // waiting lanes needed before a warp handles events
  // trace mode (per-path outputs for a list of paths)
  const int32_t *px, *py, *ps;
  float* outL;
  int32_t *outFlags, *outColl;
  int64_t* outSteps;
  int32_t* seq;
  int32_t seq_cap;
  int32_t* seq_len;
  // learned radiance cache (trace and cached modes)
  int cache_depth;                          // > 0: a path ends into the cache at this collision
  float* cache_rec;                         // [path][8]: x (3), beta, d (3), L so far
  int vtx_cap;                              // trace mode: training samples from the first vtx_cap collisions
  float* vtx;                               // [path][vtx_cap][8]: x (3), target, d (3), valid
  float survive;                            // in (0, 1): Russian roulette after the last training vertex
  int roulette_from;                        // ... played after collisions >= this one (0-based)
  float ext[3];                             // domain extent in grid units (positions are stored over it)
  // extended medium (EXT instantiations): extra per-cell channels, voxel medium
  int ext_flags;                            // 1 emission, 2 per-cell albedo, 4 per-cell g, 8 voxel medium
  float emission_scale;                     // emitted radiance per unit temperature
  const float4* chan;                       // per cell: temperature, albedo, g, -
  const float* vmaj;                        // per cell: voxel majorant
  const float* voxel;                       // voxel densities [nz][ny][nx] of the voxel medium
  int vdim[3];
  float vn;                                 // voxels per grid unit (a power of two)
  // batch of grids (BATCH instantiations)
  const void* jobs;                         // BatchJob<Walker::Params>[njobs]
  int njobs;
  unsigned long long* job_done;             // per job: paths finished
  unsigned long long* job_time;             // per job: %globaltimer at its last path; [njobs]: first block's start
};

// One job of a batch (BATCH instantiations): a grid, a camera, a medium and an
// image; paths [base, base + paths) of the launch are this job's.
constexpr int BATCH_MAX_JOBS = 256;
template <class WP>
struct BatchJob {
  WP wp;                                    // the job's grid (walker parameters)
  CamF cam;
  MedF med;
  float sun_inv[32];                        // direction table of the job's sun
  float* sum;
  float* sumsq;
  uint64_t seed;
  long long base, paths;
  int spp, sample_offset;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

enum : int { EXT_EMISSION = 1, EXT_ALBEDO = 2, EXT_G = 4, EXT_VOXEL = 8 };
// Russian roulette on training paths: the draw after collision b is slot b of this stream.
constexpr uint32_t ROULETTE_STREAM = 0x10000u;
// Random numbers of delta / ratio tracking: slot k (the k-th draw of the segment)
// of stream 1 + 2b (free flight of bounce b) or 2 + 2b (its shadow ray), so that
// ending one segment early never shifts the draws of another.

// Pixel of the pix-th pixel in render order: TV_TILE x TV_TILE tiles, row-major
// tiles, row-major inside a tile (when the tiles divide the image).
__device__ __forceinline__ void render_pixel(long long pix, int W, int H, int* px, int* py) {
  if (TV_TILE > 1 && W % TV_TILE == 0 && H % TV_TILE == 0) {
    const long long tile = pix / (TV_TILE * TV_TILE);
    const int in = (int)(pix - tile * (TV_TILE * TV_TILE));
    const int tpr = W / TV_TILE;
    *px = (int)(tile % tpr) * TV_TILE + in % TV_TILE;
    *py = (int)(tile / tpr) * TV_TILE + in / TV_TILE;
  } else {
    *px = (int)(pix % W);
    *py = (int)(pix / W);
  }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
  return v;
}

// IntersectGrid (Sec. 3): slab test of the ray with the domain box [0, C] in grid space.
__device__ __forceinline__ bool box_intersect(const int C[3], float3 o, float3 d, float* t_in) {
  float tn = 0.f, tf = INFINITY;
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float hi = (float)C[a];
    if (dd[a] == 0.f) {
      if (oo[a] < 0.f || oo[a] > hi) return false;
      continue;
    }
    const float t1 = (0.f - oo[a]) / dd[a], t2 = (hi - oo[a]) / dd[a];
    tn = fmaxf(tn, fminf(t1, t2));
    tf = fminf(tf, fmaxf(t1, t2));
  }
  *t_in = tn;
  return tn < tf;
}

// EXT: the extended medium of the extra channels (Sec. 3): per-cell albedo and g,
// emission (collision estimator, beta (1 - albedo) scale T at every real
// collision), and the voxel medium -- the density at x is the voxel holding x --
// tracked against the per-cell voxel majorants: delta tracking for free flights
// (a tentative collision is real when u * majorant < rho(x), else the flight
// goes on from x with a new free path), ratio tracking for shadow rays.
// BATCH: one launch over the paths of many jobs (BatchJob): a lane's new path
// id selects its job (binary search over the jobs' first ids), and the walker,
// camera, medium, seed and image follow the job.
template <class Walker, int MODE, bool EXT = false, bool BATCH = false>
__global__ void __launch_bounds__(EST_BLOCK, TV_EST_MIN_BLOCKS) k_estimate(const typename Walker::Params wp,
                                                                          const EstParams ep) {
  constexpr bool TRACE = MODE == MODE_TRACE;
  const bool voxel = EXT && (ep.ext_flags & EXT_VOXEL);
  using Job = BatchJob<typename Walker::Params>;
  const Job* jobs = static_cast<const Job*>(ep.jobs);
  __shared__ long long job_base[BATCH ? BATCH_MAX_JOBS : 1];
  const Job* job = nullptr;                            // BATCH: the lane's current job
  float sig_l = 0.f;                                   // BATCH: its sigma per unit density (hi word)
  extern __shared__ __align__(16) double smem_d[];
  __shared__ float sun_inv[Walker::NDIR];
  Walker W(wp, smem_d);
  auto med = [&]() -> const MedF& {
    if constexpr (BATCH) return job->med;
    else return ep.med;
  };
  const MedF& M0 = ep.med;
  __shared__ unsigned long long blk_stat[8];           // the block's rarer frame counters (see below)
  if (threadIdx.x < 8) blk_stat[threadIdx.x] = 0ull;
  if (BATCH) {
    for (int i = threadIdx.x; i < ep.njobs; i += blockDim.x) job_base[i] = jobs[i].base;
    if (threadIdx.x == 0) atomicMin(ep.job_time + ep.njobs, global_ns());
  } else if (threadIdx.x == 0) {
    const MedF& M = M0;
    const ff3 w = {ff_make(M.sun_w[0]), ff_make(M.sun_w[1]), ff_make(M.sun_w[2])};
    float inv[Walker::NDIR];
    W.dir_table(w, inv);
    for (int i = 0; i < Walker::NDIR; ++i) sun_inv[i] = inv[i];
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;

  int state = S_IDLE, mode = M_FREE, ev = 0;
  long long pid = 0;
  uint32_t pixel = 0, sample = 0;
  ff3 o = {ff_make(0.f), ff_make(0.f), ff_make(0.f)};   // segment origin
  ff3 d = o;                                           // path direction (float-float on camera rays)
  float t = 0.f;                                       // segment parameter
  ff acc = ff_make(0.f);                               // optical depth of the segment so far
  float lim = 0.f;                                     // its limit: free path, or shadow cut-off
  float beta = 1.f;
  ff L = ff_make(0.f);
  int bounce = 0, seg_steps = 0, flags = 0, ncoll = 0, saved = 0, seqn = 0;
  int nv = 0;                                          // cache training vertices recorded
  bool queried = false;                                // the path ended into the cache
  uint32_t nseg = 0;                                   // EXT: delta-tracking draws of the current segment
  float gcur = M0.g;                                   // EXT: phase parameter of the last collision
  float Tr = 1.f;                                      // EXT: ratio-tracking transmittance
  ff3 os = {ff_make(0.f), ff_make(0.f), ff_make(0.f)}; // EXT: shadow segment origin (voxel medium)
  long long psteps = 0;
  // the frame's counters: cell steps in registers (added at every segment end), the
  // rarer ones -- paths, collisions, escapes, truncations, step limits, misses -- in
  // one shared set per block, so that they hold no registers through the cell loop
  uint32_t c_steps = 0, c_shadow = 0;
  auto bump = [&](int i) {
    if (ep.stats) atomicAdd(&blk_stat[i], 1ull);
  };

  auto record = [&](int v) {
    if (TRACE) {
      if (seqn < ep.seq_cap) ep.seq[pid * ep.seq_cap + seqn] = v;
      ++seqn;
    }
  };
  auto finish = [&]() {
    bump(0);
    const float Lf = ff_float(L);
    if (TRACE) {
      if (ep.outL) ep.outL[pid] = Lf;
      if (ep.outFlags) ep.outFlags[pid] = flags;
      if (ep.outColl) ep.outColl[pid] = ncoll;
      if (ep.outSteps) ep.outSteps[pid] = psteps;
      if (ep.seq_len) ep.seq_len[pid] = seqn < ep.seq_cap ? seqn : ep.seq_cap;
      if (ep.vtx) {
        // training targets: the rest of this path's estimate after each recorded vertex
        float4* v = reinterpret_cast<float4*>(ep.vtx) + 2 * (long long)ep.vtx_cap * pid;
        for (int j = 0; j < ep.vtx_cap; ++j) {
          float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
          if (j < nv) {
            a = v[2 * j];
            b = v[2 * j + 1];
            const float bj = a.w;
            a.w = bj > 0.f ? (Lf - b.w) / bj : 0.f;
            b.w = bj > 0.f ? 1.f : 0.f;
            if (bj <= 0.f) a = b = make_float4(0.f, 0.f, 0.f, 0.f);
          }
          v[2 * j] = a;
          v[2 * j + 1] = b;
        }
      }
    }
    if (MODE == MODE_RENDER) {
      float* sum = BATCH ? job->sum : ep.sum;
      float* sumsq = BATCH ? job->sumsq : ep.sumsq;
      atomicAdd(sum + pixel, Lf);
      if (sumsq) atomicAdd(sumsq + pixel, Lf * Lf);
      if (BATCH) {
        const long long jb = job - jobs;
        if (atomicAdd(ep.job_done + jb, 1ull) + 1ull == (unsigned long long)job->paths)
          ep.job_time[jb] = global_ns();
      }
    }
    if (MODE != MODE_RENDER && ep.cache_rec && !queried) {
      float4* r = reinterpret_cast<float4*>(ep.cache_rec) + 2 * pid;
      r[0] = make_float4(0.f, 0.f, 0.f, 0.f);
      r[1] = make_float4(0.f, 0.f, 0.f, Lf);
    }
    state = S_IDLE;
  };
  // cells of a finished segment into the frame's counters (free flights, shadow rays)
  auto count_steps = [&](int n) {
    if (mode == M_FREE) c_steps += (uint32_t)n;
    else c_shadow += (uint32_t)n;
  };
  auto seedv = [&]() -> uint64_t {
    if constexpr (BATCH) return job->seed;
    else return ep.seed;
  };
  auto draw = [&](uint32_t stream) { return rng_u(seedv(), pixel, sample, nseg++, stream); };
  // voxel medium: density of the voxel holding x (exact floor of the float-float coordinate)
  auto voxel_at = [&](const ff3& x) -> float {
    const ff xs[3] = {x.x, x.y, x.z};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float hs = xs[a].hi * ep.vn;
      float fl = floorf(hs);
      if (fl == hs && xs[a].lo < 0.f) fl -= 1.f;
      int i = (int)fl;
      idx[a] = i < 0 ? 0 : (i > ep.vdim[a] - 1 ? ep.vdim[a] - 1 : i);
    }
    return __ldg(ep.voxel + ((size_t)idx[2] * ep.vdim[1] + idx[1]) * ep.vdim[0] + idx[0]);
  };
  // a free flight from o along d: SampleFreePath gives the optical depth to consume
  auto start_free = [&](int b) {
    float inv[Walker::NDIR];
    W.dir_table(d, inv);
    W.begin(o, inv);
    t = 0.f;
    acc = ff_make(0.f);
    lim = -logf(1.0f - rng_u(seedv(), pixel, sample, 2 + 3 * b));
    seg_steps = 0;
    nseg = 0;
    mode = M_FREE;
    state = S_WALK;
  };

  int ev_min = ep.ev_min;                       // 1 once the launch's path ids are all taken
  for (;;) {
    // ---- regeneration: idle lanes of the warp take consecutive path ids ----
    const unsigned idle = __ballot_sync(~0u, state == S_IDLE);
    const unsigned busy = __ballot_sync(~0u, state == S_WALK || state == S_EVENT);
    if (idle && (busy == 0 || __popc(idle) >= ep.regen_min)) {
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(ep.counter, (unsigned long long)__popc(idle));
      base = __shfl_sync(~0u, base, leader);
      if (base + (unsigned long long)__popc(idle) >= (unsigned long long)ep.total) ev_min = 1;
      if (state == S_IDLE) {
        pid = (long long)(base + __popc(idle & lt));
        if (pid >= ep.total) {
          state = S_DONE;
        } else {
          // ---- a new path: camera ray, IntersectGrid, GridIntersectionPoint ----
          int px, py, s;
          if (TRACE) {
            px = ep.px[pid]; py = ep.py[pid]; s = ep.ps[pid];
          } else {
            // all samples of a pixel together; pixels tile by tile (row-major tiles), which keeps the
            // cells the warps in flight touch close together
            long long local = pid;
            int spp = ep.spp, soff = ep.sample_offset, cw = ep.cam.W, chh = ep.cam.H;
            if constexpr (BATCH) {
              // the job of this path: last job whose first path id <= pid
              int lo = 0, hi = ep.njobs;
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (job_base[mid] <= pid) lo = mid + 1; else hi = mid;
              }
              job = jobs + (lo - 1);
              W.set_job(&job->wp);
              sig_l = job->med.sig_hi;
              local = pid - job->base;
              spp = job->spp; soff = job->sample_offset; cw = job->cam.W; chh = job->cam.H;
            }
            const long long pix = local / spp;
            s = soff + (int)(local - pix * spp);
            render_pixel(pix, cw, chh, &px, &py);
          }
          const int camW = BATCH ? job->cam.W : ep.cam.W;
          pixel = (uint32_t)(py * camW + px);
          sample = (uint32_t)s;
          flags = 0; ncoll = 0; psteps = 0; seqn = 0; L = ff_make(0.f); beta = 1.f; bounce = 0;
          nv = 0; queried = false;
          const MedF& M = med();
          if (EXT) gcur = M.g;
          const double u0 = rng_u(seedv(), pixel, sample, 0), u1 = rng_u(seedv(), pixel, sample, 1);
          const CamF& c = BATCH ? job->cam : ep.cam;
          const double sx = (2.0 * (((double)px + u0) / (double)c.W) - 1.0) * c.tanF * c.aspect;
          const double sy = (2.0 * (((double)py + u1) / (double)c.H) - 1.0) * c.tanF;
          double dx = c.fwd[0] + sx * c.right[0] - sy * c.up[0];
          double dy = c.fwd[1] + sx * c.right[1] - sy * c.up[1];
          double dz = c.fwd[2] + sx * c.right[2] - sy * c.up[2];
          const double inv = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
          dx *= inv; dy *= inv; dz *= inv;
          d = ff3{ff{(float)dx, (float)(dx - (double)(float)dx)}, ff{(float)dy, (float)(dy - (double)(float)dy)},
                  ff{(float)dz, (float)(dz - (double)(float)dz)}};
          const float3 dir = make_float3(d.x.hi, d.y.hi, d.z.hi);
          const float3 eye = make_float3((float)c.eye[0], (float)c.eye[1], (float)c.eye[2]);
          float tin;
          if (!W.intersect(eye, dir, &tin)) {
            L = ff_make(M.Lenv); flags = 4; bump(7); bump(4);
            finish();
          } else {
            // the entry point: any error along the ray is harmless (no medium outside the box)
            o = ff3{ff_add(ff{(float)c.eye[0], (float)(c.eye[0] - (double)(float)c.eye[0])}, ff_mul_f(d.x, tin)),
                    ff_add(ff{(float)c.eye[1], (float)(c.eye[1] - (double)(float)c.eye[1])}, ff_mul_f(d.y, tin)),
                    ff_add(ff{(float)c.eye[2], (float)(c.eye[2] - (double)(float)c.eye[2])}, ff_mul_f(d.z, tin))};
            if (!W.locate(make_float3(ff_float(o.x), ff_float(o.y), ff_float(o.z)))) {
              flags = 16;
              finish();
            } else {
              start_free(0);
            }
          }
        }
      }
    }

    // ---- events, handled together by the lanes that wait for one ----
    const unsigned pend = __ballot_sync(~0u, state == S_EVENT);
    const unsigned walking = __ballot_sync(~0u, state == S_WALK);
    if (pend && (walking == 0 || __popc(pend) >= ev_min) && state == S_EVENT) {
      const MedF& M = med();
      const float* const sun_tab = BATCH ? job->sun_inv : sun_inv;
      if (mode == M_FREE) {
        if (ev == EV_LIMIT) {
          // collision at parameter acc: albedo weight, then next-event estimation towards the sun
          o = ff3{ff_add(o.x, ff_mul(acc, d.x)), ff_add(o.y, ff_mul(acc, d.y)), ff_add(o.z, ff_mul(acc, d.z))};
          bool real = true;
          if (voxel) {
            // delta tracking: a tentative collision against the cell's voxel majorant
            const float rx = voxel_at(o);
            const float mj = __ldg(ep.vmaj + W.cell());
            real = draw(1u + 2u * bounce) * mj < rx;
            if (!real) {
              // a null collision: fly on from o with a fresh free path, in the same cell
              record(-1);
              float inv[Walker::NDIR];
              W.dir_table(d, inv);
              W.begin(o, inv);
              t = 0.f;
              acc = ff_make(0.f);
              lim = -logf(1.0f - draw(1u + 2u * bounce));
              seg_steps = 0;
              state = S_WALK;
            }
          }
          if (real) {
            if (EXT) {
              const float4 ch = __ldg(ep.chan + W.cell());
              const float alb = (ep.ext_flags & EXT_ALBEDO) ? ch.y : M.albedo;
              if (ep.ext_flags & EXT_G) gcur = ch.z;
              if (ep.ext_flags & EXT_EMISSION) L = ff_add(L, ff_make(beta * (1.0f - alb) * ep.emission_scale * ch.x));
              beta *= alb;
            } else {
              beta *= M.albedo;
            }
            ++ncoll; bump(3);
            record(-1);
            saved = W.save();
            W.begin(o, sun_tab);
            t = 0.f;
            acc = ff_make(0.f);
            if (voxel) {
              Tr = 1.f;
              os = o;
              nseg = 0;
              lim = -logf(1.0f - draw(2u + 2u * bounce));
            } else {
              lim = TRACE ? INFINITY : SHADOW_TAU_CUTOFF;
            }
            seg_steps = 0;
            mode = M_SHADOW;
            state = S_WALK;
          }
        } else {
          L = ff_add(L, ff_make(beta * M.Lenv)); bump(4);
          finish();
        }
      } else if (voxel && ev == EV_LIMIT) {
        // ratio tracking: a tentative collision on the shadow ray scales the transmittance
        const ff3 w = {ff_make(M.sun_w[0]), ff_make(M.sun_w[1]), ff_make(M.sun_w[2])};
        os = ff3{ff_add(os.x, ff_mul(acc, w.x)), ff_add(os.y, ff_mul(acc, w.y)), ff_add(os.z, ff_mul(acc, w.z))};
        Tr *= 1.0f - voxel_at(os) / __ldg(ep.vmaj + W.cell());
        if (!TRACE && Tr < 8.271806e-25f) {
          // below 2^-80 the sun adds nothing visible: end the walk here (not in trace mode)
          Tr = 0.f;
          ev = EV_BOUNDARY;
        } else {
          W.begin(os, sun_tab);
          t = 0.f;
          acc = ff_make(0.f);
          lim = -logf(1.0f - draw(2u + 2u * bounce));
          seg_steps = 0;
          state = S_WALK;
        }
      } else {
        // the shadow walk ended: add the sun seen through it
        record(-1);
        const float tr = voxel ? Tr : (ev == EV_BOUNDARY ? expf(-ff_float(acc)) : 0.0f);
        const float gg = EXT ? gcur : M.g;
        const float cs = d.x.hi * M.sun_w[0] + d.y.hi * M.sun_w[1] + d.z.hi * M.sun_w[2];
        L = ff_add(L, ff_make(beta * hg_eval(gg, cs) * M.E * tr));
        const float4 xq = make_float4(ff_float(o.x) / ep.ext[0], ff_float(o.y) / ep.ext[1],
                                      ff_float(o.z) / ep.ext[2], beta);
        if (TRACE && ep.vtx && nv < ep.vtx_cap) {
          float4* v = reinterpret_cast<float4*>(ep.vtx) + 2 * ((long long)ep.vtx_cap * pid + nv);
          v[0] = xq;
          v[1] = make_float4(d.x.hi, d.y.hi, d.z.hi, ff_float(L));
          ++nv;
        }
        if (bounce + 1 >= M.max_bounces) {
          flags |= 2; bump(5);
          finish();
        } else if (MODE != MODE_RENDER && ep.cache_depth > 0 && bounce + 1 == ep.cache_depth) {
          // the path ends into the radiance cache, which stands for the rest of it
          float4* r = reinterpret_cast<float4*>(ep.cache_rec) + 2 * pid;
          r[0] = xq;
          r[1] = make_float4(d.x.hi, d.y.hi, d.z.hi, ff_float(L));
          queried = true;
          finish();
        } else if (TRACE && ep.vtx && nv >= ep.vtx_cap && bounce >= ep.roulette_from && ep.survive > 0.f &&
                   ep.survive < 1.f &&
                   rng_u(seedv(), pixel, sample, (uint32_t)bounce, ROULETTE_STREAM) >= ep.survive) {
          // a training path past its last training vertex ends by Russian roulette
          flags |= 32;
          finish();
        } else {
          // (a training path that survives the roulette carries throughput / survive)
          if (TRACE && ep.vtx && nv >= ep.vtx_cap && bounce >= ep.roulette_from && ep.survive > 0.f &&
              ep.survive < 1.f)
            beta = __fdiv_rn(beta, ep.survive);
          // SamplePhaseFunction, then a new free flight from the collision point
          const float3 nd = hg_scatter(gg, rng_u(seedv(), pixel, sample, 3 + 3 * bounce),
                                       rng_u(seedv(), pixel, sample, 4 + 3 * bounce),
                                       make_float3(d.x.hi, d.y.hi, d.z.hi));
          d = ff3{ff_make(nd.x), ff_make(nd.y), ff_make(nd.z)};
          ++bounce;
          W.restore(saved);
          start_free(bounce);
        }
      }
    }
    if (__all_sync(~0u, state == S_DONE)) break;

    // ---- cells: ReadDensity and MarchThroughCells (or the shadow walk) ----
#pragma unroll 1
    for (int k = 0; k < TV_STEPS_PER_ROUND && state == S_WALK; ++k) {
      record(W.cell());
      ++seg_steps;
      if (TRACE) ++psteps;
      const Hop h = W.hop(t);
      if (!h.ok) { count_steps(seg_steps - 1); flags |= 16; finish(); break; }
      // the voxel medium walks the cells' majorants
      const float rho = voxel ? __ldg(ep.vmaj + W.cell()) : h.rho;
      // optical depth of the cell, (sigma_unit * rho) * (t_exit - t), added to the segment's
      // sum with Kahan compensation: acc.hi is the running sum, acc.lo the negated low part
      // it lost (the sum is acc.hi - acc.lo)
      const float sigf = BATCH ? sig_l : M0.sig_hi;
      const float y = (sigf * rho) * (h.texit - t) - acc.lo;
      const float sum = acc.hi + y;
      // (the limit is a float: comparing the rounded sum decides all but exact ties, which
      // only move a collision by less than one unit in the last place of the free path)
      if (rho > 0.f && !(sum < lim)) {
        // the segment's optical-depth limit falls inside this cell: place it in float-float
        const ff sig = two_prod(sigf, rho);
        acc = ff{acc.hi, -acc.lo};
        if (mode == M_FREE || voxel) acc = ff_add(ff_make(t), ff_div(ff_sub(ff_make(lim), acc), sig));
        count_steps(seg_steps);
        ev = EV_LIMIT;
        state = S_EVENT;
        break;
      }
      acc.lo = (sum - acc.hi) - y;
      acc.hi = sum;
      t = h.texit;
      if (!W.advance()) {
        acc = ff{acc.hi, -acc.lo};          // the segment's optical depth as a float-float value
        count_steps(seg_steps);
        ev = EV_BOUNDARY;
        state = S_EVENT;
      }
    }
    // a segment that walks too many cells (a corrupt grid) ends its path
    if (state == S_WALK && seg_steps >= SEG_STEP_LIMIT) {
      count_steps(seg_steps);
      flags |= 8; bump(6);
      finish();
    }
  }

  if (ep.stats) {
    const unsigned long long ws = warp_sum(c_steps), wsh = warp_sum(c_shadow);
    if (lane == 0) {
      atomicAdd(&blk_stat[1], ws);
      atomicAdd(&blk_stat[2], wsh);
    }
  }
  __syncthreads();
  if (ep.stats && threadIdx.x < 8 && blk_stat[threadIdx.x])
    atomicAdd(reinterpret_cast<unsigned long long*>(ep.stats) + threadIdx.x, blk_stat[threadIdx.x]);
}

// Launch the persistent estimator: as many resident blocks as fit, one wave.
template <class Walker, int MODE, bool EXT = false, bool BATCH = false>
void launch_estimate(const typename Walker::Params& wp, const EstParams& ep, cudaStream_t st, int blocks_per_sm = 0) {
  int dev = 0, sms = 0, per_sm = 0;
  TV_CUDA(cudaGetDevice(&dev));
  TV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t shm = Walker::smem_bytes();
  TV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_estimate<Walker, MODE, EXT, BATCH>, EST_BLOCK,
                                                       shm));
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  if (per_sm < 1) per_sm = 1;
  long long blocks = (long long)sms * per_sm;
  const long long need = (ep.total + EST_BLOCK - 1) / EST_BLOCK;
  if (blocks > need) blocks = need < 1 ? 1 : need;
  // a launch whose paths all start in the first wave is its own tail: handle events at once
  EstParams e = ep;
  if (e.total <= blocks * EST_BLOCK) e.ev_min = 1;
  k_estimate<Walker, MODE, EXT, BATCH><<<(unsigned)blocks, EST_BLOCK, shm, st>>>(wp, e);
  TV_LAUNCH();
}

}  // namespace tv
