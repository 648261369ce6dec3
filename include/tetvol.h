/*
 * tetvol: GB300 (sm_103a) path tracing of heterogeneous media stored on
 * adaptive, conforming tetrahedral grids built by longest-edge bisection,
 * after Benyoub & Dupuy, "Adaptive Tetrahedral Grids for Volumetric
 * Path-Tracing" (SIGGRAPH Talks 2025).
 *
 * C ABI of libtetvol.so.  Conventions for every entry point:
 *  - pointers named *device* or documented as device memory are CUDA device
 *    pointers owned by the caller; the library never frees them;
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream); work is
 *    enqueued on it and the call returns without waiting unless stated;
 *  - the return value is TG_OK or a negative TG_E* status; no C++ exception
 *    crosses the ABI; tg_error_string() names a status.
 *
 * Spaces.  World space is where the volume box and the camera live.  Grid
 * space tiles the volume box with unit cubes of n^3 voxels, n the largest
 * power of two dividing nx, ny and nz; a cube is n * voxel_size world units.
 * Vertex coordinates are integers in units of 2^-K cube, with
 * K = max(ceil(max_depth / 3) + 1, log2(n) + 1).
 */
#ifndef TETVOL_H
#define TETVOL_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TG_OK = 0,
  TG_EINVAL = -1,        /* bad argument (sizes, NULL, limits)                         */
  TG_ENOMEM = -2,        /* device allocation failed                                   */
  TG_ECUDA = -3,         /* a CUDA call failed                                         */
  TG_ESTEPLIMIT = -4,    /* a walk exceeded its step limit (corrupt grid)              */
  TG_EROUNDLIMIT = -5,   /* the build did not converge within its round limit          */
  TG_EGRID = -6          /* the grid is not conforming (a face without its partner)    */
};

enum { TG_DENSITY_FP32 = 0, TG_DENSITY_BF16 = 1, TG_DENSITY_FP16 = 2 };

/* Pinhole camera (world space).  Film x grows with the right vector
 * normalize(cross(forward, up)), film y grows downwards. */
typedef struct {
  float pos[3], target[3], up[3];
  float fov_y_deg;
  int32_t width, height;
} tg_camera;

/* Homogeneous phase function and lights of the medium.  sigma_scale is the
 * extinction per world unit at density 1; sun_dir is the unit direction the
 * sunlight travels; the environment radiance is collected by escaping paths. */
typedef struct {
  float albedo, g, sigma_scale;
  int32_t max_bounces;              /* maximum number of collisions of a path (>= 1) */
  float sun_dir[3];
  float sun_irradiance, env_radiance;
} tg_medium;

/* Dense density volume density[nz][ny][nx] (x fastest), values in [0, 1]. */
typedef struct {
  float box_min[3];
  float voxel_size;
  int32_t nx, ny, nz;
} tg_volume_desc;

/* Render counters in device memory, accumulated with atomics (zero them first). */
typedef struct {
  unsigned long long paths;         /* paths completed                                   */
  unsigned long long tet_steps;     /* cells entered by free-flight segments             */
  unsigned long long shadow_steps;  /* cells entered by shadow (next-event) segments     */
  unsigned long long collisions;
  unsigned long long escapes;       /* paths that left the grid (incl. camera misses)    */
  unsigned long long truncated;     /* paths stopped at max_bounces                      */
  unsigned long long step_limit;    /* segments stopped by the walk step limit           */
  unsigned long long misses;        /* camera rays that miss the grid                    */
} tg_stats;

typedef struct tg_grid tg_grid;    /* device-resident grid, owned by the library */

/*
 * leb_build - Sec. 2 (Grid Construction): build the adaptive conforming grid.
 * Six Kuhn tetrahedra per unit cube are bisected by Maubach's longest-edge rule
 * while the subdivision criteria select them:
 *   split(T) = depth(T) < max_depth
 *            and (max(D) - min(D)) / mean(D) > variation_threshold  (criterion 1)
 *            and T is not entirely outside the view frustum and its longest edge
 *                spans more than target_footprint_px pixels at its nearest depth
 *                                                                    (criterion 2)
 * with D the density values of the voxel centres inside the closed tetrahedron
 * (the voxel of its centroid when there are none); and every leaf holding a
 * vertex at one of its edge midpoints is bisected too, until no leaf is
 * selected (the conformity-preserving propagation of Sec. 2).
 *   density  float[nz][ny][nx]: device memory, or page-locked (pinned) host
 *            memory that the device addresses directly -- the build reads each
 *            value once, in its quantisation kernel, so a pinned host volume
 *            needs no separate upload.  Pageable host memory is refused with
 *            TG_EINVAL before any kernel runs.  Read during the call only.
 *   cam      host struct, or NULL to switch the camera criterion off (as does
 *            target_footprint_px <= 0); variation_threshold < 0 switches
 *            criterion 1 off.
 *   max_depth in [0, 50]; density_format one of TG_DENSITY_*.
 * Synchronous: returns after the grid is complete.  *out is released with
 * tg_grid_free.  Errors: TG_EINVAL, TG_ENOMEM, TG_ECUDA, TG_EROUNDLIMIT, TG_EGRID.
 */
int leb_build(const float* density, const tg_volume_desc* vol, const tg_camera* cam,
              float target_footprint_px, float variation_threshold, int32_t max_depth,
              int32_t density_format, void* cuda_stream, tg_grid** out);

/*
 * leb_rebuild - leb_build for a new camera (or footprint) on the same volume,
 * reusing a previous grid of it: every node of the LEB tree that `prev` had
 * (leaves and interior nodes, whose statistics a grid keeps) takes its
 * statistics of D from there instead of scanning voxels; only nodes that `prev`
 * never had are scanned.  The result is identical to leb_build with the same
 * arguments.  Only `density` and the volume description must be those `prev`
 * was built from (the statistics depend on nothing else; dims and K are
 * checked, TG_EINVAL otherwise): camera, footprint, threshold and max_depth may
 * all change.  `prev` must be a built grid (not imported) and stays valid.
 */
int leb_rebuild(const tg_grid* prev, const float* density, const tg_volume_desc* vol, const tg_camera* cam,
                float target_footprint_px, float variation_threshold, int32_t max_depth, int32_t density_format,
                void* cuda_stream, tg_grid** out);

/* tg_grid_info - size and shape of a grid built by leb_build (Sec. 2): the
 * number of leaves (tetrahedra), the deepest LEB level present, the build's
 * rounds of bisection.  Any output pointer may be NULL.  bytes: device bytes the
 * renderer reads (records + codes); K: vertex coordinate scale exponent.
 * Host-only (no CUDA call).  TG_EINVAL for a NULL grid. */
int tg_grid_info(const tg_grid* g, int64_t* num_tets, int32_t* max_depth, int64_t* bytes,
                 int32_t* K, int32_t* rounds);

/*
 * tg_grid_export - copy the grid into caller-owned device arrays (any may be NULL),
 * cells in depth-first order of their LEB codes:
 *   codes    uint64[N]   root id << 56 | path bits left-aligned in bits 55..6 | depth
 *   verts    int32[N][4][3]  LEB-ordered vertices (x0..x3), units of 2^-K cube
 *   tag      int32[N]    Maubach tag k: the refinement edge is x0-xk
 *   nbr      int32[N][4] cell across the face opposite vertex f, -1 on the boundary
 *   nid      uint8[N][4] face orientation id p + 9 s: outward normal (-1)^s P[p],
 *                        P = {x, y, z, x+y, x-y, y+z, y-z, x+z, x-z} (Sec. 3: 18 orientations)
 *   plane    float[N][4] plane offset P[p] . v of the face, in cubes
 *   density  float[N]    stored density of the cell (after BF16/FP16 rounding)
 *   majorant float[N]    max(D)
 *   count, sum, qmin, qmax: statistics of D in units of 2^-24 density
 * Asynchronous on cuda_stream.
 */
int tg_grid_export(const tg_grid* g, uint64_t* codes, int32_t* verts, int32_t* tag, int32_t* nbr,
                   uint8_t* nid, float* plane, float* density, float* majorant, uint32_t* count,
                   uint64_t* sum, uint32_t* qmin, uint32_t* qmax, void* cuda_stream);

/*
 * tg_grid_import - wrap grid arrays produced elsewhere (same layout as the export;
 * device pointers, copied) into a tg_grid for rendering.  vol describes the box;
 * K the vertex scale exponent.  Lets the renderer be tested on a grid built by
 * another implementation.  Synchronous.
 */
int tg_grid_import(const tg_volume_desc* vol, int32_t K, int64_t num_tets, const uint64_t* codes,
                   const int32_t* nbr, const uint8_t* nid, const float* plane, const float* density,
                   int32_t density_format, void* cuda_stream, tg_grid** out);

/* tg_grid_free - release a grid and every device buffer it owns.  The paper has
 * no counterpart (resource management of this library).  NULL is ignored; the
 * grid must not be in use by work still queued on any stream. */
void tg_grid_free(tg_grid* g);

/* tg_release_build_memory - leb_build, leb_rebuild and tg_grid_channels take
 * their buffers from a stream-ordered memory pool the library keeps per device,
 * and freed buffers stay in it for the next build (a production-size build's
 * temporaries are tens of GB; reusing them saves about 45 ms per build).  This
 * call waits for the current device and returns the pool's unused memory to the
 * driver.  The paper has no counterpart.  TG_ECUDA if CUDA fails. */
int tg_release_build_memory(void);

/*
 * tet_render - Sec. 3 (Algorithm 1) on the grid: W*H*spp paths, path (px, py, s)
 * for s in [sample_offset, sample_offset + spp), each a camera ray through the
 * jittered pixel that walks the grid cell by cell (exit face among the <= 3
 * faces whose stored normal faces the ray, neighbour link to the next cell),
 * consumes an exponential optical depth per flight, scatters by
 * Henyey-Greenstein, adds the sun at every collision through a shadow walk, and
 * adds the environment when it leaves the grid.  Each path's estimate f is added
 * to accum_sum[py][px] and f^2 to accum_sumsq (may be NULL); both are
 * caller-owned device float[H][W], never cleared by the call, so progressive
 * calls compose.  stats: device tg_stats or NULL.  Random numbers are Philox4x32-10,
 * key (seed lo, seed hi ^ pixel), counter (s, slot / 4, 0, 0).
 * Asynchronous.  Errors: TG_EINVAL (also when sample_offset + spp > INT32_MAX:
 * sample indices are int32, and the render, grid_render, tet_render_ext,
 * tet_render_cached, tet_render_noalloc and batch entry points all refuse a range
 * that would wrap), TG_ECUDA.  A walk that exceeds its step
 * limit ends its path and is counted in stats->step_limit.
 * Each call takes its own scratch (the path counter) from the library's
 * stream-ordered pool on its stream, so calls on different streams may overlap,
 * on the same grid or not.
 */
int tet_render(const tg_grid* g, const tg_camera* cam, const tg_medium* med, int32_t spp, uint64_t seed,
               int32_t sample_offset, float* accum_sum, float* accum_sumsq, tg_stats* stats,
               void* cuda_stream);

/*
 * grid_render - the regular-grid comparator (the "1024^3 regular grid" reference
 * of Sec. 4): the same estimator as tet_render, walking the voxels of the dense
 * volume with a 3D DDA instead of the tetrahedra.  Same arguments and semantics.
 * Like tet_render, each call takes its own scratch on its stream.
 */
int grid_render(const float* density, const tg_volume_desc* vol, const tg_camera* cam, const tg_medium* med,
                int32_t spp, uint64_t seed, int32_t sample_offset, float* accum_sum, float* accum_sumsq,
                tg_stats* stats, void* cuda_stream);

/*
 * tet_trace_paths / grid_trace_paths - per-path outputs for n listed paths
 * (px, py, sample: device int32[n]): estimate L, flags (bit1 truncated, bit2
 * camera miss, bit3 step limit), collisions, cells entered, and (tet only) the
 * visited cell sequence of all segments with -1 after each segment, truncated
 * to seq_cap (seq: device int32[n][seq_cap], seq_len: int32[n]).  Outputs may
 * be NULL.  Asynchronous.
 */
int tet_trace_paths(const tg_grid* g, const tg_camera* cam, const tg_medium* med, uint64_t seed, int64_t n,
                    const int32_t* px, const int32_t* py, const int32_t* sample, float* L, int32_t* flags,
                    int32_t* collisions, int64_t* steps, int32_t* seq, int32_t seq_cap, int32_t* seq_len,
                    void* cuda_stream);
int grid_trace_paths(const float* density, const tg_volume_desc* vol, const tg_camera* cam,
                     const tg_medium* med, uint64_t seed, int64_t n, const int32_t* px, const int32_t* py,
                     const int32_t* sample, float* L, int32_t* flags, int32_t* collisions, int64_t* steps,
                     void* cuda_stream);

/*
 * tet_optical_depth - the walk alone (Sec. 3): for n rays in grid space
 * (origin, dir: device float[n][3]), the optical depth sigma * sum(rho_T * l_T)
 * from where the ray enters the grid to where it leaves, the cells entered and
 * the visited sequence (as above, one segment).  Asynchronous.
 */
int tet_optical_depth(const tg_grid* g, int64_t n, const float* origin, const float* dir, float sigma,
                      float* tau, int64_t* steps, int32_t* seq, int32_t seq_cap, int32_t* seq_len,
                      void* cuda_stream);

/*
 * tet_render_noalloc - the frame of tet_render, for callers that may not let a
 * library allocate device memory (applications that hand out all device memory
 * from their own pool or budget, and loops that cannot afford the implicit
 * synchronisation of cudaMalloc).  The paper has no counterpart: this is a
 * property of the library, not of the method.
 *   Allocates nothing.  Its scratch (the estimator's path counter and 16 bytes
 *   per path) is a static device array of TG_NOALLOC_MAX_PATHS paths (8 MiB),
 *   held by every device that loads the library until the process exits.
 *   W * H * spp above TG_NOALLOC_MAX_PATHS is rejected with TG_EINVAL.
 *   The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 *   All calls share the array and its contents persist between calls: calls
 *   that overlap on the GPU (other streams, other threads) race.  Serialise them.
 *   Same arguments and accumulation (+=) as tet_render, without stats; each
 *   pixel's samples are summed in sample order, so the image is the same from
 *   run to run.
 */
#define TG_NOALLOC_MAX_PATHS (1 << 19)
int tet_render_noalloc(const tg_grid* g, const tg_camera* cam, const tg_medium* med, int32_t spp, uint64_t seed,
                       int32_t sample_offset, float* accum_sum, float* accum_sumsq, void* cuda_stream);

/* ==========================================================================
 * Extra channels and the voxel medium.  Sec. 3: the grid "supports extra
 * channels for, e.g., temperature, albedo, phase function parameters"; the
 * explosion of the paper's last figure has density and temperature.
 * ========================================================================== */

/*
 * tg_grid_channels - per-cell channels of a grid built by leb_build (not of an
 * imported grid: TG_EINVAL): for each of temperature, albedo and anisotropy
 * a (device float[nz][ny][nx] on the grid's voxel lattice, values in [0, 1],
 * NULL = absent), the mean over the cell's D (the voxels whose centres lie in
 * the closed cell, else the centroid's voxel), quantised like the density
 * (round(v 2^24)); the phase parameter is g = 2a - 1 clamped to [-0.99, 0.99].
 * Also the cell's voxel majorant (max q + 1) / 2^24 over the voxels of
 * `density` touching the cell's bounding box: at least the voxel density
 * anywhere in the cell.  Replaces earlier channels.  Synchronous.
 */
int tg_grid_channels(tg_grid* g, const float* density, const float* temperature, const float* albedo,
                     const float* aniso, void* cuda_stream);
/* chan: device float[N][4] (temperature, albedo, g, 0), vmaj: device float[N]; NULL allowed. */
int tg_grid_export_channels(const tg_grid* g, float* chan, float* vmaj, void* cuda_stream);

enum { TG_EXT_EMISSION = 1, TG_EXT_ALBEDO = 2, TG_EXT_G = 4, TG_EXT_VOXEL = 8 };
/* The extended medium of a render (flags are ORed; channels must have been computed):
 *  EMISSION: at every real collision the path adds beta (1 - albedo) Le, Le =
 *    emission_scale * temperature of the cell (collision estimator of emission);
 *  ALBEDO, G: the cell's albedo / g replace the medium's;
 *  VOXEL: the medium is `density` (device float[nz][ny][nx], the grid's voxel
 *    lattice): the density at x is the voxel holding x.  Free flights are
 *    tracked against the cells' voxel majorants (delta tracking: a tentative
 *    collision is real when u * majorant < rho(x), in fp32), shadow rays by
 *    ratio tracking; the k-th such draw of the free flight (shadow ray) of
 *    bounce b uses Philox counter (s, k / 4, 1 + 2b (2 + 2b), 0), word k % 4. */
typedef struct {
  int32_t flags;
  float emission_scale;
  const float* density;
} tg_ext;

/* tet_render / tet_trace_paths with the extended medium (same arguments and
 * semantics otherwise; the trace variant has no visited-cell output). */
int tet_render_ext(const tg_grid* g, const tg_camera* cam, const tg_medium* med, const tg_ext* ext, int32_t spp,
                   uint64_t seed, int32_t sample_offset, float* accum_sum, float* accum_sumsq, tg_stats* stats,
                   void* cuda_stream);
int tet_trace_ext_paths(const tg_grid* g, const tg_camera* cam, const tg_medium* med, const tg_ext* ext,
                        uint64_t seed, int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                        float* L, int32_t* flags, int32_t* collisions, int64_t* steps, void* cuda_stream);

/* ==========================================================================
 * Batched heterogeneous rendering: many grids (of one density format),
 * cameras, media and images rendered by one persistent launch, captured in a
 * CUDA graph.  Not in the paper: a property of the library.
 * ========================================================================== */
typedef struct {
  const tg_grid* grid;
  tg_camera cam;
  tg_medium med;
  int32_t spp;                /* >= 1 */
  int32_t sample_offset;
  uint64_t seed;
  float* accum_sum;           /* device float[H][W], += */
  float* accum_sumsq;         /* device float[H][W] or NULL, += */
} tg_job;
typedef struct tg_batch tg_batch;

/*
 * tg_batch_create - plan a batch of njobs (1..256) jobs.  Every path of every
 * job is one work item of a single persistent launch: a warp lane's new path id
 * selects its job, and the walker, camera, medium, random numbers (key: the
 * job's seed and pixel, as tet_render) and image follow the job, so each image
 * receives exactly what tet_render of its job would add.  With autotune != 0 the
 * launch knobs -- idle lanes before a warp refills (4, 8, 16), waiting lanes
 * before it handles events (8, 12, 16), resident blocks per SM (all, one less)
 * and the job order (as given, or costliest first by paths x cells^(1/3)) -- are
 * chosen on this batch by one pass of coordinate descent (each knob in turn
 * takes the value whose timed launch, rendered into a scratch image, is
 * fastest); otherwise 8, 12, all, as given.  The launch (counter resets
 * and kernel) is then captured in a CUDA graph.  The grids and images must stay
 * valid while the batch exists.  Synchronous.  TG_EINVAL for bad jobs or mixed
 * density formats.
 */
int tg_batch_create(const tg_job* jobs, int32_t njobs, int32_t autotune, void* cuda_stream, tg_batch** out);
/* tg_batch_render - one frame of every job: a single CUDA-graph launch on the stream. */
int tg_batch_render(tg_batch* b, void* cuda_stream);
/* tg_batch_info - knobs[4] = regen, events, blocks per SM (0 = all), order; job_ms[njobs] (host) = time
 * from the first block's start to the end of each job's last path in the latest render (synchronous). */
int tg_batch_info(const tg_batch* b, int32_t* knobs, double* job_ms);
void tg_batch_free(tg_batch* b);

/* ==========================================================================
 * Learned radiance cache.  A small MLP R(x, d) ends paths after one or two
 * collisions: it stands for the radiance that the rest of a path brings back,
 * is trained online on the tracer's own path vertices, and the plain tracer
 * (tet_render) stays the unbiased reference.  Not in the paper; it follows the
 * neural radiance caching idea (Mueller et al., SIGGRAPH 2021) on this grid.
 *
 * Network (fp32 master parameters, one flat device float[RC_NUM_PARAMS]):
 *   e(x, d): 128 features -- x (3), d (3), sin and cos of 2^l pi x_a for l < 12,
 *            sin and cos of 2^l pi d_a for l < 4, zeros; in that order, each
 *            sin directly before its cos, axis-major
 *   h1 = relu(W1 e + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3), R = w4 . h3 + b4
 *   layout: W1[64][128], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4
 * The three matrix products run on the tensor cores with BF16 operands (e, h1,
 * h2 and the weights rounded to nearest even) and FP32 accumulation; biases,
 * h3, the output layer and all bias gradients stay FP32.
 *
 * Records (device float[n][8], 32 bytes each):
 *   query / cached path: x (3), beta, d (3), L
 *   training sample:      x (3), target, d (3), valid
 * x is the grid-space position divided by the domain extent (in [0,1]^3), d the
 * unit direction the path arrived with, beta the path throughput after the
 * albedo at x, L the estimate gathered before the cache takes over.
 * ========================================================================== */
#define RC_NUM_PARAMS 16641

/*
 * tg_random_paths - n training paths: pixel i uniform over the W x H image,
 * drawn as floor(u * W * H) from word 0 of Philox4x32-10 with key (seed lo,
 * seed hi) and counter (i lo, i hi, 0x52434143, 0); sample[i] = sample_base + i.
 * px, py, sample: device int32[n].  Asynchronous.  TG_EINVAL on bad sizes.
 */
int tg_random_paths(uint64_t seed, int64_t n, int32_t width, int32_t height, int32_t sample_base, int32_t* px,
                    int32_t* py, int32_t* sample, void* cuda_stream);

/*
 * tet_cache_samples - training samples from full paths: the n listed paths run
 * to their end as in tet_trace_paths; the first max_vertices (<= 64) collisions
 * of path i, after their next-event estimate, become samples
 * samples[i][j] = (x, target, d, valid) with target = (L_final - L_j) / beta_j,
 * the rest of the path's estimate per unit throughput (L_j: the estimate after
 * vertex j's NEE); slots past the path's last collision are all zero.
 * samples: device float[n][max_vertices][8]; L: device float[n] or NULL.
 * survive in (0, 1): Russian roulette once a path has recorded its max_vertices
 * samples -- before each further scattering the path goes on with probability
 * survive (the draw after collision b is slot b of Philox stream 0x10000, counter
 * (sample, b / 4, 0x10000, 0)) and its throughput is divided by survive, so every
 * target keeps its expectation while the paths end sooner; 0 or 1: no roulette.
 * roulette_from >= 0: the roulette is played only after collisions b >= roulette_from
 * (0-based), so only paths longer than that are cut; 0: after every collision
 * past the last sample.
 * Asynchronous; each call takes its own scratch on its stream.
 * TG_EINVAL for survive outside [0, 1] or a negative roulette_from.
 */
int tet_cache_samples(const tg_grid* g, const tg_camera* cam, const tg_medium* med, uint64_t seed, int64_t n,
                      const int32_t* px, const int32_t* py, const int32_t* sample, int32_t max_vertices,
                      float* samples, float* L, float survive, int32_t roulette_from, void* cuda_stream);

/*
 * tet_cache_queries - the cached estimator's paths for n listed paths: a path
 * ends into the cache at its cache_depth-th collision (>= 1), after that
 * collision's NEE, unless it escaped or was truncated before.
 * rec[i] = (x, beta, d, L): beta = 0 (and x = d = 0) for a path that did not
 * reach the cache; its estimate is then L.  rec: device float[n][8].
 * The cached estimate of path i is L + beta * max(R(x, d), 0).  Asynchronous.
 */
int tet_cache_queries(const tg_grid* g, const tg_camera* cam, const tg_medium* med, uint64_t seed, int64_t n,
                      const int32_t* px, const int32_t* py, const int32_t* sample, int32_t cache_depth,
                      float* rec, void* cuda_stream);

/*
 * rc_mlp_infer - R(x, d) for n records (queries or samples; only x and d are
 * read): y: device float[n].  params: device float[RC_NUM_PARAMS].
 * One fused kernel (encoding, three tensor-core layers, output) over tiles of
 * 128 records.  Asynchronous.  If a tensor-core completion wait ever runs out
 * (it should not), the affected rows are NaN and rc_timeouts() counts it.
 */
int rc_mlp_infer(const float* params, const float* rec, int64_t n, float* y, void* cuda_stream);

/*
 * rc_mlp_grad - the L2 loss sum_i valid_i (R(x_i, d_i) - target_i)^2 over n
 * training samples and its gradient: grad (device float[RC_NUM_PARAMS]) += the
 * gradient of that sum (not divided by the count); loss (device float[3]):
 * loss[0] += the sum, loss[1] += sum_i valid_i.  One fused forward + backward
 * kernel; weight gradients accumulate in tensor memory across a block's tiles
 * and each block adds its sums into grad with 16-byte atomics, so grad must be
 * 16-byte aligned (TG_EINVAL otherwise).  Asynchronous.
 */
int rc_mlp_grad(const float* params, const float* samples, int64_t n, float* grad, float* loss, void* cuda_stream);

/*
 * rc_adam - one Adam step (Kingma & Ba 2015) on the mean gradient
 * grad / max(loss[1], 1), step counted from 1; m and v (device
 * float[RC_NUM_PARAMS]) are the moment estimates.  Afterwards grad, loss[0] and
 * loss[1] are zero and loss[2] = loss[0] / max(loss[1], 1) of the step.
 * Asynchronous.  TG_EINVAL for step < 1 or a bad hyper-parameter.
 */
int rc_adam(float* params, float* m, float* v, float* grad, float* loss, int32_t step, float lr, float beta1,
            float beta2, float eps, void* cuda_stream);

/*
 * tet_render_cached - a frame of the cached estimator: as tet_render (same
 * pixels, samples, random numbers and accumulation), but every path that
 * reaches its cache_depth-th collision ends there into the cache:
 * L + beta * max(R(x, d), 0) per path.  Three launches: the tracer writing one
 * record per path (32 bytes x W x H x spp, this call's own scratch from the
 * library's stream-ordered pool, given back on the stream after the last
 * launch), the fused MLP completing the records, and a per-pixel sum in sample
 * order.  Asynchronous; calls on different streams may overlap.
 */
int tet_render_cached(const tg_grid* g, const tg_camera* cam, const tg_medium* med, int32_t spp, uint64_t seed,
                      int32_t sample_offset, int32_t cache_depth, const float* params, float* accum_sum,
                      float* accum_sumsq, tg_stats* stats, void* cuda_stream);

/* rc_timeouts - number of tensor-core completion waits that ran out since the
 * library was loaded (0 in a healthy run).  Synchronises the device. */
int rc_timeouts(int64_t* count);

/* tg_error_string - a static, human-readable name for a status code (TG_OK and
 * the TG_E* codes; "unknown status" otherwise).  The paper has no counterpart.
 * Never fails; needs no GPU. */
const char* tg_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif
