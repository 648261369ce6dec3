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
 *   density  device float[nz][ny][nx]; read during the call only.
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

/* Size and shape of a grid.  Any output pointer may be NULL.  bytes: device bytes
 * the renderer reads (records + codes); K: vertex coordinate scale exponent. */
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

void tg_grid_free(tg_grid* g);

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
 * Asynchronous.  Errors: TG_EINVAL, TG_ECUDA.  A walk that exceeds its step
 * limit ends its path and is counted in stats->step_limit.
 * Calls that overlap on the same grid share its scratch counter: serialise them.
 */
int tet_render(const tg_grid* g, const tg_camera* cam, const tg_medium* med, int32_t spp, uint64_t seed,
               int32_t sample_offset, float* accum_sum, float* accum_sumsq, tg_stats* stats,
               void* cuda_stream);

/*
 * grid_render - the regular-grid comparator (the "1024^3 regular grid" reference
 * of Sec. 4): the same estimator as tet_render, walking the voxels of the dense
 * volume with a 3D DDA instead of the tetrahedra.  Same arguments and semantics.
 * Uses a library-owned scratch counter per device: serialise overlapping calls.
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

const char* tg_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif
