/*
 * CPU oracle of the adaptive tetrahedral-grid volumetric path tracer
 * (Benyoub & Dupuy, "Adaptive Tetrahedral Grids for Volumetric Path-Tracing",
 * SIGGRAPH Talks 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; it is plain, slow and meant
 * to be checked against the paper by eye.  Floating point is fp64 and the
 * translation unit is compiled with -ffp-contract=off.
 *
 * All pointers are host pointers.  Every function returns 0 on success or a
 * negative status: -1 invalid argument, -2 out of memory, -4 walk step limit,
 * -5 build round limit, -6 inconsistent grid (non-conforming mesh).
 */
#ifndef TETVOL_ORACLE_H
#define TETVOL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float pos[3], target[3], up[3]; float fov_y_deg; int32_t width, height; } orc_camera;
typedef struct {
  float albedo, g, sigma_scale;    /* sigma_scale: extinction per world unit at density 1 */
  int32_t max_bounces;             /* maximum number of collisions of a path            */
  float sun_dir[3];                /* direction the sunlight travels (unit)              */
  float sun_irradiance, env_radiance;
} orc_medium;

typedef struct orc_grid orc_grid;

/* Sec. 2: LEB construction of the adaptive conforming grid from a dense volume
 * density[nz][ny][nx] (values in [0,1]).  cam may be NULL (camera criterion off);
 * footprint_px <= 0 also switches the camera criterion off; theta < 0 switches
 * the density-variation criterion off.  density_format: 0 fp32, 1 bf16, 2 fp16. */
int orc_build(const float* density, int32_t nx, int32_t ny, int32_t nz,
              const float box_min[3], float voxel_size, const orc_camera* cam,
              float footprint_px, float theta, int32_t max_depth, int32_t density_format,
              int32_t max_rounds, int32_t nthreads, orc_grid** out);
void orc_grid_free(orc_grid* g);
int orc_grid_info(const orc_grid* g, int64_t* num_tets, int32_t* max_depth_reached,
                  int32_t* K, int32_t* rounds, int32_t* cubes /*[3]*/, int32_t* voxels_per_cube);
/* codes u64[N]; verts int32[N][4][3] in units of 2^-K cube (LEB vertex order);
 * tag int32[N]; nbr int32[N][4] (-1 on the domain boundary); nid uint8[N][4]
 * in [0,18); plane float[N][4]; density float[N] (value after storage rounding);
 * majorant float[N] (max density of D); count u32, sum u64, qmin/qmax u32 [N].
 * Any output pointer may be NULL. */
int orc_grid_export(const orc_grid* g, uint64_t* codes, int32_t* verts, int32_t* tag,
                    int32_t* nbr, uint8_t* nid, float* plane, float* density, float* majorant,
                    uint32_t* count, uint64_t* sum, uint32_t* qmin, uint32_t* qmax);

/* Sec. 3, Algorithm 1 (+ sun next-event estimation): per-path estimates.
 * flags bit0 degenerate (near tie somewhere), bit1 truncated at max_bounces,
 * bit2 camera ray missed the grid, bit3 walk step limit.
 * seq: visited cell sequence (all segments, -1 between segments) truncated to seq_cap. */
int orc_render_paths(const orc_grid* g, const orc_camera* cam, const orc_medium* med, uint64_t seed,
                     int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                     double* L, int32_t* flags, int32_t* collisions, int64_t* steps,
                     int32_t* seq, int32_t seq_cap, int32_t* seq_len, int32_t nthreads);
/* The learned radiance cache's two uses of the tracer (8 doubles per record):
 *  cache_depth > 0: the path ends into the cache at its cache_depth-th collision,
 *    after that collision's next-event estimate; query[i] = x (3, grid space over
 *    the domain extent), beta (throughput after the albedo there; 0 when the path
 *    ended before), d (3, arrival direction), L (estimate so far).
 *  max_vertices > 0: training samples from the path's first max_vertices
 *    collisions (the path itself runs to its end when cache_depth = 0):
 *    vertices[i][j] = x (3), target = (L_final - L after the vertex's NEE) / beta_j,
 *    d (3), valid (1, or 0 with all zeros past the path's last vertex).
 *  L[i], flags[i]: the path's own estimate and flags (NULL allowed; flags bit5:
 *    ended by the roulette below).
 *  survive in (0, 1): once a path has recorded its max_vertices vertices, Russian
 *    roulette before every further scattering -- the path goes on with probability
 *    survive (the draw after collision b is slot b of Philox stream 0x10000) and its
 *    throughput is divided by survive; 0 or 1: no roulette.
 *  roulette_from >= 0: the roulette is played only after collisions b >= roulette_from
 *    (0-based); 0: after every collision past the last vertex. */
int orc_cache_paths(const orc_grid* g, const orc_camera* cam, const orc_medium* med, uint64_t seed,
                    int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                    int32_t cache_depth, double* query, int32_t max_vertices, double* vertices,
                    double* L, int32_t* flags, float survive, int32_t roulette_from, int32_t nthreads);
int orc_render(const orc_grid* g, const orc_camera* cam, const orc_medium* med, int32_t spp,
               uint64_t seed, int32_t sample_offset, double* sum, double* sumsq, int64_t* steps,
               int32_t nthreads);

/* Extra per-tet channels (Sec. 3): the mean over D (like the density) of a
 * temperature, an albedo and an anisotropy volume (g = 2a - 1, clamped to
 * +-0.99), each quantised like the density (NULL: channel absent), and the voxel
 * majorant (max q + 1) / 2^24 over the voxels touching the tet's bounding box. */
int orc_grid_channels(orc_grid* g, const float* density, const float* temperature, const float* albedo,
                      const float* aniso, int32_t nthreads);
/* chan float[N][3] (temperature, albedo, g), vmaj float[N]; either may be NULL. */
int orc_grid_export_channels(const orc_grid* g, float* chan, float* vmaj);

/* The extended estimator: flags 1 emission (collision estimator, Le =
 * emission_scale * temperature), 2 per-tet albedo, 4 per-tet g, 8 voxel medium
 * (density = the voxel holding x, from `density` [nz][ny][nx]) tracked against
 * the tet majorants: delta tracking for free flights (acceptance decided in fp32
 * as u * majorant < rho), ratio tracking for shadow rays; the k-th such draw of
 * the free flight (shadow ray) of bounce b is slot k of Philox stream 1 + 2b
 * (2 + 2b): counter (sample, k / 4, stream, 0). */
typedef struct { int32_t flags; float emission_scale; const float* density; } orc_ext;
int orc_render_ext_paths(const orc_grid* g, const orc_camera* cam, const orc_medium* med, const orc_ext* ext,
                         uint64_t seed, int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                         double* L, int32_t* flags, int32_t* collisions, int64_t* steps, int32_t nthreads);

/* The regular-grid comparator: same estimator on the voxel grid (3D DDA). */
int orc_dda_paths(const float* density, int32_t nx, int32_t ny, int32_t nz, const float box_min[3],
                  float voxel_size, const orc_camera* cam, const orc_medium* med, uint64_t seed,
                  int64_t n, const int32_t* px, const int32_t* py, const int32_t* sample,
                  double* L, int32_t* flags, int32_t* collisions, int64_t* steps, int32_t nthreads);
int orc_dda_render(const float* density, int32_t nx, int32_t ny, int32_t nz, const float box_min[3],
                   float voxel_size, const orc_camera* cam, const orc_medium* med, int32_t spp,
                   uint64_t seed, int32_t sample_offset, double* sum, double* sumsq, int64_t* steps,
                   int32_t nthreads);

/* Walk only: optical depth sigma * sum(rho_T * chord_T) along rays given in grid
 * space (unit cube = 1), from where they enter the domain to where they leave. */
int orc_optical_depth(const orc_grid* g, int64_t n, const double* origin, const double* dir,
                      double sigma, double* tau, int64_t* steps, int32_t* max_faces_tested,
                      int32_t* flags, int32_t* seq, int32_t seq_cap, int32_t* seq_len);

/* Descent profile of points (grid space) through the LEB hierarchy, independent
 * of any built grid: for every depth 0..max_depth the node code, its statistics
 * (count, sum, qmin, qmax), its stored density and whether the criterion splits it.
 * Arrays are [n][max_depth+1]. */
int orc_path_profile(const float* density, int32_t nx, int32_t ny, int32_t nz, const float box_min[3],
                     float voxel_size, const orc_camera* cam, float footprint_px, float theta,
                     int32_t max_depth, int32_t density_format, int64_t n, const double* points,
                     uint64_t* codes, uint32_t* count, uint64_t* sum, uint32_t* qmin, uint32_t* qmax,
                     float* density_out, uint8_t* split, int32_t nthreads);

/* Primitives exposed for pinning. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint64_t seed, uint32_t pixel, uint32_t sample, uint32_t slot);
void orc_hg_sample(double g, double u1, double u2, const double dir_in[3], double dir_out[3]);
double orc_hg_pdf(double g, double cos_theta);
int orc_locate(const orc_grid* g, int64_t n, const double* points, int32_t* leaf);

#ifdef __cplusplus
}
#endif
#endif
