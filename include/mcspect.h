/*
 * mcspect.h -- C ABI of the GB300 Monte Carlo SPECT library (libmcspect.so).
 *
 * The library estimates the SPECT system matrix of the inverse Monte Carlo
 * model, Eq. (IMC) of Sec. 5.1,
 *     P_j = sum_i T_ij S_i,
 * by analog photon transport on the GPU, and reconstructs the source S with
 * the ML-EM update of Eq. (MLEM), Sec. 5.1.  Matrix rows j are detector bins
 * (view-major, then axial bin, then transaxial bin); columns i (called v
 * below) are voxels (x fastest).
 *
 * Conventions for every entry point:
 *   - returns MC_OK (0) or a negative MC_E* code; no exception crosses the
 *     ABI; mc_last_error() gives a message for the calling thread;
 *   - "_host" pointers are host memory, "_dev" pointers are device memory of
 *     the current CUDA device; the caller owns and frees every buffer it
 *     passes; an mc_system is owned by the library until mc_system_free;
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Entry
 *     points that take device buffers only enqueue work on `stream` and
 *     return without waiting unless stated otherwise;
 *   - an mc_system is not thread-safe: calls on one system must not overlap
 *     on the GPU (they share the system's work vectors).
 */
#ifndef MCSPECT_H
#define MCSPECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* exported from libmcspect.so */
#if defined(__GNUC__)
#define MC_API __attribute__((visibility("default")))
#else
#define MC_API
#endif

#define MC_OK 0
#define MC_EINVAL (-1)   /* bad argument (null pointer, size, range) */
#define MC_ENOMEM (-2)   /* device or host allocation failed */
#define MC_ECUDA (-3)    /* a CUDA call or kernel launch failed */

/* transport precision */
#define MC_FP32 0 /* production: float arithmetic, 23-bit uniforms */
#define MC_FP64 1 /* verification: double arithmetic, 32-bit uniforms */

/* what the transport tallies */
#define MC_TALLY_ALL 0
#define MC_TALLY_PRIMARY 1
/* Flag, or-ed with either of the above: forced detection (the paper's
 * variance-reduction section, "forced detection").  Instead of detecting
 * the photon where it escapes, a weighted copy is forced to every view at
 * each interaction location -- the emission point and every real
 * collision (with MC_TALLY_PRIMARY: the emission point only).  The copy's
 * direction is uniform in the collimator's acceptance cone about the view's
 * normal, drawn from its own Philox block (counter (k, 1 + n, h_lo, h_hi)
 * for view k and interaction n of history h); its weight is the
 * probability of not being absorbed at the collision (1 - mu_pe/mu; 1 at
 * emission) times the angular probability of that direction (Omega/(4 pi)
 * at emission, Omega times the Klein-Nishina density per steradian at a
 * collision, 0 below the window) times the collimator's open fraction f(x)
 * times the exact transmission along the ray to the grid boundary; it is
 * binned like an analog detection.  Weights are tallied in fixed point,
 * q = rint(w 2^48), and summed as integers, so a build's matrix does not
 * depend on event order.  The result is a weighted system (entries are
 * weight sums, float values only); builds are limited to < 2^32 weighted
 * events (about 2.4e7 histories at 120 views). */
#define MC_TALLY_FORCED 2
/* Flag, with MC_TALLY_PRIMARY only: forced direction (same section of the
 * paper).  The emission direction is drawn from the band |d_z| < sin(psi),
 * tan(psi) = hole_diam/hole_len -- the directions from which some view's
 * collimator can be reached -- with cos(theta) uniform in the band (the
 * same draws, scaled), and every detection carries the band's share of the
 * sphere, w = sin(psi).  Exact for unscattered photons (an unscattered
 * photon outside the band is never detected); scattered photons from
 * emissions outside the band would be missed, hence primary-only.  The
 * result is a weighted system. */
#define MC_TALLY_FORCED_DIRECTION 4

/* storage type of matrix values used by the projectors */
#define MC_VAL_F32 0
#define MC_VAL_F16 1
#define MC_VAL_BF16 2
/* the conventional reduced-precision storage, kept for comparison: the
 * entries A_jv = C_jv / n_v themselves rounded to half / bfloat16 (half
 * loses precision below 6.1e-5, where A becomes subnormal) */
#define MC_VAL_F16_A 3
#define MC_VAL_BF16_A 4

/* history fates */
#define MC_FATE_ABSORBED 0
#define MC_FATE_BELOW_WINDOW 1
#define MC_FATE_ESCAPE 2
#define MC_FATE_CAP 3

/* Voxelised attenuation map (Sec. 3: patient size, shape, composition).
 * Grid centred on the origin; voxel (i,j,k) covers
 * [i h - nx h/2, (i+1) h - nx h/2) x ... ; material index per voxel into a
 * table of at most 256 materials.  mu(m,E) = 0.1 rho_m (N_A (Z/A)_m
 * sigma_KN(E) + photo_k Z_eff,m^4 / E^3) per mm, E in keV. */
typedef struct mc_phantom {
  int32_t nx, ny, nz;
  double voxel_mm;
  const uint8_t *material_host; /* nz*ny*nx, x fastest */
  int32_t n_materials;          /* 1..256 */
  const double *rho_host;       /* g/cm^3, [n_materials] */
  const double *z_over_a_host;  /* [n_materials] */
  const double *z_eff_host;     /* [n_materials] */
} mc_phantom;

/* Acquisition (Sec. 3): one parallel-hole collimated head per view; view k
 * at angle theta_k = (start_deg + k (arc_deg / n_views)) degrees, outward
 * normal (cos, sin, 0), transaxial axis (-sin, cos, 0), axial axis z.  The
 * collimator front face is at radius_mm from the axis (it must clear the
 * grid), the crystal at radius_mm + hole_len_mm.  Detection window
 * [(1 - window_frac/2) e0_kev, (1 + window_frac/2) e0_kev]. */
typedef struct mc_geometry {
  int32_t n_views;
  double start_deg, arc_deg;
  int32_t n_bins_u, n_bins_v; /* transaxial, axial */
  double bin_mm;
  double radius_mm;
  double hole_len_mm, hole_diam_mm;
  double fwhm_mm; /* Gaussian intrinsic blur */
  double e0_kev, window_frac;
  double photo_k;
  int32_t precision; /* MC_FP32 or MC_FP64 */
  int32_t tally;     /* MC_TALLY_ALL, or MC_TALLY_PRIMARY: only photons that
                        reach the camera unscattered (the attenuation + blur
                        matrix of dual-matrix OS, Sec. 5.3); either may be
                        or-ed with MC_TALLY_FORCED */
} mc_geometry;

typedef struct mc_system mc_system; /* opaque, device resident */

typedef struct mc_system_info {
  int64_t n_rows;        /* M = n_views * n_bins_v * n_bins_u */
  int64_t n_cols;        /* N = voxels */
  int64_t nnz;           /* distinct (row, col) pairs with a count */
  int64_t n_events;      /* detections tallied */
  uint64_t first_history, n_histories;
  uint64_t fates[4];     /* ABSORBED, BELOW_WINDOW, ESCAPE, CAP */
  uint32_t max_count;    /* largest C_jv */
  int32_t value_type;    /* MC_VAL_* used by the projectors */
  double build_ms_transport; /* device time of the build's transport kernel */
  double build_ms_assembly;  /* ... of matrix assembly (sort, CSR/CSC, sums) */
  double build_ms_detect;    /* ... of the collimator/detector kernel */
  int32_t spmv_fwd, spmv_bwd; /* projector kernels: 0 = streaming layout,
                                 else lanes per row (column) group */
  int32_t weighted;           /* 1: entries are summed forced-detection
                                 weights (counts = weighted events per entry) */
  int32_t pad;
} mc_system_info;

/* Per-history trace (verification): 48 bytes, this exact layout. */
typedef struct mc_history_record {
  uint8_t fate, n_events; /* n_events saturates at 255 */
  uint16_t pad;
  uint32_t n_virtual, n_real, n_compton, n_draws;
  uint32_t pad2;
  double e_final_kev;
  int32_t event_row[4]; /* first four detections' rows */
} mc_history_record;

/* Transport + tally (Sec. 2; Sec. 5.1, T_ij estimated by Monte Carlo).
 * Runs histories 0 .. n_histories-1 of the stream keyed by `seed`; history h
 * starts in voxel h mod N.  The result holds C_jv (integer counts), n_v
 * (histories started in voxel v) and the matrix A = C diag(1/n_v) used by
 * the projectors, in CSR and CSC form.  Host inputs are copied; the call
 * returns after the matrix is built (it synchronises `stream`).
 * Errors: MC_EINVAL (bad sizes, front face inside the grid, n_histories 0),
 * MC_ENOMEM, MC_ECUDA. */
MC_API int mc_build_system(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t n_histories,
                    uint64_t seed, void *stream, mc_system **out);

/* A phantom + geometry made resident on the device (map, view table,
 * attenuation coefficients), for repeated builds without host traffic.
 * Host inputs are copied; the call synchronises `stream`.
 * Errors: as mc_build_system. */
typedef struct mc_plan mc_plan;
MC_API int mc_plan_create(const mc_phantom *phantom, const mc_geometry *geometry, void *stream, mc_plan **out);

/* Transport + tally of histories first .. first+count-1 from a plan; same
 * result as mc_build_system_range with the plan's inputs. */
MC_API int mc_plan_build(mc_plan *plan, uint64_t first, uint64_t count, uint64_t seed, void *stream,
                         mc_system **out);

/* Release a plan (NULL is accepted). */
MC_API int mc_plan_free(mc_plan *plan);

/* The tally of a history range without assembly (Sec. 2 transport, the
 * detections that estimate T_ij of Eq. (IMC), Sec. 5.1): the events of
 * histories first .. first+count-1 of the plan, one key v * M + j per
 * detection (row j, voxel v, M = the plan's rows), in no fixed order, into
 * the caller's device buffer keys_dev[capacity].  *n_events_out receives
 * the number of events and fates_host[4] (nullable) the history fates.  The
 * tally is deterministic: if it does not fit (MC_EINVAL, *n_events_out set)
 * repeat the call with a larger buffer.  MC_EINVAL for weighted plans
 * (forced detection or forced direction).  Synchronises `stream`. */
MC_API int mc_plan_tally(mc_plan *plan, uint64_t first, uint64_t count, uint64_t seed, uint64_t *keys_dev,
                         int64_t capacity, int64_t *n_events_out, uint64_t *fates_host, void *stream);

/* Routing of tally events to the parts of a view-partitioned system (the
 * split of one reconstruction over several GPUs; the back-projection sum of
 * Eq. (MLEM) runs over detector bins, so bins split by views).  The
 * n_rows / rows_per_view views are cut into n_parts contiguous blocks, part
 * p holding views [p V / n_parts, (p + 1) V / n_parts) (integer division).
 * keys_dev[n_events] (v * n_rows + j) are written to out_dev[n_events]
 * grouped by part (part 0 first; no fixed order inside a part), each key
 * renumbered to its part's rows: v * M_p + (j - first row of part p), M_p =
 * the part's views x rows_per_view.  part_counts_host[n_parts] receives the
 * events per part.  MC_EINVAL if n_rows is not a multiple of rows_per_view
 * or n_parts is not in 1 .. min(views, 1024).  Synchronises `stream`. */
MC_API int mc_events_route(const uint64_t *keys_dev, int64_t n_events, int64_t n_rows, int64_t rows_per_view,
                           int32_t n_parts, uint64_t *out_dev, int64_t *part_counts_host, void *stream);

/* Matrix from device event keys v * n_rows + j (duplicates add), e.g. the
 * routed events of one part; n_v is that of the history range [first,
 * first+count).  The caller's keys are not modified.  MC_EINVAL for a key
 * >= n_rows * n_cols.  Synchronises `stream`. */
MC_API int mc_system_from_keys(int64_t n_rows, int64_t n_cols, const uint64_t *keys_dev, int64_t n_keys,
                               uint64_t first, uint64_t count, void *stream, mc_system **out);

/* As mc_build_system for histories first .. first+count-1 only (chunked or
 * resumed runs): the counts and n_v of disjoint ranges add up exactly to
 * those of their union. */
MC_API int mc_build_system_range(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t first,
                          uint64_t count, uint64_t seed, void *stream, mc_system **out);

/* Matrix from an explicit event list (row j, column v), e.g. tallies made
 * elsewhere; n_v is that of the history range [first, first+count).
 * Duplicates add.  Errors: MC_EINVAL for an index out of range. */
MC_API int mc_system_from_events(int64_t n_rows, int64_t n_cols, const int32_t *rows_host, const int32_t *cols_host,
                          int64_t n_events, uint64_t first, uint64_t count, void *stream, mc_system **out);

/* Weighted matrix from an explicit list of forced-detection events (row j,
 * column v, fixed-point weight q = rint(w 2^48)), e.g. tallies made
 * elsewhere (paper's variance-reduction section, forced detection; see
 * MC_TALLY_FORCED).  Weights of equal (j, v) add as exact integers; n_v is
 * that of the history range [first, first+count).  The system is weighted:
 * float values only, no ordered subsets.  Errors: MC_EINVAL for an index out
 * of range or >= 2^32 events. */
MC_API int mc_system_from_weighted_events(int64_t n_rows, int64_t n_cols, const int32_t *rows_host,
                                          const int32_t *cols_host, const uint64_t *weights_host, int64_t n_events,
                                          uint64_t first, uint64_t count, void *stream, mc_system **out);

/* The entries of the tally matrix as doubles, in the CSC and CSR orders of
 * the exports below (either pointer may be NULL): the counts C_jv, or for a
 * weighted system the weight sums q * 2^-48 (exact).  nnz values each.
 * Synchronises `stream`. */
MC_API int mc_system_export_values(const mc_system *sys, double *csc_values_host, double *csr_values_host,
                                   void *stream);

/* Release a system and its device memory (NULL is accepted). */
MC_API int mc_system_free(mc_system *sys);

MC_API int mc_system_info_get(const mc_system *sys, mc_system_info *info);

/* Copy the count matrix to the host in CSC form: col_ptr[n_cols+1],
 * row_idx[nnz] (ascending within a column), counts[nnz]; n_v[n_cols].
 * Any pointer may be NULL to skip that array.  Synchronises `stream`. */
MC_API int mc_system_export_csc(const mc_system *sys, int64_t *col_ptr_host, int32_t *row_idx_host, uint32_t *counts_host,
                         uint32_t *n_v_host, void *stream);

/* Same in CSR form: row_ptr[n_rows+1], col_idx[nnz] ascending within a row. */
MC_API int mc_system_export_csr(const mc_system *sys, int64_t *row_ptr_host, int32_t *col_idx_host, uint32_t *counts_host,
                         void *stream);

/* Storage type of the values the projectors read (the matrix of Eq. (IMC),
 * Sec. 5.1; accumulation stays FP32 in every type).  MC_VAL_F32 (default),
 * MC_VAL_F16 and MC_VAL_BF16 store the integer counts C_jv -- exact up to
 * 2^24, 2048 and 256 -- and fold 1/n_v into the image; MC_EINVAL if a count
 * is not exact in the requested type unless allow_rounding is non-zero, in
 * which case the counts are rounded and ML-EM normalises with the rounded
 * counts' column sums (it runs on the matrix the projectors read).
 * MC_VAL_F16_A / MC_VAL_BF16_A store round(C_jv / n_v) and reconstruct with
 * that rounded matrix (its own column sums as the sensitivity); they are
 * always rounded.  Weighted systems keep MC_VAL_F32.  The FP64 projectors
 * (mc_project_f64, mc_backproject_f64) always use the exact matrix. */
MC_API int mc_system_set_value_type(mc_system *sys, int32_t value_type, int32_t allow_rounding);

/* Projector kernels of a system: fwd (forward projection, CSR) and bwd
 * (back-projection, CSC) each 0 = streaming layout (entries of runs of whole
 * rows staged in shared memory, then one fixed-order sum per row: warps of
 * 32 R rows, R = 1, 2 or 4 rows per lane, when rows average fewer than 16
 * entries, else one warp per row in tiles of ~4096 entries), 1, 2, 4, 8,
 * 16 or 32 = that many lanes per row (column), or -1 = keep.  Every layout
 * gives the same sums up to FP32 rounding order.  The streaming layout needs
 * every row (column) shorter than 2048 entries: MC_EINVAL otherwise (the
 * system is left unchanged).  Synchronises `stream`. */
MC_API int mc_system_set_spmv_layout(mc_system *sys, int32_t fwd, int32_t bwd, void *stream);

/* Forward projection q = A x (Eq. (IMC)): x_dev[N], q_dev[M], float. */
MC_API int mc_project(const mc_system *sys, const float *x_dev, float *q_dev, void *stream);

/* Ratio of Eq. (MLEM): r_j = y_j / (A x)_j, 0 where (A x)_j = 0:
 * x_dev[N], y_dev[M], r_dev[M], float.  Uses the system's work vector, like
 * the other projector calls on one system. */
MC_API int mc_project_ratio(const mc_system *sys, const float *x_dev, const float *y_dev, float *r_dev, void *stream);

/* Poisson log-likelihood of Sec. 5.1 (up to a constant) of an image:
 * *value_dev = sum_j y_j ln q_j - q_j, q = A x, bins with y_j = 0 adding
 * -q_j, and bins whose row of A is empty left out of the y_j ln q_j sum
 * (q_j = 0 for every image there; ML-EM ignores them the same way);
 * FP64 accumulation.  x_dev[N], y_dev[M] float; value_dev one double. */
MC_API int mc_loglik(const mc_system *sys, const float *x_dev, const float *y_dev, double *value_dev, void *stream);

/* Back-projection b = A^T r: r_dev[M], b_dev[N], float. */
MC_API int mc_backproject(const mc_system *sys, const float *r_dev, float *b_dev, void *stream);

/* Sensitivity s_v = sum_j A_jv (the normaliser of Eq. (MLEM)), FP64:
 * s_dev[N] double. */
MC_API int mc_sensitivity(const mc_system *sys, double *s_dev, void *stream);

/* Uniform start image: x_v = sum(y) / sum(s) where s_v > 0, else 0. */
MC_API int mc_mlem_init(mc_system *sys, const float *y_dev, float *x_dev, void *stream);

/* Pieces of ML-EM over a system split into parts (each part holding some
 * detector rows, Eq. (MLEM) summing over them): the FP64 sum of a float
 * vector (*out_dev = sum of v_dev[n], fixed order), and the uniform start
 * image from a sensitivity summed over the parts: x_v = sum_y / sum(sens)
 * where sens_v > 0, else 0 (sens_dev[n] double, x_dev[n] float).  The
 * update x_v <- x_v b_v / s_v from a back-projection summed over the parts
 * is mc_pgd_step with alpha = 1 and no prior. */
MC_API int mc_vector_sum(int64_t n, const float *v_dev, double *out_dev, void *stream);
MC_API int mc_mlem_start(int64_t n, const double *sens_dev, double sum_y, float *x_dev, void *stream);

/* n_iter ML-EM updates of Eq. (MLEM), in place on x_dev[N]:
 *   x_v <- x_v / s_v * sum_j A_jv y_j / (A x)_j,
 * with y_j / (A x)_j taken as 0 where (A x)_j = 0 and x_v = 0 where s_v = 0.
 * If loglik_host is not NULL it receives n_iter values
 * L(x^k) = sum_j y_j ln q_j - q_j (FP64; bins with y_j = 0 add -q_j, bins
 * with an empty row are left out of the log term, as in mc_loglik) for the
 * iterates before each update, and the call synchronises `stream`. */
MC_API int mlem_iterate(mc_system *sys, const float *y_dev, float *x_dev, int32_t n_iter, double *loglik_host,
                 void *stream);

/* Ordered subsets (Sec. 5.3, OSEM): the system made of the rows of views
 * subset, subset + n_subsets, subset + 2 n_subsets, ... of a full system
 * whose rows are view-major with rows_per_view rows per view (n_bins_v *
 * n_bins_u for systems built here).  Its row i is parent row
 * (subset + (i / rows_per_view) n_subsets) rows_per_view + i % rows_per_view;
 * columns, n_v and counts are the parent's.  Errors: MC_EINVAL if the parent
 * is itself a subset or the sizes do not fit. */
MC_API int mc_system_subset(const mc_system *parent, int64_t rows_per_view, int32_t n_subsets, int32_t subset,
                            void *stream, mc_system **out);

/* n_iter sweeps of ordered-subset EM (Sec. 5.3) with the dual-matrix
 * update of Eq. (DMOS) and the additive term of Eq. (Sohlberg OSEM), in
 * place on x_dev[N]: for s = 0 .. n_subsets-1,
 *   q = C_s x,  r_i = y_o / (q_i + add_o) (0 if not positive), o the parent
 *   row of subset row i,
 *   x_v <- x_v / sum_i B_s,iv * sum_i B_s,iv r_i   (x_v kept where the sum is
 *   0: the voxel is outside subset s's view)
 * with C_s = fwd[s] (reprojection, e.g. all photons) and B_s = back[s]
 * (back-projection, e.g. MC_TALLY_PRIMARY).  fwd[s] and back[s] must be
 * subset s of n_subsets (n_subsets = 1: full systems) of the same shape.
 * y_dev and add_dev (nullable: no additive term) have the parent's rows.
 * fwd = back with one subset and no additive term is mlem_iterate from a
 * start image that is 0 off the support (as mc_mlem_init gives). */
MC_API int osem_iterate(mc_system *const *fwd, mc_system *const *back, int32_t n_subsets, const float *y_dev,
                        const float *add_dev, float *x_dev, int32_t n_iter, void *stream);

/* Double-precision projectors (same matrix, FP64 accumulation): q = A x and
 * b = A^T r on double device vectors; for derivative checks and FP64
 * reference images. */
MC_API int mc_project_f64(const mc_system *sys, const double *x_dev, double *q_dev, void *stream);
MC_API int mc_backproject_f64(const mc_system *sys, const double *r_dev, double *b_dev, void *stream);

/* Quadratic 6-neighbour smoothness prior on an nx*ny*nz image (x fastest):
 *   R(x) = beta/2 sum over neighbouring voxel pairs (x_v - x_w)^2,
 *   grad_v = beta sum over the 6 (fewer at the border) neighbours (x_v - x_w).
 * grad_dev (N values) and value_dev (one double) may each be NULL.  The
 * paper reconstructs by plain ML-EM (Sec. 5.1); this penalty is an addition
 * for the penalised Poisson likelihood. */
MC_API int mc_prior_quadratic(int32_t nx, int32_t ny, int32_t nz, double beta, const float *x_dev, float *grad_dev,
                              double *value_dev, void *stream);
MC_API int mc_prior_quadratic_f64(int32_t nx, int32_t ny, int32_t nz, double beta, const double *x_dev,
                                  double *grad_dev, double *value_dev, void *stream);

/* One preconditioned projected-gradient step on the penalised negative
 * log-likelihood  sum_j (q_j - y_j ln q_j) + R(x)  (Poisson likelihood of
 * Sec. 5.1), in place on x_dev[n]:
 *   x_v <- max(0, x_v - alpha (x_v / s_v) (s_v - bp_v + gp_v)),
 * with s the sensitivity (mc_sensitivity), bp = A^T (y / A x) and gp the
 * prior gradient (NULL: none); x_v = 0 where s_v = 0.  alpha = 1 without a
 * prior is one ML-EM update (Eq. (MLEM)). */
MC_API int mc_pgd_step(int64_t n, double alpha, const double *sens_dev, const float *bp_dev, const float *gp_dev,
                       float *x_dev, void *stream);

/* SpMV autotuner: times the forward and back-projection kernels of `sys`
 * (streaming layout, row groups of 1..32 lanes) on its own matrix and keeps
 * the fastest of each (reported by mc_system_info_get).  Synchronises. */
MC_API int mc_system_autotune(mc_system *sys, void *stream);

/* Batched ML-EM (serving many acquisitions): n systems with their
 * projections y_dev[k] (rows of system k) and images x_dev[k] (columns of
 * system k), all device memory owned by the caller and kept alive while the
 * batch exists.  mc_batch_mlem sets every image to its uniform start
 * (mc_mlem_init) and runs n_iter updates of Eq. (MLEM) for all of them: one
 * forward and one back-projection launch per iteration over all systems,
 * captured once into a CUDA graph per n_iter and replayed.  Every system
 * must be a full (not ordered-subset) FP32 system, of any projector layout:
 * the batch makes its own work units over each system's non-empty rows and
 * columns (warp chunks; tiles of one warp per row where rows or columns
 * average 16 or more entries, which then must be shorter than 2048 entries,
 * else MC_EINVAL).  Results equal mlem_iterate's up to FP32 rounding order.
 * Systems in a batch must not be used by other calls while it runs. */
typedef struct mc_batch mc_batch;
MC_API int mc_batch_create(mc_system *const *systems, int32_t n, const float *const *y_dev, float *const *x_dev,
                           mc_batch **out);
MC_API int mc_batch_mlem(mc_batch *batch, int32_t n_iter, void *stream);
/* The same reconstruction as mc_batch_mlem (equal images) with all n_iter
 * iterations of all systems in one persistent cooperative launch: the
 * blocks stay resident and meet at a grid-wide barrier between the forward
 * and back-projection halves of every iteration (the start images and the
 * write-back are four short launches around it).  Not captured in a graph.
 * MC_ECUDA if the device cannot launch cooperatively. */
MC_API int mc_batch_mlem_persistent(mc_batch *batch, int32_t n_iter, void *stream);
MC_API int mc_batch_free(mc_batch *batch);

/* ML-EM like mlem_iterate, for callers that must not allocate device
 * memory: a reconstruction service that plans its memory up front (a device
 * allocation or free can synchronise the whole device and stall concurrent
 * work, or fail under a fixed memory cap), or host code whose device memory
 * is owned by another allocator.  mlem_iterate may allocate its
 * log-likelihood buffer on first use; this entry point never calls
 * cudaMalloc, cudaFree or any allocating routine.  The paper has no
 * counterpart: it is a deployment variant of the ML-EM update above.
 *
 * Its work vectors live in one static device array of ~18 MiB that every GPU
 * loading the library keeps until the process exits.  Limits: n_rows and
 * n_cols at most 2^21 each (2,097,152) and at most 4096 log-likelihood
 * values per call; larger requests return MC_EINVAL with a message.  The
 * first call on a device looks up the array's device address (no
 * allocation).  All calls on a device share the array and leave their values
 * in it: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  The current device must be the one the system was built on
 * (MC_EINVAL otherwise: the array is per device).  Results equal
 * mlem_iterate's on the same inputs. */
MC_API int mlem_iterate_noalloc(const mc_system *sys, const float *y_dev, float *x_dev, int32_t n_iter,
                                double *loglik_host, void *stream);

/* Verification: per-history trace records of histories first ..
 * first+count-1 (records written to out_host[count]).  Synchronises. */
MC_API int mc_trace_histories(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t seed, uint64_t first,
                       uint64_t count, mc_history_record *out_host);

/* Verification of the Compton sampler (Sec. 3: a scatter lowers the energy
 * and changes the direction): sample i uses history i's stream; writes
 * cos(theta) and E'/E.  precision MC_FP32 or MC_FP64.  Synchronises. */
MC_API int mc_debug_kn(double e_kev, int32_t precision, uint64_t seed, uint64_t n, double *cos_out_host,
                double *eps_out_host);

/* Verification of Woodcock tracking: n photons of energy e_kev start at
 * p0_host[3] with direction d_host[3] (photon i uses history i's stream);
 * *through_host = how many leave the grid without a real collision. */
MC_API int mc_debug_beam(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t seed, uint64_t n,
                  const double *p0_host, const double *d_host, double e_kev, uint64_t *through_host);

/* Verification of the float forced-detection traversal's distance map
 * (the transmission of Sec. 4's forced detection, a line integral of mu):
 * out_host[v] (nz*ny*nx bytes, x fastest, caller-owned) = the largest
 * D <= 16 such that every voxel of the grid within chessboard distance D - 1
 * of voxel v holds v's material (voxels outside the grid do not count).
 * MC_EINVAL for an invalid phantom or a NULL out_host.  Synchronises. */
MC_API int mc_debug_distance_map(const mc_phantom *phantom, uint8_t *out_host);

/* Number of kernels this library has launched in this process (all
 * devices, all threads); for launch accounting in benchmarks. */
MC_API uint64_t mc_kernel_launches(void);

/* Message of the last error on this thread ("" if none). */
MC_API const char *mc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MCSPECT_H */
