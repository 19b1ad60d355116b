/*
 * lens.h -- C ABI of the GB300 parametric strong-lensing evaluator.
 *
 * The library evaluates a lens model -- a sum of elliptical dPIE potentials
 * plus SIS and point-mass terms -- at many image-plane points, and builds on
 * that evaluation the maps and the chi2 of a parametric cluster-lens fit
 * (Schaefer, Fourestey & Kneib, "Lenstool-HPC"):
 *   - deflection (gradient) maps over a rectangular grid          Sec. 4.1, Eq. 10
 *   - kappa / gamma / magnification maps from the summed Hessian  Sec. 2.4, Eqs. 7-9;
 *                                                                  Sec. 2.1, Eqs. 4-5
 *   - chi2 of multiple-image constraints, source-plane form       Sec. 2.2, Eq. 6, Fig. 3
 *   - chi2 with predicted images from a ray-shot triangulated grid Sec. 2.3, Fig. 4;
 *                                                                  Sec. 4.2, Fig. 8
 *
 * Conventions (all calls):
 *   - Units are arcsec; angles in radians counter-clockwise from +x to the
 *     major axis; x to the right.
 *   - dPIE profile (Eliasdottir et al. 2007, cited in Sec. 2.2):
 *       kappa = (b0/2)[(rcore^2 + rho^2)^-1/2 - (rcut^2 + rho^2)^-1/2],
 *       rho^2 = x^2/(1+eps)^2 + y^2/(1-eps)^2 in the halo frame.
 *     SIS: alpha = b0 theta/|theta|.  Point mass: alpha = b0^2 theta/|theta|^2.
 *     At the exact centre of an SIS or point mass the deflection and Hessian
 *     are defined as zero.
 *   - Deflections and Hessians scale linearly with the distance ratio
 *     D_ls/D_s ("dls_ds").
 *   - Grids have inclusive corners: x_i = xmin + i (xmax-xmin)/(nx-1), and
 *     map planes are row-major [ny][nx] (j along y).
 *   - Every compute call is asynchronous on the caller's CUDA stream
 *     ("stream" is a cudaStream_t; NULL means the legacy default stream).
 *     Output buffers are caller-owned DEVICE memory; host-side descriptors
 *     (lens_halo, lens_grid, lens_constraints) are read before the call
 *     returns and may be freed afterwards.
 *   - Return value: LENS_OK (0) or a negative LENS_E* code; nothing is
 *     enqueued when a call returns an error.  lens_strerror() names a code;
 *     lens_last_error() gives a message for the calling thread's last error.
 *   - A context is not thread-safe: one host thread at a time per context.
 *     Its calls may target different streams and run concurrently on the
 *     GPU: a call's working memory is allocated and freed in stream order on
 *     that call's stream (from a memory pool of the context), so calls on
 *     different streams never share it (lens_chi2_image_noalloc excepted: see
 *     there).  No call but lens_destroy synchronises the device: releasing a
 *     model or constraint set, growing a buffer or replacing a cache frees
 *     the old memory on a stream of the context that first waits for every
 *     launch the context enqueued before the release.  Work captured into a
 *     CUDA graph is not tracked that way: release nothing a captured graph
 *     still reads before its last replay has finished.
 */
#ifndef LENS_H
#define LENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- codes */
#define LENS_OK 0
#define LENS_EINVAL (-1)    /* bad argument: NULL pointer, size <= 0, non-finite
                               or out-of-domain halo parameter, bad grid      */
#define LENS_ENOMEM (-2)    /* device allocation would exceed the context's
                               memory budget, or cudaMalloc failed            */
#define LENS_ENOTFOUND (-3) /* unknown model or constraint-set handle        */
#define LENS_ECAPACITY (-4) /* an internal image buffer overflowed; the chi2
                               of the affected parameter sets is NaN          */
#define LENS_ECUDA (-5)     /* a CUDA runtime call failed                     */
#define LENS_ETIMEOUT (-6)  /* lens_wait: the work did not finish in time, or
                               a device-side bounded wait gave up            */

/* Halo types. */
#define LENS_DPIE 0
#define LENS_SIS 1
#define LENS_POINT 2

/* Map precision.
 * LENS_FP64:  every potential in double precision; output planes are double.
 * LENS_MIXED: potentials whose strength b0 is below the context's FP64
 *             threshold are evaluated in FP32 with compensated accumulation,
 *             the others in FP64; output planes are float. */
#define LENS_FP64 0
#define LENS_MIXED 1

/* Source-plane chi2 variants (lens_chi2_source). */
#define LENS_CHI2_SRC_MAPPED 0   /* sum |A (bary - beta)|^2 / sigma^2, A = (I - H)^-1 */
#define LENS_CHI2_SRC_MU 1       /* sum |bary - beta|^2 |mu| / sigma^2                */
#define LENS_CHI2_SRC_PLAIN 2    /* sum |bary - beta|^2 / sigma^2                     */

typedef struct lens_ctx lens_ctx;
typedef int64_t lens_model_t; /* > 0 when valid */
typedef int64_t lens_cset_t;  /* > 0 when valid */

/* One potential.  dPIE uses every field: 0 <= eps < 1, 0 < rcore < rcut,
 * b0 > 0.  SIS and point mass use (x0, y0, b0) with b0 > 0; the remaining
 * fields must be finite and are ignored. */
typedef struct {
  int32_t type;
  double x0, y0, theta, eps, rcore, rcut, b0;
} lens_halo;

/* Rectangular grid, inclusive corners; nx, ny >= 2, xmax > xmin, ymax > ymin,
 * at most 2^31 - 1 nodes (node indices are 32-bit) and at most 524 280 rows
 * (65 535 CTA rows of 8 grid rows); a grid beyond these is LENS_EINVAL. */
typedef struct {
  double xmin, xmax, ymin, ymax;
  int32_t nx, ny;
} lens_grid;

/* Multiple-image constraints (HOST pointers).  Source i owns images
 * img_off[i] .. img_off[i+1]-1 (img_off[0] = 0, non-decreasing); x, y are
 * image positions, sigma their positional error (> 0), dls_ds[i] the
 * source's distance ratio D_ls/D_s (> 0). */
typedef struct {
  int32_t nsrc;
  const int32_t *img_off;
  const double *x;
  const double *y;
  const double *sigma;
  const double *dls_ds;
} lens_constraints;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  mem_budget_bytes bounds the
 * device memory the context may hold (models, constraint sets, caches,
 * working memory of the calls in progress on the host); 0 means no bound.
 * The context allocates from a device memory pool of its own, which keeps
 * the memory it has held for reuse until lens_destroy.  *out receives the
 * context. */
int lens_create(lens_ctx **out, int device, size_t mem_budget_bytes);

/* Release every model, constraint set and buffer of the context and free it.
 * Synchronises the device first (the one call that does).  NULL is
 * accepted. */
int lens_destroy(lens_ctx *ctx);

/* Potentials with b0 >= threshold_b0 are evaluated in FP64 by LENS_MIXED
 * maps (default 5 arcsec) -- in double-float on the FP32 pipe instead (about
 * 1e-13 relative, FP64 where that fails) by the deflection and Hessian maps
 * of a model with fewer than 400 other potentials per such potential, where
 * the FP64 unit (1/64 of the FP32 rate) would set the pace.  Applies to
 * models uploaded afterwards. */
int lens_set_fp64_threshold(lens_ctx *ctx, double threshold_b0);

/* LENS_MIXED deflection and Hessian maps: where the deflection at a node is
 * small next to the summed magnitudes of its FP32 terms -- near a zero of
 * alpha, where the terms cancel -- their rounding error (measured at about
 * 1.6e-7 of that sum) would exceed 1e-6 |alpha|.  Such nodes (|alpha| <
 * r x the sum of |alpha_i| over the FP32 potentials, each term's |alpha_i|
 * taken as |alpha_x'| + |alpha_y'| in its own frame) are listed by the map
 * kernel and recomputed, every potential in double-float (~1e-13), by a
 * second kernel on the same stream; every plane of those nodes is
 * rewritten.  r = LENS_REPAIR_RATIO_DEFAULT = 0.16 by default: outside the
 * repaired nodes the measured error then stays below 0.83 of 1e-6 |alpha|
 * (the FP32 error never exceeded 1.32e-7 of the sum on the models measured);
 * r = 0 turns the repair off.
 * The list is working memory of the call (4 bytes per grid point, stream
 * ordered).  LENS_EINVAL for r < 0 or not finite. */
int lens_set_repair_ratio(lens_ctx *ctx, double r);
#define LENS_REPAIR_RATIO_DEFAULT 0.16

/* Device bytes currently held by the context (including released model
 * blocks kept for reuse by later uploads; those are freed first when an
 * allocation would exceed the budget). */
size_t lens_mem_used(const lens_ctx *ctx);
/* Device bytes holding an uploaded model (its records and the staged halo
 * table they were built from); 0 for an unknown model. */
size_t lens_model_bytes(lens_ctx *ctx, lens_model_t model);

/* ------------------------------------------------------------------ models */

/* Upload n >= 1 potentials (host array, copied).  Validates every field
 * (LENS_EINVAL on the first bad one) and orders the potentials on the host,
 * copies the table (n x 64 bytes) and one int32 slot per potential to the
 * device, where one kernel precomputes every potential's constants in double
 * precision into its records (Sec. 3.2 structure-of-arrays discussion; here
 * a packed per-potential record read by all threads at once).  Synchronous.
 * The model is immutable and owned by the context until lens_model_release. */
int lens_model_upload(lens_ctx *ctx, const lens_halo *h, int32_t n, lens_model_t *out);
int lens_model_release(lens_ctx *ctx, lens_model_t model);

/* ------------------------------------------------------------------- maps */

/* Deflection map (Sec. 4.1, Eq. 10; lens equation Sec. 2.1 Eq. 1):
 * d_out holds 2 planes [2][ny][nx] -- alpha_x, alpha_y -- of float
 * (LENS_MIXED) or double (LENS_FP64), 16-byte aligned. */
int lens_grad_map(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                  void *d_out, void *stream);

/* Deflection + Hessian maps (Sec. 2.4, Eqs. 7-9; Sec. 2.1, Eqs. 4-5):
 * d_out holds 6 planes [6][ny][nx] -- alpha_x, alpha_y, kappa, gamma1,
 * gamma2, mu -- with kappa = (psi_xx+psi_yy)/2, gamma1 = (psi_xx-psi_yy)/2,
 * gamma2 = psi_xy of the summed Hessian and mu = 1/((1-kappa)^2 - gamma1^2 -
 * gamma2^2).  Element type as for lens_grad_map. */
int lens_hessian_map(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                     void *d_out, void *stream);

/* Lensing potential map (Sec. 2.4's list of map kinds; the potential of
 * Sec. 2.1 Eq. 2): d_out holds phi [ny][nx], the summed potential times
 * dls_ds, with each dPIE term x alpha_x' + y alpha_y' - b q s ln
 * sqrt((psi+s)^2 + u^2 x^2) (core minus cut, halo frame), SIS b r and point
 * mass theta_E^2 ln r (0 at the centre); phi is defined up to this constant.
 * When beta (host, {x, y} in arcsec) is not NULL, a second plane follows:
 * the time-delay (Fermat) surface tau = |theta - beta|^2 / 2 - phi in
 * arcsec^2 (times (1+z_l) D_l D_s / (c D_ls) it is the delay; the distances
 * are the caller's).  The planes are double for both precisions (phi
 * carries an additive constant of order b0 r_cut ln r_cut that float would
 * round to ~1e-2), 8-byte aligned; errors as for lens_grad_map, and
 * LENS_EINVAL for a non-finite beta.  LENS_MIXED evaluates the potentials
 * below the FP64 threshold in FP32 (logarithms by the MUFU log2), the rest in
 * FP64; LENS_FP64 evaluates every potential in FP64. */
int lens_potential_map(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                       const double *beta, void *d_out, void *stream);

/* The same maps written to page-locked HOST memory h_out ([2 or 6][ny][nx],
 * float for LENS_MIXED, double for LENS_FP64, from cudaHostAlloc or
 * cudaHostRegister; LENS_EINVAL otherwise).  The grid is computed in about 8
 * row bands on two streams of the context and each band is copied to the
 * host as soon as it is done, so the copy overlaps the rest of the map; the
 * values equal those of lens_grad_map / lens_hessian_map.  Asynchronous:
 * h_out is complete when `stream` reaches this point.  Uses two device band
 * buffers owned by the context (counted in lens_mem_used); calls on
 * different streams go through them one after the other, in call order. */
int lens_grad_map_host(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                       void *h_out, void *stream);
int lens_hessian_map_host(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds,
                          int32_t precision, void *h_out, void *stream);

/* ----------------------------------------------------------- chi2 batches */

/* Bind a constraint table to a model for batched chi2 evaluation.
 * var_halo[0], var_halo[1] (distinct, < n) are the two potentials whose
 * parameters each parameter set replaces; every other potential is static,
 * and its FP64 deflection and Hessian at the constraint positions are
 * computed here once (the static cache).  Synchronous (on a stream of the
 * context).  The constraint table is copied.  The chi2 calls take the
 * returned handle in place of a (model, constraints, var_halo) triple per
 * call, so the static cache stays resident across the calls of a fit. */
int lens_cset_create(lens_ctx *ctx, lens_model_t model, const lens_constraints *c, const int32_t var_halo[2],
                     lens_cset_t *out);
int lens_cset_release(lens_ctx *ctx, lens_cset_t cset);

/* Source-plane chi2 of P parameter sets (Sec. 2.2, Eq. 6 and Fig. 3):
 * each set replaces (x0, y0, eps, theta, rcore, rcut, b0) of var_halo[0]
 * then var_halo[1] -- d_params is DEVICE double [P][14].  For every image
 * beta = theta - r alpha(theta) (Sec. 2.1, Eq. 1), the source estimate is the
 * barycentre of its images, and d_chi2[p] (DEVICE double [P]) receives the
 * variant's sum.  The static potentials' cache is FP64; the two varying
 * potentials are evaluated in double-float (pairs of floats, ~1e-13 relative;
 * FP64 where that fails); the back-trace, barycentres and sums are FP64.  A
 * parameter set outside the dPIE domain yields NaN. */
int lens_chi2_source(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, int32_t variant,
                     double *d_chi2, void *stream);

/* Source-plane chi2 with the cluster members' scaling relations free as
 * well (Sec. 2.2: a cluster model's free parameters include the members'
 * scaling relations, b0_i = b0* s_i and r_cut,i = r_cut* s_i): d_params is
 * DEVICE double [P][16], the 14 parameters of lens_chi2_source followed by
 * f_b and f_t, which multiply b0 of every static potential and r_cut of every
 * static dPIE (r_core stays).  The static sums are recomputed for every set
 * in double-float (~1e-13 relative per potential; the r_cut-dependent
 * constants rebuilt from f_t r_cut in double-float; FP64 where that fails)
 * in batches of 512 sets, into working memory of the call (as
 * lens_chi2_source_nocache).  NaN for a set outside the domain (f_b or f_t
 * not positive, or f_t r_cut <= r_core for a member). */
int lens_chi2_source_scaled(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, int32_t variant,
                            double *d_chi2, void *stream);

/* The static cache made a function of the members' r_cut factor: the static
 * sums at f_b = 1 and `nodes` (8..128) Chebyshev points of f_t in
 * [ft_min, ft_max] (second kind, x_k = mid + half cos(pi k / (nodes-1)),
 * computed as lens_chi2_source_scaled does), after which
 * lens_chi2_source_scaled (and 16-parameter lens_mcmc_step) takes each set's
 * sums from their barycentric interpolant in f_t (Berrut and Trefethen 2004)
 * times f_b, instead of recomputing every member: the sums are analytic in
 * f_t, so the interpolant converges geometrically (32 nodes on [0.5, 2]:
 * the sums to ~1e-12, the chi2 to a median ~1e-13 and at most ~5e-9 of
 * the recomputed one on the 1000-potential model, within the chi2
 * tolerance of the definition).
 * Sets with f_t outside [ft_min, ft_max] then give NaN (a bounded prior).
 * LENS_EINVAL when ft_min would put a member's r_cut at or below its r_core;
 * nodes = 0 drops the cache.  Synchronous; device memory nodes x images x
 * 40 bytes. */
int lens_cset_scaling_cache(lens_ctx *ctx, lens_cset_t cset, double ft_min, double ft_max, int32_t nodes);

/* One Metropolis step of W independent Markov chains over the varying
 * parameters (the Bayesian fit of Sec. 2.2: likelihood exp(-chi2/2) of the
 * source-plane chi2 of Eq. 6, flat prior over the domain).  nparams = 14:
 * the two varying potentials, chi2 as lens_chi2_source; nparams = 16: also
 * the members' scaling factors, chi2 as lens_chi2_source_scaled.  d_params
 * (DEVICE double [W][nparams]) and d_chi2 (DEVICE double [W], each chain's
 * current chi2; NaN makes the chain take any valid proposal) are updated in
 * place.  Chain w proposes theta' = theta + sigma z with d_sigma DEVICE
 * double [nparams] (standard deviations) and z standard normal, and moves
 * when ln u < -(chi2' - chi2) / (2 temperature); a proposal outside the
 * domain is refused.  z and u come from Philox4x64-10 (Salmon et al. 2011)
 * with key (seed, 0) and counters (step, w, j, 0): word x gives
 * ((x >> 11) + 1/2) 2^-53; j = 0..3 give 16 words, 8 Box-Muller pairs
 * (sqrt(-2 ln u_2i) (cos, sin)(2 pi u_2i+1)) of which the first nparams
 * normals are used, and word 0 of j = 4 is u; the same (seed, step) replays
 * the same step.  d_scratch: DEVICE double [(nparams + 2) W] (proposals, the
 * uniforms, the proposals' chi2); d_accepted: DEVICE int32 [W] (1 = moved)
 * or NULL.  temperature > 0; variant as for lens_chi2_source.  Asynchronous
 * on `stream`: three launches for nparams = 14 (no allocation), the scaled
 * chi2's batches of 512 for 16 (with its working memory).  A CUDA graph
 * captured from it replays the captured step's draws (seed and step are
 * launch arguments); lens_mcmc_step_dev keeps the step in device memory. */
int lens_mcmc_step(lens_ctx *ctx, lens_cset_t cset, double *d_params, double *d_chi2, int32_t W, int32_t nparams,
                   const double *d_sigma, double temperature, uint64_t seed, uint64_t step, int32_t variant,
                   double *d_scratch, int32_t *d_accepted, void *stream);

/* lens_mcmc_step with the step counter in device memory: d_step is DEVICE
 * uint64 [1]; the step draws its Philox counters (step, w, j, 0) with step =
 * *d_step as the proposals are formed, and its last kernel adds 1 to
 * *d_step.  A CUDA graph captured from one call therefore draws the next
 * step's numbers at every replay (with lens_mcmc_step, seed and step are
 * launch arguments and a replay repeats the captured step).  The caller
 * sets *d_step before the first step (any value; the same value replays the
 * same sequence).  Arguments, errors and asynchrony otherwise as
 * lens_mcmc_step; LENS_EINVAL when d_step is NULL. */
int lens_mcmc_step_dev(lens_ctx *ctx, lens_cset_t cset, double *d_params, double *d_chi2, int32_t W,
                       int32_t nparams, const double *d_sigma, double temperature, uint64_t seed, uint64_t *d_step,
                       int32_t variant, double *d_scratch, int32_t *d_accepted, void *stream);

/* lens_chi2_source without the static cache: the deflection and Hessian of
 * every static potential at every image are recomputed for every parameter
 * set (double-float, summed in FP64; batches of 512 sets in working memory
 * of the call), as in the paper's fit, which evaluates every potential for
 * every model (Sec. 2.2, Sec. 4.2).  Same arguments, results (to ~1e-10
 * relative) and errors as lens_chi2_source; the per-set cost is N potentials
 * x images instead of 2 x images.  Working memory 512 x images x 40 bytes,
 * allocated and freed in stream order on `stream` (LENS_ENOMEM over the
 * budget). */
int lens_chi2_source_nocache(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, int32_t variant,
                             double *d_chi2, void *stream);

/* Autotuner of lens_chi2_source's launch shape (threads per CTA x CTAs per
 * SM, 8 candidates) for this constraint set: runs each candidate on d_params
 * (DEVICE [P][14]) into d_chi2 (DEVICE [P]) on `stream`, times it (best of
 * 3 after a warm-up), and keeps the fastest for every later lens_chi2_source
 * call on the set.  Synchronous.  *chosen (may be NULL) = threads*100 +
 * CTAs-per-SM cap (0 = no cap); *best_ms (may be NULL) its time. */
int lens_chi2_autotune(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, double *d_chi2,
                       void *stream, int32_t *chosen, float *best_ms);

/* Image-plane chi2 of P parameter sets (Sec. 2.2, Eq. 6 with the brute-force
 * image search of Sec. 2.3, Fig. 4 and Sec. 4.2): per set, the grid is
 * ray-shot to each source's plane, every triangle containing the source's
 * barycentre seeds a Newton solve of the lens equation with the full model,
 * solutions closer than 1e-3 arcsec merge, and each constraint is matched to
 * the nearest predicted image of its source.  d_chi2: DEVICE double [P];
 * d_nimg_found: DEVICE int32 [P][nsrc] (may be NULL) receives the number of
 * distinct images found per source (-1 for every source of a set whose
 * candidate buffer, 4096 candidates, overflowed).  A source without images,
 * or an overflow, makes that set's chi2 NaN; an overflow also sets the
 * context's error flag, which the next lens_wait reports as LENS_ECAPACITY
 * (and clears).  At most 1024 sources per constraint set (LENS_EINVAL
 * beyond, nothing launched).  The first call on a (constraint set, grid)
 * pair computes and keeps the static potentials' deflection on the grid;
 * each call's candidate buffers are working memory allocated and freed in
 * stream order on `stream`. */
int lens_chi2_image(lens_ctx *ctx, lens_cset_t cset, const lens_grid *grid, const double *d_params, int32_t P,
                    double *d_chi2, int32_t *d_nimg_found, void *stream);

/* Predicted images of P parameter sets: the search of lens_chi2_image
 * (Sec. 2.3, Fig. 4; Sec. 4.2) without the matching.  Per set p, d_images
 * (DEVICE double [P][max_per_set][3]) receives (x, y, source index) of each
 * distinct image of every source's barycentre, in no particular order, and
 * d_count[p] (DEVICE int32 [P]) their number (-1 on a candidate-buffer
 * overflow, 0 for a set outside the model's domain; only the first
 * max_per_set are written). */
int lens_find_images(lens_ctx *ctx, lens_cset_t cset, const lens_grid *grid, const double *d_params, int32_t P,
                     double *d_images, int32_t max_per_set, int32_t *d_count, void *stream);

/* Image-plane chi2 that allocates nothing (the paper has no counterpart).
 * For callers that reserve all device memory up front and may not call
 * cudaMalloc/cudaFree at call time -- e.g. a long-running sampler or request
 * loop: those calls can synchronise the whole device and can fail under
 * memory pressure mid-run.  Same arguments, results and error behaviour as
 * lens_chi2_image, but every working buffer lives in one fixed file-scope
 * device array of LENS_NOALLOC_SCRATCH_BYTES, held by every GPU that loads
 * the library until the process exits.  The context, model and constraint
 * set must already exist (they allocate when created).
 *   - The first call on a device looks up that array's device address; make
 *     that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's contents; each
 *     call rewrites everything it reads.  Calls whose work overlaps on the
 *     GPU (different streams, or different contexts on one device) race.
 *   - LENS_EINVAL, with a message, when the grid's static deflection
 *     (8 bytes per node) plus the buffers of one parameter set do not fit. */
#define LENS_NOALLOC_SCRATCH_BYTES (16u << 20)
int lens_chi2_image_noalloc(lens_ctx *ctx, lens_cset_t cset, const lens_grid *grid, const double *d_params,
                            int32_t P, double *d_chi2, int32_t *d_nimg_found, void *stream);

/* ---------------------------------------------------------- request loop */
/* A server runs map and chi2 requests of uneven sizes on `slots` CUDA
 * streams of its own, admitting queued requests whenever a slot is free and
 * their device buffers fit in the server's pool -- one allocation of
 * pool_bytes made at creation and counted against the context budget.  The
 * order is shortest expected GPU time first, less the time already waited (a
 * large request waits at most about its own run time); a request that does
 * not fit may be overtaken until it has been passed over 64 times.  Work of different slots overlaps on the device; each
 * request runs the same kernels as the direct calls on its own buffers, so
 * its result does not depend on what else is in flight.  Models and
 * constraint sets stay resident in the context.  Not part of the paper's
 * method: it serves the maps (Sec. 2.4) and chi2 (Sec. 2.2) above. */
#define LENS_REQ_MAP 0
#define LENS_REQ_CHI2_SOURCE 1
#define LENS_REQ_CHI2_IMAGE 2

typedef struct lens_server lens_server;

typedef struct {
  int32_t kind;          /* LENS_REQ_*                                          */
  int64_t handle;        /* model (maps) or constraint set (chi2)               */
  lens_grid grid;        /* maps and image-plane chi2                           */
  double dls_ds;         /* maps                                                */
  int32_t precision;     /* maps: LENS_MIXED or LENS_FP64                       */
  int32_t hessian;       /* maps: 0 = 2 deflection planes, 1 = all 6 planes      */
  int32_t variant;       /* source-plane chi2                                   */
  int32_t P;             /* chi2: number of parameter sets                      */
  const double *params;  /* chi2: HOST double [P][14], copied at submit         */
  void *result;          /* PAGE-LOCKED host destination: the map planes (as
                            lens_grad_map / lens_hessian_map lay them out) or
                            double [P] chi2; written when the ticket completes */
} lens_request;

typedef struct {
  int64_t ticket;
  int32_t status;        /* LENS_OK or the error that ended the request         */
  double queue_ms;       /* submit -> admitted onto a slot                      */
  double latency_ms;     /* submit -> completion observed by lens_server_progress */
} lens_completion;

typedef struct {
  int32_t queued, inflight;
  size_t pool_bytes, pool_used, pool_peak;
} lens_server_info;

int lens_server_create(lens_ctx *ctx, int32_t slots, size_t pool_bytes, lens_server **out);
/* Waits for the work in flight, drops queued requests, frees the pool. */
int lens_server_destroy(lens_server *s);
/* Validate and queue; never blocks on the GPU (the first image-plane request
 * for a new (constraint set, grid) pair builds that pair's static deflection
 * synchronously).  LENS_ENOMEM if the request can never fit in the pool. */
int lens_server_submit(lens_server *s, const lens_request *r, int64_t *ticket);
/* Non-blocking: retire finished requests into done[0..cap) (*n_done of them),
 * then admit queued requests onto free slots. */
int lens_server_progress(lens_server *s, lens_completion *done, int32_t cap, int32_t *n_done);
/* Remove a request that has not been admitted yet (LENS_ENOTFOUND otherwise). */
int lens_server_cancel(lens_server *s, int64_t ticket);
int lens_server_stats(const lens_server *s, lens_server_info *info);

/* --------------------------------------------------------------- control */

/* Exercises the device-side failure path (no counterpart in the paper): a
 * one-thread kernel waits on an mbarrier that nothing completes, gives up
 * after `polls` (1..2^20) tries as every bounded wait of the library does,
 * and sets the context's error flag, so the next lens_wait returns
 * LENS_ETIMEOUT (and clears it).  Asynchronous on `stream`; nothing faults
 * and the context stays usable. */
int lens_selftest_wait(lens_ctx *ctx, int32_t polls, void *stream);

/* The FP64 reciprocal and reciprocal square root the FP64 evaluators use
 * (MUFU approximation + two Newton-Raphson steps) next to CUDA's division
 * and rsqrt, for testing: for each of the n doubles at d_x (device, positive
 * normal values), d_out (device, [4][n]) receives rcp, 1/x, rsqrt, CUDA
 * rsqrt.  Asynchronous on `stream`. */
int lens_selftest_math(lens_ctx *ctx, const double *d_x, int32_t n, double *d_out, void *stream);

/* Wait until all work enqueued on `stream` has finished, polling without
 * blocking the thread for more than timeout_ms (>= 0) milliseconds.
 * LENS_ETIMEOUT if it has not finished by then (the work keeps running). */
int lens_wait(lens_ctx *ctx, void *stream, int64_t timeout_ms);

const char *lens_strerror(int code);
const char *lens_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LENS_H */
