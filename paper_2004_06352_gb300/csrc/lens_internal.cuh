// Internal declarations of the GB300 lens library (not part of the C ABI).
//
// Device model store: every uploaded model keeps
//   rec32  float  [n_light][32]  packed FP32 constants of the potentials
//                                evaluated in FP32 (one 128-byte record per
//                                potential; all threads of a CTA read the same
//                                record, so a packed record is a broadcast)
//   pos64  double [n_light][4]   x0, y0, cos(theta), sin(theta) in FP64: the
//                                per-tile offsets of each potential are formed
//                                from these in double precision
//   heavy  double [n_heavy][16]  FP64 records of the potentials whose strength
//                                b0 is at or above the FP64 threshold
//   all64  double [n][16]        FP64 records of every potential, in upload
//                                order (FP64 maps, chi2 static cache, Newton)
#pragma once

#include <cstdint>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/lens.h"

namespace lens {

// ---------------------------------------------------------------- records
// FP32 record (32 floats).  Kinds, stored as int bits in slot K_KIND.
enum Kind32 : int { K32_DPIE = 0, K32_DPIE_SERIES = 1, K32_SIS = 2, K32_POINT = 3 };
enum Rec32 : int {
  R_C = 0, R_S, R_Q2, R_U2,          // rotation, q^2, u^2
  R_KC, R_KT, R_SC, R_ST,            // q^2 sc^2, q^2 st^2, sc, st
  R_DK, R_DS, R_Q2SC, R_Q2ST,       // q^2 (st^2 - sc^2), st-sc, q^2 sc, q^2 st
  R_UDK, R_Q2DS, R_U2SC2, R_U2ST2,   // u dK, q^2 (st-sc), u^2 sc^2, u^2 st^2
  R_CB, R_SB, R_KAPS, R_IU,          // rotation times b q, kappa scale b q / 2, 1/u
  R_C1, R_C2, R_C3, R_C4,            // shear rotation by 2 theta with the scale folded in
  R_U, R_UDS, R_UQ2DS, R_CBU,        // u, u dS, u q^2 dS, R_CB / u
  R_KIND, R_B, R_SBU, R_KAPSU        // kind, SIS b / point-mass b^2, R_SB / u, R_KAPS / u
};
// (the u-folded fields are set for K32_DPIE only: its u >= U_SERIES32)
constexpr int REC32 = 32;

// FP64 record (16 doubles).
enum Kind64 : int { K64_DPIE = 0, K64_DPIE_SERIES = 1, K64_SIS = 2, K64_POINT = 3 };
enum Rec64 : int {
  D_X0 = 0, D_Y0, D_C, D_S, D_Q2, D_U, D_U2, D_BQ, D_SC, D_ST, D_DS, D_SS, D_C2T, D_S2T, D_KIND, D_B
};
constexpr int REC64 = 16;

// u = sqrt(1 - q^2) below which the FP32 / FP64 paths always use the
// polynomial / series forms of atan(w)/w and atanh(w)/w (|w| < u there).
constexpr double U_SERIES32 = 0.12;
constexpr double U_SERIES64 = 1e-4;

// Host + device: FP64 record from user parameters (shared by model upload
// and by the chi2 kernels, which rebuild the varying potentials per set).
__host__ __device__ inline void make_rec64(int type, double x0, double y0, double theta, double eps, double rcore,
                                           double rcut, double b0, double *r) {
  for (int k = 0; k < REC64; ++k) r[k] = 0.0;
  r[D_X0] = x0;
  r[D_Y0] = y0;
  if (type == LENS_SIS || type == LENS_POINT) {
    r[D_C] = 1.0;
    r[D_KIND] = type == LENS_SIS ? K64_SIS : K64_POINT;
    r[D_B] = type == LENS_SIS ? b0 : b0 * b0;
    return;
  }
  double q = (1.0 - eps) / (1.0 + eps);
  double u = 2.0 * sqrt(eps) / (1.0 + eps);
  double b = b0 * (1.0 + eps);
  double sc = rcore * (1.0 + eps), st = rcut * (1.0 + eps);
  const double c = cos(theta), s = sin(theta);
  r[D_C] = c;
  r[D_S] = s;
  r[D_Q2] = q * q;
  r[D_U] = u;
  r[D_U2] = u * u;
  r[D_BQ] = b * q;
  r[D_SC] = sc;
  r[D_ST] = st;
  r[D_DS] = st - sc;
  r[D_SS] = st + sc;
  r[D_C2T] = (c - s) * (c + s);  // double-angle formulas
  r[D_S2T] = 2.0 * s * c;
  r[D_KIND] = u < U_SERIES64 ? K64_DPIE_SERIES : K64_DPIE;
}

// Host + device: FP32 record of one potential (constants formed in FP64).
__host__ __device__ inline void make_rec32(int type, double theta, double eps, double rcore, double rcut, double b0,
                                           float *r) {
  for (int k = 0; k < REC32; ++k) r[k] = 0.f;
  int kind;
  if (type == LENS_SIS || type == LENS_POINT) {
    r[R_C] = 1.f;
    kind = type == LENS_SIS ? K32_SIS : K32_POINT;
    r[R_B] = (float)(type == LENS_SIS ? b0 : b0 * b0);
  } else {
    double e = eps;
    double q = (1.0 - e) / (1.0 + e), u = 2.0 * sqrt(e) / (1.0 + e);
    double q2 = q * q, u2 = u * u;
    double b = b0 * (1.0 + e), bq = b * q;
    double sc = rcore * (1.0 + e), st = rcut * (1.0 + e);
    double c2 = cos(2.0 * theta), s2 = sin(2.0 * theta);
    bool series = u < U_SERIES32;
    kind = series ? K32_DPIE_SERIES : K32_DPIE;
    r[R_C] = (float)cos(theta);
    r[R_S] = (float)sin(theta);
    r[R_Q2] = (float)q2;
    r[R_U2] = (float)u2;
    r[R_KC] = (float)(q2 * sc * sc);
    r[R_KT] = (float)(q2 * st * st);
    r[R_SC] = (float)sc;
    r[R_ST] = (float)st;
    r[R_DK] = (float)(q2 * (st - sc) * (st + sc));
    r[R_DS] = (float)(st - sc);
    r[R_Q2SC] = (float)(q2 * sc);
    r[R_Q2ST] = (float)(q2 * st);
    r[R_Q2DS] = (float)(q2 * (st - sc));
    r[R_U2SC2] = (float)(u2 * sc * sc);
    r[R_U2ST2] = (float)(u2 * st * st);
    r[R_CB] = (float)(cos(theta) * bq);
    r[R_SB] = (float)(sin(theta) * bq);
    r[R_KAPS] = (float)(0.5 * bq);
    r[R_IU] = (float)(series ? 0.0 : 1.0 / u);
    r[R_U] = (float)u;
    if (!series) {
      r[R_UDK] = (float)(u * q2 * (st - sc) * (st + sc));
      r[R_UDS] = (float)(u * (st - sc));
      r[R_UQ2DS] = (float)(u * q2 * (st - sc));
      r[R_CBU] = (float)(cos(theta) * bq / u);
      r[R_SBU] = (float)(sin(theta) * bq / u);
      r[R_KAPSU] = (float)(0.5 * bq / u);
    }
    r[R_C1] = (float)(c2 * 0.5 * bq);
    r[R_C2] = (float)(s2 * bq);
    r[R_C3] = (float)(s2 * 0.5 * bq);
    r[R_C4] = (float)(-c2 * bq);
  }
#ifdef __CUDA_ARCH__
  r[R_KIND] = __int_as_float(kind);
#else
  std::memcpy(&r[R_KIND], &kind, sizeof(int));
#endif
}


// Host + device: are the parameters inside the model's domain?
__host__ __device__ inline bool halo_params_ok(int type, double x0, double y0, double theta, double eps, double rcore,
                                               double rcut, double b0) {
  if (!(isfinite(x0) && isfinite(y0) && isfinite(theta) && isfinite(eps) && isfinite(rcore) && isfinite(rcut) &&
        isfinite(b0)))
    return false;
  if (!(b0 > 0.0)) return false;
  if (type == LENS_SIS || type == LENS_POINT) return true;
  if (type != LENS_DPIE) return false;
  return eps >= 0.0 && eps < 1.0 && rcore > 0.0 && rcut > rcore;
}

// ---------------------------------------------------------------- objects
// Double-float record of one potential: 16 (hi, lo) float pairs.
enum RecDF : int {
  F_X0 = 0, F_Y0, F_C, F_S, F_Q2, F_U2, F_KC, F_KT, F_SC, F_ST, F_Q2SC, F_Q2ST, F_Q2SS, F_Q2DS, F_SS, F_BQ,
  // Hessian: cos 2theta, sin 2theta, (1+q^2) s^2 and u^2 s^2 of both terms,
  // q^2 (st^2 - sc^2), b q / 2
  F_C2, F_S2, F_DC0, F_DT0, F_U2SC2, F_U2ST2, F_KTC, F_HB
};
constexpr int RECDF = 24;
// SIS and point-mass records carry F_U2 = -1 and -2 (never negative for a
// dPIE) and b, theta_E^2 in F_BQ.

// Host + device: double-float record from user parameters; pair k goes to
// r[k * stride].
__host__ __device__ inline void make_recdf(int type, double x0, double y0, double theta, double eps, double rcore,
                                           double rcut, double b0, float2 *r, int stride = 1) {
  double v[RECDF];
  for (int k = 0; k < RECDF; ++k) v[k] = 0.0;
  v[F_X0] = x0;
  v[F_Y0] = y0;
  if (type == LENS_SIS || type == LENS_POINT) {
    v[F_C] = 1.0;
    v[F_U2] = type == LENS_SIS ? -1.0 : -2.0;
    v[F_BQ] = type == LENS_SIS ? b0 : b0 * b0;
  } else {
    const double q = (1.0 - eps) / (1.0 + eps), u = 2.0 * sqrt(eps) / (1.0 + eps);
    const double q2 = q * q, sc = rcore * (1.0 + eps), st = rcut * (1.0 + eps);
    const double c = cos(theta), s = sin(theta);
    v[F_C] = c;
    v[F_S] = s;
    v[F_Q2] = q2;
    v[F_U2] = u * u;
    v[F_KC] = q2 * sc * sc;
    v[F_KT] = q2 * st * st;
    v[F_SC] = sc;
    v[F_ST] = st;
    v[F_Q2SC] = q2 * sc;
    v[F_Q2ST] = q2 * st;
    v[F_Q2SS] = q2 * (st + sc);
    v[F_Q2DS] = q2 * (st - sc);
    v[F_SS] = st + sc;
    v[F_BQ] = b0 * (1.0 + eps) * q;
    v[F_C2] = (c - s) * (c + s);  // cos 2 theta, sin 2 theta by the double-angle formulas
    v[F_S2] = 2.0 * s * c;
    v[F_DC0] = (1.0 + q2) * sc * sc;
    v[F_DT0] = (1.0 + q2) * st * st;
    v[F_U2SC2] = u * u * sc * sc;
    v[F_U2ST2] = u * u * st * st;
    v[F_KTC] = q2 * (st - sc) * (st + sc);
    v[F_HB] = 0.5 * v[F_BQ];
  }
  for (int k = 0; k < RECDF; ++k) {
    const float h = (float)v[k];
    r[(size_t)k * stride] = make_float2(h, (float)(v[k] - (double)h));
  }
}

struct Model {
  void *block = nullptr;    // one device allocation holding every array below
  size_t payload = 0;       // bytes of the records and staged table in it (bytes: the block's size)
  int32_t n = 0, n_light = 0, n_heavy = 0;
  int32_t koff[5] = {0, 0, 0, 0, 0};  // light potentials sorted by kind: Kind32 k occupies [koff[k], koff[k+1])
  float *rec32 = nullptr;
  double *pos64 = nullptr;
  float *cen32 = nullptr;   // [n_light][4]: x0, y0 as hi/lo float pairs (hi x, hi y, lo x, lo y)
  double *heavy = nullptr;
  double *all64 = nullptr;
  float2 *recdf = nullptr;  // [RECDF][n] double-float records, field-major, upload order (image polish)
  float2 *heavydf = nullptr;  // [n_heavy][RECDF] double-float records of the heavy potentials (image refinement)
  std::vector<lens_halo> host;
  size_t bytes = 0;
};

struct GridCache {
  double xmin, xmax, ymin, ymax;
  int32_t nx, ny;
  float *alpha32 = nullptr;  // [2][ny][nx] deflection of the static potentials, D_ls/D_s = 1 (LENS_MIXED map)
  size_t bytes = 0;
};

struct CSet {
  lens_model_t model = 0;
  int32_t nsrc = 0, nimg = 0;
  int32_t var[2] = {0, 0};
  int32_t *img_off = nullptr;   // [nsrc+1]
  int32_t *src_of = nullptr;    // [nimg]
  double *x = nullptr, *y = nullptr, *sigma = nullptr;  // [nimg]
  double *isig2 = nullptr;      // [nimg] 1 / sigma^2
  double *ratio = nullptr;      // [nsrc]
  double *stat = nullptr;       // [nimg][5]: ax, ay, hxx, hyy, hxy of the static potentials (D_ls/D_s = 1)
  double *var_base = nullptr;   // [2][16] FP64 records of the varying potentials' base types (type in D_KIND)
  int32_t var_type[2] = {0, 0};
  Model *stat_model = nullptr;  // every potential except the two varying ones
  int32_t tuned_cfg = -1;       // launch shape of the source-plane chi2 picked by the autotuner
  int32_t ng = 0;               // distinct source distance ratios
  int32_t *grp_off = nullptr;   // [ng+1] sources of ratio group g: grp_src[grp_off[g] .. grp_off[g+1]-1]
  int32_t *grp_src = nullptr;   // [nsrc]
  double *grp_ratio = nullptr;  // [ng]
  float *grp_ratio32 = nullptr; // [ng] the same rounded to FP32 (image search)
  std::vector<GridCache> grids;
  size_t bytes = 0;
  // members' scaling cache: the static sums at f_b = 1 and nodes Chebyshev
  // points of f_t in [ft_min, ft_max] ([nodes][nimg][5]), or none
  double *scale_cache = nullptr;
  double *scale_x = nullptr;    // [nodes] the f_t points
  int32_t scale_nodes = 0;
  double ft_min = 0.0, ft_max = 0.0;
};

}  // namespace lens

struct lens_ctx {
  int device = 0;
  size_t budget = 0, used = 0;
  double fp64_threshold = 5.0;
  // LENS_MIXED deflection / Hessian maps: a node is recomputed in
  // double-float where |alpha| < repair_ratio x the summed magnitude of its
  // FP32 terms (0: never)
  double repair_ratio = LENS_REPAIR_RATIO_DEFAULT;
  int64_t next_id = 1;
  std::vector<std::pair<int64_t, lens::Model *>> models;
  std::vector<std::pair<int64_t, lens::CSet *>> csets;
  int *d_err = nullptr;          // device-side error word (bounded waits)
  // Device memory comes from a memory pool of the context's own, in stream
  // order: long-lived blocks (models, constraint sets, caches) are allocated
  // on alloc_st and freed on release_st once the work the context enqueued
  // before the release has finished (release_st waits on the marks below:
  // the GPU waits, the host and the other streams do not); a call's working
  // memory is allocated and freed on the call's own stream, so calls on
  // different streams never share it.
  cudaMemPool_t pool = nullptr;
  cudaStream_t alloc_st = nullptr, release_st = nullptr;
  // one event per stream the context has launched work on, recorded after
  // the latest such launch
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> marks;
  uint64_t mark_gen = 0, release_gen = 0;  // marks recorded / marks release_st has waited for
  // maps streamed to host memory: two device row-band buffers, two compute
  // streams and a copy stream (created on first use)
  void *band = nullptr;
  size_t band_bytes = 0;
  // released model blocks kept for reuse, and the page-locked staging
  // buffer of model uploads
  std::vector<std::pair<void *, size_t>> block_cache;
  size_t cached_bytes = 0;
  void *h_stage = nullptr;
  size_t h_stage_bytes = 0;
  cudaStream_t upload_st = nullptr;  // model uploads (record building on the device)
  cudaStream_t pipe_cs[2] = {nullptr, nullptr}, pipe_cp = nullptr;
  cudaEvent_t pipe_start = nullptr, pipe_done[2] = {nullptr, nullptr}, pipe_copied[2] = {nullptr, nullptr};
};

namespace lens {

// Thread-local last error message.
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);
#define LENS_CUDA_TRY(call)                                                                              \
  do {                                                                                                   \
    cudaError_t e__ = (call);                                                                            \
    if (e__ != cudaSuccess) return ::lens::fail(LENS_ECUDA, "%s: %s", #call, cudaGetErrorString(e__));   \
  } while (0)

Model *find_model(lens_ctx *ctx, lens_model_t id);
CSet *find_cset(lens_ctx *ctx, lens_cset_t id);
int dev_alloc(lens_ctx *ctx, void **p, size_t bytes);
// Frees p once every launch the context has enqueued so far has finished
// (stream-ordered; never blocks the host or other streams).
void dev_free(lens_ctx *ctx, void *p, size_t bytes);
// Records that the context enqueued work on st (no-op while st captures a
// graph: a graph's launches happen when the caller replays it).
void mark_stream(lens_ctx *ctx, cudaStream_t st);
// Makes st wait for every launch the context has enqueued so far.
void wait_marks(lens_ctx *ctx, cudaStream_t st);
// The context's upload stream (created on first use; NULL if that fails):
// model records and the constraint sets' caches are built on it.
cudaStream_t upload_stream(lens_ctx *ctx);
// Working memory of one call, in stream order on the call's stream: freed
// (on that stream, after the call's launches) when the object goes.
struct CallScratch {
  lens_ctx *ctx;
  cudaStream_t st;
  void *p = nullptr;
  size_t bytes = 0;
  CallScratch(lens_ctx *c, cudaStream_t s) : ctx(c), st(s) {}
  int alloc(size_t n);
  ~CallScratch();
  CallScratch(const CallScratch &) = delete;
  CallScratch &operator=(const CallScratch &) = delete;
};
// Marks the stream when the entry point returns (see mark_stream).
struct StreamMark {
  lens_ctx *ctx;
  cudaStream_t st;
  StreamMark(lens_ctx *c, cudaStream_t s) : ctx(c), st(s) {}
  ~StreamMark() { mark_stream(ctx, st); }
};
int build_model(lens_ctx *ctx, const lens_halo *h, int32_t n, Model **out);
void free_model(lens_ctx *ctx, Model *m);
int check_grid(const lens_grid *g);

// Kernel launchers (lens_maps.cu / lens_chi2.cu).
// Maps of grid rows [row0, row0 + rows) (rows < 0: to the last row) into
// out[planes][rows][nx]; the positions are those of the full grid.
// repair: recompute in double-float the nodes where FP32 cancellation
// leaves too few significant digits (working memory on st; off for the
// image search's static deflection, which must allocate nothing there).
// repair_mem: memory for the repair list (map_repair_bytes), else working
// memory of the call.
int launch_map_mixed(lens_ctx *ctx, const Model *m, const lens_grid *g, double dls, bool hess, void *out,
                     cudaStream_t st, int row0 = 0, int rows = -1, bool repair = true, void *repair_mem = nullptr);
size_t map_repair_bytes(const lens_grid *g, int rows = -1);
int launch_map_fp64(lens_ctx *ctx, const Model *m, const lens_grid *g, double dls, bool hess, void *out,
                    cudaStream_t st, int row0 = 0, int rows = -1);
int map_tile_rows(bool hess);  // rows per CTA tile of the mixed map kernel
// potential map (and, when beta is not NULL, the Fermat potential about beta)
int launch_pot_map(lens_ctx *ctx, const Model *m, const lens_grid *g, double dls, int32_t precision,
                   const double *beta, void *out, cudaStream_t st);
int launch_wait_selftest(lens_ctx *ctx, unsigned polls, cudaStream_t st);
int launch_math_selftest(const double *x, int n, double *out, cudaStream_t st);
int launch_mcmc_step(lens_ctx *ctx, const Model *m, const CSet *c, double *d_params, double *d_chi2, int32_t W,
                     const double *d_sigma, double temperature, unsigned long long seed, unsigned long long step,
                     int32_t variant, int32_t np, double *d_scratch, int32_t *d_accepted, cudaStream_t st,
                     unsigned long long *d_step = nullptr);
int build_static_cache(lens_ctx *ctx, const Model *m, CSet *c);
int launch_chi2_source(lens_ctx *ctx, const Model *m, const CSet *c, const double *d_params, int32_t P,
                       int32_t variant, double *d_chi2, cudaStream_t st);
size_t chi2_nocache_scratch_bytes(const CSet *c);
int launch_chi2_source_scaled(lens_ctx *ctx, const Model *m, const CSet *c, const double *d_params, int32_t P,
                              int32_t variant, double *d_chi2, cudaStream_t st);
int build_scaling_cache(lens_ctx *ctx, const Model *m, CSet *c, const double *d_nodes16, int32_t nodes);
int launch_chi2_source_nocache(lens_ctx *ctx, const Model *m, const CSet *c, const double *d_params, int32_t P,
                               int32_t variant, double *d_chi2, cudaStream_t st);
int autotune_chi2_source(lens_ctx *ctx, CSet *c, const double *d_params, int32_t P, double *d_chi2, cudaStream_t st,
                         int32_t *chosen, float *best_ms);
int launch_chi2_image(lens_ctx *ctx, const Model *m, CSet *c, const lens_grid *g, const double *d_params, int32_t P,
                      double *d_chi2, int32_t *d_nfound, cudaStream_t st, double *d_images = nullptr,
                      int32_t img_max = 0, int32_t *d_img_count = nullptr);
// lists = false: the smaller scratch of the single-kernel refinement
size_t chi2_image_scratch_bytes(const CSet *c, int32_t batch, bool lists = true);
// Limits of the image-plane chi2 kernels: sources per constraint set (the
// image search keeps every source of a distance group in fixed shared
// arrays) and the dynamic shared memory of the back-trace kernel.
constexpr int32_t IMG_MAX_SRC = 1024;
constexpr size_t IMG_SRC_SMEM_MAX = 200 * 1024;
// LENS_OK when constraint set c and grid g are within those limits (and the
// grid's triangle count fits the search's 32-bit cell indices); every path
// into run_chi2_image checks this before anything is launched.
int check_chi2_image_limits(const CSet *c, const lens_grid *g);
const GridCache *find_grid_cache(const CSet *c, const lens_grid *g);
int build_grid_cache(lens_ctx *ctx, CSet *c, const lens_grid *g, cudaStream_t st);
int run_chi2_image(lens_ctx *ctx, CSet *c, const GridCache *gc, const double *d_params, int32_t P,
                   double *d_chi2, int32_t *d_nfound, void *scratch, int32_t batch, cudaStream_t st,
                   double *d_images = nullptr, int32_t img_max = 0, int32_t *d_img_count = nullptr,
                   bool lists = true);

// device error word bits (read and cleared by lens_wait)
constexpr int ERRBIT_WAIT = 1;
constexpr int ERRBIT_CAPACITY = 2;

}  // namespace lens
