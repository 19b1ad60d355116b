// Batched chi2 of multiple-image constraints (Sec. 2.2, Eq. 6, Fig. 3).
//
// Static cache: when a constraint set is bound to a model, the FP64
// deflection and Hessian of every potential except the two varying ones are
// summed at each constraint position once (one CTA per image, deterministic
// tree reduction).  A parameter set then costs two FP64 potential
// evaluations per image instead of N.
//
// Source-plane kernel: persistent CTAs loop over parameter sets; per set the
// CTA rebuilds the two varying potentials, back-traces every image
// (beta = theta - r alpha, Sec. 2.1 Eq. 1), forms each source's barycentre
// and reduces the chi2 with warp shuffles in a fixed order.
//
// No-cache form: the static sum is recomputed for every parameter set (a
// batch of sets at a time, into scratch memory, in double-float) before the
// same source-plane kernel runs; this is the per-set cost when any potential
// may vary, as in the paper's fit, where every potential is evaluated for
// every model.
//
// The two varying potentials are evaluated in double-float (FP32 pipe,
// ~1e-13 relative), FP64 only where that fails; the static cache itself is
// FP64.
// The double-float division as a called function in this file's kernels:
// smaller code for the source-plane kernel, whose warps stall on
// instruction fetch (4096 sets: 0.373 -> 0.359 ms); the image-plane and map
// kernels keep it inlined (slower called: 12.56 -> 12.68 ms, 10.035 -> 10.055 ms).
#ifndef LENS_DF_NOINLINE_DIV
#define LENS_DF_NOINLINE_DIV 1
#endif
#include "lens_device.cuh"

namespace lens {
namespace {

constexpr int CACHE_THREADS = 128;
constexpr int NOCACHE_BATCH = 512;  // parameter sets per batch of the no-cache form

// grid (nimg, copies): copy c of the sums goes to stat + c * nimg * 5
__global__ void __launch_bounds__(CACHE_THREADS) k_static_cache(const double *__restrict__ all64, int n, int v0,
                                                                int v1, const double *__restrict__ x,
                                                                const double *__restrict__ y, double *stat) {
  __shared__ double s_red[(CACHE_THREADS / 32) * 5];
  const int img = blockIdx.x;
  stat += (size_t)blockIdx.y * gridDim.x * 5;
  const double X = x[img], Y = y[img];
  double v[5] = {0, 0, 0, 0, 0};
  for (int h = threadIdx.x; h < n; h += CACHE_THREADS) {
    if (h == v0 || h == v1) continue;
    double ax, ay, k, g1, g2;
    eval64<true>(all64 + (size_t)h * REC64, X, Y, ax, ay, k, g1, g2);
    v[0] += ax;
    v[1] += ay;
    v[2] += k;
    v[3] += g1;
    v[4] += g2;
  }
  block_sum<5, CACHE_THREADS>(v, s_red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) stat[(size_t)img * 5 + k] = v[k];
}

struct Chi2SrcArgs {
  const double *stat, *x, *y, *isig2, *ratio, *params;
  long long stat_stride;  // doubles between the static sums of consecutive sets (0: one shared cache)
  int pstride;            // doubles per parameter set (14; 16 with the members' scaling factors)
  const int32_t *img_off, *src_of;
  int nsrc, nimg, P, variant;
  int type0, type1;
  double *chi2;
};

// Parameter sets whose varying potentials' records one warp builds at a
// time (one thread per record: the FP64 record arithmetic runs 32 lanes wide
// instead of on two threads per set).
constexpr int SRC_BATCH = 16;

// resident warps per SM the source-plane kernel is compiled for (0: as its
// registers allow, 118 at 128 threads; 20 warps: 96 registers and spills,
// same speed; 24: 80 registers, 5 % slower)
#ifndef LENS_SRC_WARPS
#define LENS_SRC_WARPS 0
#endif
// both records of varying potential v of a parameter set, out of line
__device__ __noinline__ bool var_recs_cold(const double *q, int type0, int type1, int v, double *s_rec,
                                           float2 *s_rdf) {
  const double *w = q + 7 * v;
  const bool ok = load_var_rec64(q, type0, type1, v, s_rec);
  make_recdf(v == 0 ? type0 : type1, w[0], w[1], w[3], w[2], w[4], w[5], w[6], s_rdf + v * RECDF);
  return ok;
}

// One kernel per Hessian mode (LENS_SRC_SPLIT): HESS = 1 for the variants
// that need the Hessian, 0 for the plain residuals (72 registers instead of
// 118: 0.241 -> 0.230 ms per 4096 sets; the Hessian variants unchanged);
// -1: one kernel for all, the variant chosen at run time.
#ifndef LENS_SRC_SPLIT
#define LENS_SRC_SPLIT 1
#endif
template <int THREADS, int HESS = -1>
__global__ void __launch_bounds__(THREADS, LENS_SRC_WARPS * 32 / THREADS) k_chi2_source(const Chi2SrcArgs a) {
  static_assert(THREADS >= 2 * SRC_BATCH, "one thread per record of a batch");
  extern __shared__ double sm[];
  double *s_beta = sm;                   // [nimg][2]
  double *s_m = s_beta + 2 * a.nimg;     // [nimg][3]: r hxx, r hyy, r hxy
  double *s_bary = s_m + 3 * a.nimg;     // [nsrc][2]
  double *s_red = s_bary + 2 * a.nsrc;   // [THREADS/32]
  __shared__ double s_rec[SRC_BATCH][2 * REC64];   // FP64 records of the batch's varying potentials
  __shared__ float2 s_rdf[SRC_BATCH][2 * RECDF];   // the same in double-float
  __shared__ int s_ok[SRC_BATCH][2];
  // this CTA's sets are p = blockIdx.x + j gridDim.x, taken SRC_BATCH at a time
  for (long long p0 = blockIdx.x; p0 < a.P; p0 += (long long)gridDim.x * SRC_BATCH) {
    __syncthreads();  // the previous batch's records are no longer read
    if (threadIdx.x < 2 * SRC_BATCH) {
      const int k = threadIdx.x >> 1, v = threadIdx.x & 1;
      const long long p = p0 + (long long)k * gridDim.x;
      if (p < a.P) {
        const double *q = a.params + p * a.pstride;
        const double *w = q + 7 * v;  // x0, y0, eps, theta, rcore, rcut, b0
        if (LENS_COLD_CALLS) {
          s_ok[k][v] = var_recs_cold(q, a.type0, a.type1, v, s_rec[k], s_rdf[k]);
        } else {
          s_ok[k][v] = load_var_rec64(q, a.type0, a.type1, v, s_rec[k]);
          make_recdf(v == 0 ? a.type0 : a.type1, w[0], w[1], w[3], w[2], w[4], w[5], w[6], s_rdf[k] + v * RECDF);
        }
      }
    }
    __syncthreads();
    for (int k = 0; k < SRC_BATCH; ++k) {
      const long long p = p0 + (long long)k * gridDim.x;
      if (p >= a.P) break;  // uniform over the CTA
      if (!(s_ok[k][0] && s_ok[k][1])) {
        if (threadIdx.x == 0) a.chi2[p] = __longlong_as_double(0x7ff8000000000000ll);
        continue;
      }
      const bool hess = HESS < 0 ? a.variant != LENS_CHI2_SRC_PLAIN : HESS == 1;
      backtrace_set<THREADS, HESS>(a.stat + p * a.stat_stride, a.x, a.y, a.ratio, a.src_of, a.img_off, a.nimg,
                                   a.nsrc, s_rec[k], s_rdf[k], s_beta, hess ? s_m : nullptr, s_bary);
      double acc[1] = {0.0};
      for (int j = threadIdx.x; j < a.nimg; j += THREADS) {
        const int i = a.src_of[j];
        const double dbx = s_bary[2 * i] - s_beta[2 * j], dby = s_bary[2 * i + 1] - s_beta[2 * j + 1];
        const double is2 = a.isig2[j];
        if (a.variant == LENS_CHI2_SRC_PLAIN) {
          acc[0] += (dbx * dbx + dby * dby) * is2;
        } else {
          // A^-1 = I - r H (Sec. 2.1 Eq. 4)
          const double a11 = 1.0 - s_m[3 * j], a22 = 1.0 - s_m[3 * j + 1], a12 = -s_m[3 * j + 2];
          const double det = a11 * a22 - a12 * a12;
          const double id = det != 0.0 ? rcp64(det) : 1.0 / det;
          if (a.variant == LENS_CHI2_SRC_MU) {
            acc[0] += (dbx * dbx + dby * dby) * fabs(id) * is2;
          } else {
            const double rx = (a22 * dbx - a12 * dby) * id, ry = (a11 * dby - a12 * dbx) * id;
            acc[0] += (rx * rx + ry * ry) * is2;
          }
        }
      }
      block_sum<1, THREADS>(acc, s_red);
      if (threadIdx.x == 0) a.chi2[p] = acc[0];
    }
  }
}

}  // namespace

// Synchronous on the context's upload stream (no other stream waits).
int build_static_cache(lens_ctx *ctx, const Model *m, CSet *c) {
  cudaStream_t st = upload_stream(ctx);
  if (!st) return fail(LENS_ECUDA, "upload stream creation failed");
  k_static_cache<<<c->nimg, CACHE_THREADS, 0, st>>>(m->all64, m->n, c->var[0], c->var[1], c->x, c->y, c->stat);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(LENS_ECUDA, "static cache: %s", cudaGetErrorString(e));
  return LENS_OK;
}

template <int T>
static int launch_src_cfg(lens_ctx *ctx, const CSet *c, const double *d_params, int32_t P, int32_t variant,
                          double *d_chi2, cudaStream_t st, int blocks_per_sm, const double *stat = nullptr,
                          long long stat_stride = 0, int pstride = 14) {
  const size_t smem = sizeof(double) * (5 * (size_t)c->nimg + 2 * (size_t)c->nsrc + T / 32);
  if (smem > 200 * 1024) return fail(LENS_EINVAL, "constraint set too large for one CTA (%d images)", c->nimg);
  const int H = LENS_SRC_SPLIT ? (variant == LENS_CHI2_SRC_PLAIN ? 0 : 1) : -1;
  auto kern = H < 0 ? k_chi2_source<T, -1> : H == 0 ? k_chi2_source<T, 0> : k_chi2_source<T, 1>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  int per_sm = 0, nsm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  per_sm = std::max(1, per_sm);
  if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
  const int blocks = std::max(1, std::min(P, per_sm * nsm));
  Chi2SrcArgs a;
  a.stat = stat ? stat : c->stat;
  a.stat_stride = stat_stride;
  a.x = c->x;
  a.y = c->y;
  a.isig2 = c->isig2;
  a.ratio = c->ratio;
  a.params = d_params;
  a.pstride = pstride;
  a.img_off = c->img_off;
  a.src_of = c->src_of;
  a.nsrc = c->nsrc;
  a.nimg = c->nimg;
  a.P = P;
  a.variant = variant;
  a.type0 = c->var_type[0];
  a.type1 = c->var_type[1];
  a.chi2 = d_chi2;
  kern<<<blocks, T, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "chi2 source launch: %s", cudaGetErrorString(e));
  return LENS_OK;
}

// Launch shapes the autotuner chooses from: threads per CTA x CTAs per SM
// (0 = as many as fit).
static const int SRC_CFG[][2] = {{64, 0}, {64, 8}, {128, 0}, {128, 4}, {128, 2}, {256, 0}, {256, 2}, {256, 1}};
constexpr int N_SRC_CFG = sizeof(SRC_CFG) / sizeof(SRC_CFG[0]);

static int launch_src_idx(lens_ctx *ctx, const CSet *c, const double *d_params, int32_t P, int32_t variant,
                          double *d_chi2, cudaStream_t st, int idx) {
  const int t = SRC_CFG[idx][0], b = SRC_CFG[idx][1];
  if (t == 64) return launch_src_cfg<64>(ctx, c, d_params, P, variant, d_chi2, st, b);
  if (t == 256) return launch_src_cfg<256>(ctx, c, d_params, P, variant, d_chi2, st, b);
  return launch_src_cfg<128>(ctx, c, d_params, P, variant, d_chi2, st, b);
}

int launch_chi2_source(lens_ctx *ctx, const Model *m, const CSet *c, const double *d_params, int32_t P,
                       int32_t variant, double *d_chi2, cudaStream_t st) {
  (void)m;
  const int idx = (c->tuned_cfg >= 0 && c->tuned_cfg < N_SRC_CFG) ? c->tuned_cfg : 2;
  return launch_src_idx(ctx, c, d_params, P, variant, d_chi2, st, idx);
}

// Static sums of the no-cache form, grid (nimg, sets): every static potential
// at the image in double-float (FP64 where that fails), per-thread sums in
// double-float, deterministic CTA reduction in FP64; copy c goes to
// stat + c * nimg * 5.
__global__ void __launch_bounds__(CACHE_THREADS) k_static_df(const float2 *__restrict__ recdf,
                                                             const double *__restrict__ all64, int n, int v0, int v1,
                                                             const double *__restrict__ x,
                                                             const double *__restrict__ y, double *stat) {
  __shared__ double s_red[(CACHE_THREADS / 32) * 5];
  const int img = blockIdx.x;
  stat += (size_t)blockIdx.y * gridDim.x * 5;
  const double X = x[img], Y = y[img];
  const df Xd = df_from_double(X), Yd = df_from_double(Y);
  double v[5] = {0, 0, 0, 0, 0};
  // per-thread sums in double-float, converted once (FP64 only for the
  // potentials whose double-float evaluation fails)
  df sum[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int h = threadIdx.x; h < n; h += CACHE_THREADS) {
    if (h == v0 || h == v1) continue;
    const float2 *r = recdf + h;
    df ax, ay, hh[3];
    bool ok = true;
    if (r[F_U2 * n].x < 0.f)
      circ_df<true>(r, n, Xd, Yd, ax, ay, hh);
    else
      ok = dpie_df<true, true>(r, n, Xd, Yd, ax, ay, hh);
    if (ok) {
      sum[0] = df_add(sum[0], ax);
      sum[1] = df_add(sum[1], ay);
      sum[2] = df_add(sum[2], hh[0]);
      sum[3] = df_add(sum[3], hh[1]);
      sum[4] = df_add(sum[4], hh[2]);
    } else {
      double e[5] = {0, 0, 0, 0, 0};
      eval64<true>(all64 + (size_t)h * REC64, X, Y, e[0], e[1], e[2], e[3], e[4]);
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] += e[k];
    }
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) v[k] += df_to_double(sum[k]);
  block_sum<5, CACHE_THREADS>(v, s_red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) stat[(size_t)img * 5 + k] = v[k];
}

size_t chi2_nocache_scratch_bytes(const CSet *c) { return (size_t)NOCACHE_BATCH * c->nimg * 5 * sizeof(double); }

int launch_chi2_source_nocache(lens_ctx *ctx, const Model *m, const CSet *c, const double *d_params, int32_t P,
                               int32_t variant, double *d_chi2, cudaStream_t st) {
  CallScratch scratch(ctx, st);  // the static sums of a batch, on this call's stream
  int rc0 = scratch.alloc(chi2_nocache_scratch_bytes(c));
  if (rc0) return rc0;
  double *stat = (double *)scratch.p;
  for (int32_t p0 = 0; p0 < P; p0 += NOCACHE_BATCH) {
    const int B = std::min(NOCACHE_BATCH, P - p0);
    k_static_df<<<dim3(c->nimg, B), CACHE_THREADS, 0, st>>>(m->recdf, m->all64, m->n, c->var[0], c->var[1], c->x,
                                                             c->y, stat);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LENS_ECUDA, "static sums launch: %s", cudaGetErrorString(e));
    const int rc = launch_src_cfg<128>(ctx, c, d_params + (size_t)p0 * 14, B, variant, d_chi2 + p0, st, 0, stat,
                                       (long long)c->nimg * 5);
    if (rc) return rc;
  }
  return LENS_OK;
}

// Static sums with the members' scaling relations applied, grid (nimg, sets):
// every static potential's b0 times f_b = params[14] and every static dPIE's
// r_cut times f_t = params[15] (b0_i = b0* s_i, r_cut,i = r_cut* s_i: varying
// b0* and r_cut*).  The sum is linear in b0, so f_b scales the result; the
// r_cut-dependent fields of each double-float record are rebuilt from
// st' = f_t st in double-float (q^2 st', q^2 st'^2, (1+q^2) st'^2, u^2 st'^2,
// st' + sc, q^2 (st' +- sc), q^2 (st'^2 - sc^2)).  FP64 (a record rescaled the
// same way) where the double-float evaluation fails.  Outside the domain
// (f_b <= 0, f_t r_cut,i <= r_core,i) the set's sums are NaN.
__global__ void __launch_bounds__(CACHE_THREADS) k_static_scaled(const float2 *__restrict__ recdf,
                                                                 const double *__restrict__ all64, int n, int v0,
                                                                 int v1, const double *__restrict__ x,
                                                                 const double *__restrict__ y,
                                                                 const double *__restrict__ params, double *stat) {
  __shared__ double s_red[(CACHE_THREADS / 32) * 5];
  const int img = blockIdx.x;
  stat += (size_t)blockIdx.y * gridDim.x * 5;
  const double fb = params[(size_t)blockIdx.y * 16 + 14], ft = params[(size_t)blockIdx.y * 16 + 15];
  const double X = x[img], Y = y[img];
  const df Xd = df_from_double(X), Yd = df_from_double(Y), fd = df_from_double(ft), f2 = df_mul(fd, fd);
  double v[5] = {0, 0, 0, 0, 0};
  df sum[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  bool bad = !(fb > 0.0 && ft > 0.0 && isfinite(fb) && isfinite(ft));
  for (int h = threadIdx.x; h < n && !bad; h += CACHE_THREADS) {
    if (h == v0 || h == v1) continue;
    const float2 *g = recdf + h;
    df ax, ay, hh[3];
    bool ok = true;
    if (g[F_U2 * n].x < 0.f) {
      circ_df<true>(g, n, Xd, Yd, ax, ay, hh);
    } else {
      float2 r[RECDF];
#pragma unroll
      for (int k = 0; k < RECDF; ++k) r[k] = g[k * n];
      auto D = [&](int k) { return df{r[k].x, r[k].y}; };
      auto put = [&](int k, df d) { r[k] = make_float2(d.hi, d.lo); };
      const df st = df_mul(D(F_ST), fd), sc = D(F_SC), q2st = df_mul(D(F_Q2ST), fd);
      const df ss = df_add_ss(st, sc), q2ds = df_sub(q2st, D(F_Q2SC));
      if (!(st.hi > sc.hi)) bad = true;  // r_cut' <= r_core
      put(F_ST, st);
      put(F_Q2ST, q2st);
      put(F_SS, ss);
      put(F_Q2SS, df_add_ss(q2st, D(F_Q2SC)));
      put(F_Q2DS, q2ds);
      put(F_KT, df_mul(D(F_KT), f2));
      put(F_DT0, df_mul(D(F_DT0), f2));
      put(F_U2ST2, df_mul(D(F_U2ST2), f2));
      put(F_KTC, df_mul(q2ds, ss));
      ok = dpie_df<true, true>(r, 1, Xd, Yd, ax, ay, hh);
    }
    if (ok) {
      sum[0] = df_add(sum[0], ax);
      sum[1] = df_add(sum[1], ay);
      sum[2] = df_add(sum[2], hh[0]);
      sum[3] = df_add(sum[3], hh[1]);
      sum[4] = df_add(sum[4], hh[2]);
    } else {
      double q[REC64], e[5] = {0, 0, 0, 0, 0};
      for (int k = 0; k < REC64; ++k) q[k] = all64[(size_t)h * REC64 + k];
      q[D_ST] *= ft;
      q[D_DS] = q[D_ST] - q[D_SC];
      q[D_SS] = q[D_ST] + q[D_SC];
      eval64<true>(q, X, Y, e[0], e[1], e[2], e[3], e[4]);
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] += e[k];
    }
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) v[k] = fb * (v[k] + df_to_double(sum[k]));
  const int any_bad = __syncthreads_or(bad);
  block_sum<5, CACHE_THREADS>(v, s_red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) stat[(size_t)img * 5 + k] = any_bad ? __longlong_as_double(0x7ff8000000000000ll) : v[k];
}

// Static sums of each set from the scaling cache, grid (sets of the batch):
// the barycentric Chebyshev interpolant in f_t of the cached sums (second
// kind points xs with weights (-1)^k, halved at both ends: Berrut and
// Trefethen, "Barycentric Lagrange interpolation", SIAM Review 2004), times
// f_b; NaN for f_t outside the cached interval or f_b not positive.
constexpr int MAX_SCALE_NODES = 128;
__global__ void __launch_bounds__(CACHE_THREADS) k_scaled_interp(const double *__restrict__ cache,
                                                                 const double *__restrict__ xs, int nodes,
                                                                 double ft_min, double ft_max, int nimg,
                                                                 const double *__restrict__ params, double *stat) {
  __shared__ double s_w[MAX_SCALE_NODES];
  __shared__ int s_hit;
  const double fb = params[(size_t)blockIdx.x * 16 + 14], ft = params[(size_t)blockIdx.x * 16 + 15];
  stat += (size_t)blockIdx.x * nimg * 5;
  const bool ok = fb > 0.0 && isfinite(fb) && ft >= ft_min && ft <= ft_max;
  if (threadIdx.x == 0) s_hit = -1;
  __syncthreads();
  for (int k = threadIdx.x; k < nodes; k += CACHE_THREADS) {
    const double xk = xs[k];
    const double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == nodes - 1) ? 0.5 : 1.0);
    if (ft == xk) s_hit = k;
    s_w[k] = wk / (ft - xk);
  }
  __syncthreads();
  const int hit = s_hit;
  double den = 0.0;
  if (hit < 0)
    for (int k = 0; k < nodes; ++k) den += s_w[k];
  const double iden = hit < 0 ? 1.0 / den : 0.0;
  for (int j = threadIdx.x; j < nimg; j += CACHE_THREADS) {
    double v[5];
    if (hit >= 0) {
#pragma unroll
      for (int q = 0; q < 5; ++q) v[q] = cache[((size_t)hit * nimg + j) * 5 + q];
    } else {
      double num[5] = {0, 0, 0, 0, 0};
      for (int k = 0; k < nodes; ++k) {
        const double w = s_w[k];
#pragma unroll
        for (int q = 0; q < 5; ++q) num[q] = fma(w, cache[((size_t)k * nimg + j) * 5 + q], num[q]);
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) v[q] = num[q] * iden;
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) stat[(size_t)j * 5 + q] = ok ? fb * v[q] : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// Synchronous on the context's upload stream.
int build_scaling_cache(lens_ctx *ctx, const Model *m, CSet *c, const double *d_nodes16, int32_t nodes) {
  cudaStream_t st = upload_stream(ctx);
  if (!st) return fail(LENS_ECUDA, "upload stream creation failed");
  k_static_scaled<<<dim3(c->nimg, nodes), CACHE_THREADS, 0, st>>>(m->recdf, m->all64, m->n, c->var[0], c->var[1],
                                                                  c->x, c->y, d_nodes16, c->scale_cache);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(LENS_ECUDA, "scaling cache: %s", cudaGetErrorString(e));
  return LENS_OK;
}

int launch_chi2_source_scaled(lens_ctx *ctx, const Model *m, const CSet *c, const double *d_params, int32_t P,
                              int32_t variant, double *d_chi2, cudaStream_t st) {
  CallScratch scratch(ctx, st);  // the static sums of a batch, on this call's stream
  int rc0 = scratch.alloc(chi2_nocache_scratch_bytes(c));
  if (rc0) return rc0;
  double *stat = (double *)scratch.p;
  for (int32_t p0 = 0; p0 < P; p0 += NOCACHE_BATCH) {
    const int B = std::min(NOCACHE_BATCH, P - p0);
    if (c->scale_cache)
      k_scaled_interp<<<B, CACHE_THREADS, 0, st>>>(c->scale_cache, c->scale_x, c->scale_nodes, c->ft_min,
                                                    c->ft_max, c->nimg, d_params + (size_t)p0 * 16, stat);
    else
      k_static_scaled<<<dim3(c->nimg, B), CACHE_THREADS, 0, st>>>(m->recdf, m->all64, m->n, c->var[0], c->var[1],
                                                                   c->x, c->y, d_params + (size_t)p0 * 16, stat);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LENS_ECUDA, "scaled static sums launch: %s", cudaGetErrorString(e));
    const int rc = launch_src_cfg<128>(ctx, c, d_params + (size_t)p0 * 16, B, variant, d_chi2 + p0, st, 0, stat,
                                       (long long)c->nimg * 5, 16);
    if (rc) return rc;
  }
  return LENS_OK;
}

// Time every launch shape on this constraint set and P (each once to warm
// up, then best of 3), keep the fastest.  Synchronous on st.
int autotune_chi2_source(lens_ctx *ctx, CSet *c, const double *d_params, int32_t P, double *d_chi2, cudaStream_t st,
                         int32_t *chosen, float *best_ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(LENS_ECUDA, "event creation failed");
  int best = -1;
  float best_t = 1e30f;
  int rc = LENS_OK;
  for (int k = 0; k < N_SRC_CFG && rc == LENS_OK; ++k) {
    rc = launch_src_idx(ctx, c, d_params, P, 0, d_chi2, st, k);
    for (int r = 0; r < 3 && rc == LENS_OK; ++r) {
      cudaEventRecord(e0, st);
      rc = launch_src_idx(ctx, c, d_params, P, 0, d_chi2, st, k);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(LENS_ECUDA, "autotune timing failed");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == LENS_OK && ms < best_t) {
        best_t = ms;
        best = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  c->tuned_cfg = best;
  if (chosen) *chosen = SRC_CFG[best][0] * 100 + SRC_CFG[best][1];
  if (best_ms) *best_ms = best_t;
  return LENS_OK;
}

}  // namespace lens
