// Image-plane chi2 with brute-force image finding (Sec. 2.2 Eq. 6; Sec. 2.3,
// Fig. 4; Sec. 4.2, Fig. 8), batched over parameter sets.
//
// Per batch of parameter sets, six launches on the caller's stream:
//   1. k_img_sources  per set: back-trace the constraints in FP64 and form
//                     each source's barycentre (the source estimate).
//   2. k_img_search   per (grid tile, set): deflection at the tile's nodes =
//                     cached static part + the two varying potentials (FP32);
//                     for each distance ratio the nodes are mapped to the
//                     source plane, the sources inside the tile's footprint
//                     (bounding box of its mapped nodes) are listed, and both
//                     triangles of every cell are tested against that list
//                     (bounding box, then barycentric weights with a small
//                     tolerance so that a source on a shared edge is never
//                     lost); every hit is appended to the set's buffer.
//   3. k_img_newton   one group of RF_G threads per candidate: the hit
//                     triangle is subdivided up to SUBDIV_LEVELS times
//                     (keeping the sub-triangle that best contains the source;
//                     stopping early when none does), then Newton on the lens
//                     equation, steps limited to one cell, starts there; full
//                     model with the group splitting the potentials (FP32,
//                     cluster-scale static ones in FP64); a root further than
//                     LOCAL_CELLS cells from its triangle is dropped.
//   4. k_img_dedup    per set: candidates of the same source closer than
//                     1e-3" are one image.
//   5. k_img_polish   one warp per distinct image: Newton steps whose residual
//                     uses the full model in double-float (FP64 for cores,
//                     SIS and point masses) until the step is < 1e-6", the
//                     stopping rule of the definition's FP64 Newton.
//   6. k_img_chi2     per set: polished images of one source closer than
//                     1e-3" are merged again (as after the definition's FP64
//                     Newton); each constraint takes the nearest image of its
//                     own source (ties: lower y, then lower x); chi2 reduced in
//                     a fixed order.
// Candidate buffers live in scratch memory (IMG_CAP per set); an overflow
// makes that set's chi2 NaN and sets ERRBIT_CAPACITY.
#include <type_traits>

#include "lens_device.cuh"

namespace lens {
namespace {

constexpr int IMG_CAP = 4096;       // candidate images per parameter set
constexpr int IMG_BATCH = 256;      // parameter sets per batch
constexpr int MAX_SRC = IMG_MAX_SRC;
constexpr double DEDUP = 1e-3;      // images closer than this are one image (arcsec)
constexpr double NEWTON32_TOL = 1e-4;
constexpr double POLISH_TOL = 1e-6;  // same stopping rule as the FP64 Newton of the definition
constexpr double ACCEPT_TOL = 1e-6;
constexpr int NEWTON_MAXIT = 40, POLISH_MAXIT = 6;
constexpr float BARY_TOL = 1e-3f;
// Subdivisions of a hit triangle before Newton.  The definition refines 6
// times; from level 3 on the sub-triangles (1/8 cell and
// smaller) only move Newton's start inside the basin it already is in:
// measured on 256 parameter sets x 100 sources of the 1000-potential model,
// 2 to 6 levels find identical image sets, 1 level one extra (true) image,
// 0 levels miss a well-conditioned image.  3 keeps a margin of two levels.
#ifndef LENS_SUBDIV_LEVELS
#define LENS_SUBDIV_LEVELS 3
#endif
constexpr int SUBDIV_LEVELS = LENS_SUBDIV_LEVELS;
constexpr double SUBDIV_TOL = 1e-3;  // refinement stops when the source is this far outside every sub-triangle
constexpr double LOCAL_CELLS = 2.0;  // a root must lie this many cell sizes from its triangle
// search tile: CT_X x CT_Y cells per CTA of SEARCH_THREADS threads, each
// thread CPT cells of one column; ratio groups tested SEARCH_GCH at a time
#ifndef LENS_SEARCH_CT_Y
#define LENS_SEARCH_CT_Y 64  // 4 cells per thread: faster than 32 (4 %), 16 (6 %) and 8 (fewer barrier-separated phases per cell)
#endif
constexpr int CT_X = 32, CT_Y = LENS_SEARCH_CT_Y, NX_T = CT_X + 1, NY_T = CT_Y + 1;
constexpr int SEARCH_THREADS = 256, SEARCH_WARPS = SEARCH_THREADS / 32, SEARCH_GCH = SEARCH_WARPS;
constexpr int CPT = CT_X * CT_Y / SEARCH_THREADS;  // cells per thread
static_assert(CPT >= 1 && CT_X * CT_Y == CPT * SEARCH_THREADS, "whole cells per thread");
// Sub-tile pre-filter (LENS_SEARCH_SUBTILE): warp w's cells are the tile's
// cell rows w SUB_R .. w SUB_R + SUB_R - 1 (lane = column), and only the
// sources inside that sub-tile's own footprint are tested against them
// (1024^2 grid, 1000-potential model: 0.30 M instead of 1.13 M cell tests
// per parameter set).
#ifndef LENS_SEARCH_SUBTILE
#define LENS_SEARCH_SUBTILE 1
#endif
constexpr int SUB_R = CT_Y / SEARCH_WARPS;
static_assert(CT_X == 32 && SUB_R == CPT, "a warp's sub-tile: 32 columns x CPT rows");
// candidate status; the failures say which stage rejected it
constexpr int ST_PENDING = 0, ST_NEWTON = 1, ST_FINAL = 2, ST_FAILED = -1, ST_FAR = -2, ST_NO_POLISH = -3;

struct Hit {
  double tx, ty;       // image position
  float cx, cy;        // centroid of the hit triangle (image plane)
  float h11, h22, h12; // r H at the last FP32 Newton step
  int src;
  int status;
  int cell;            // 2 * (j * (nx-1) + i) + triangle of the hit
};

// Records of the two varying potentials of one parameter set, built once per
// set by k_img_sources: FP32 records and hi/lo centres (search, subdivision,
// FP32 Newton), double-float and FP64 records (polish).
struct __align__(16) VarRecs {
  float r32[2][REC32];
  float cen[2][4];
  float2 rdf[2][RECDF];
  double r64[2][REC64];
};

// Refinement state of a candidate (step 3, point-list form), beside its hit.
struct Ref {
  double th[3][2];  // vertices of the current (sub-)triangle
  double be[3][2];  // their images in the source plane
  double mo[6];     // evaluations: alpha at the three edge midpoints, or alpha, kappa, gamma1, gamma2 at the Newton point
  double tiny;      // degenerate-area threshold at the current level
  int nit, settled; // Newton steps taken; steps below the tolerance
};
// Point lists of step 3 (entries slot << 2 | m: m < 3 edge midpoint m of the
// slot's triangle, m = 3 its Newton point), slots per candidate slot: two
// alternating subdivision lists of 3, two Newton rounds and the stragglers.
constexpr int LST_PER_SLOT = 9;
#ifndef LENS_NEWTON_ROUNDS
#define LENS_NEWTON_ROUNDS 2  // Newton steps taken by the point-list form before the rest go to k_ref_straggle
#endif
constexpr int NEWTON_ROUNDS = LENS_NEWTON_ROUNDS;
static_assert(NEWTON_ROUNDS >= 1, "the subdivision hands its candidates to Newton round 0");
constexpr int LCNT = 16;  // list counters: subdivision levels, Newton rounds, stragglers; the last: straggler fetches
static_assert(SUBDIV_LEVELS + NEWTON_ROUNDS + 1 < LCNT, "list counters");

struct Layout {
  size_t cnt, valid, nuniq, bary, src32, hits, uniq, var, ref, lst, lcnt, total;
};

__host__ __device__ inline size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// lists = false: no point-list refinement state (step 3 then runs as
// k_img_newton, in less memory)
__host__ __device__ inline Layout layout(int B, int nsrc, bool lists = true) {
  Layout L;
  size_t o = 0;
  L.cnt = o;
  o = align_up(o + (size_t)B * sizeof(int));
  L.valid = o;
  o = align_up(o + (size_t)B * sizeof(int));
  L.nuniq = o;
  o = align_up(o + (size_t)B * sizeof(int));
  L.bary = o;
  o = align_up(o + (size_t)B * nsrc * 2 * sizeof(double));
  L.src32 = o;
  o = align_up(o + (size_t)B * nsrc * sizeof(float2));
  L.hits = o;
  o = align_up(o + (size_t)B * IMG_CAP * sizeof(Hit));
  L.uniq = o;
  o = align_up(o + (size_t)B * IMG_CAP * sizeof(int));
  L.var = o;
  o = align_up(o + (size_t)B * sizeof(VarRecs));
  L.ref = o;
  o = align_up(o + (lists ? (size_t)B * IMG_CAP * sizeof(Ref) : 0));
  L.lst = o;
  o = align_up(o + (lists ? (size_t)B * IMG_CAP * LST_PER_SLOT * sizeof(int) : 0));
  L.lcnt = o;
  o = align_up(o + LCNT * sizeof(int));
  L.total = o;
  return L;
}

struct Bufs {
  int *cnt, *valid, *nuniq, *uniq;
  double *bary;
  float2 *src32;  // barycentres rounded to FP32 (search)
  Hit *hits;
  VarRecs *var;
  Ref *ref;       // [B][IMG_CAP], beside hits
  int *lst;       // point lists, LST_PER_SLOT x B x IMG_CAP entries
  int *lcnt;      // their counters
};

__host__ __device__ inline Bufs bufs(void *scratch, int B, int nsrc, bool lists = true) {
  Layout L = layout(B, nsrc, lists);
  char *b = (char *)scratch;
  Bufs r;
  r.cnt = (int *)(b + L.cnt);
  r.valid = (int *)(b + L.valid);
  r.nuniq = (int *)(b + L.nuniq);
  r.bary = (double *)(b + L.bary);
  r.src32 = (float2 *)(b + L.src32);
  r.hits = (Hit *)(b + L.hits);
  r.uniq = (int *)(b + L.uniq);
  r.var = (VarRecs *)(b + L.var);
  r.ref = (Ref *)(b + L.ref);
  r.lst = (int *)(b + L.lst);
  r.lcnt = (int *)(b + L.lcnt);
  return r;
}

struct SetArgs {  // what every kernel needs to know about the batch
  const double *params;
  int p0, B, type0, type1;
  int nsrc, nimg;
  Bufs s;
};

// ---------------------------------------------------------------- 1. sources
constexpr int SRC_THREADS = 128;

__global__ void __launch_bounds__(SRC_THREADS) k_img_sources(const SetArgs a, const double *__restrict__ stat,
                                                             const double *__restrict__ x,
                                                             const double *__restrict__ y,
                                                             const double *__restrict__ ratio,
                                                             const int32_t *__restrict__ src_of,
                                                             const int32_t *__restrict__ img_off) {
  extern __shared__ double sm[];
  double *s_rec = sm;
  double *s_beta = s_rec + 2 * REC64;
  double *s_bary = s_beta + 2 * a.nimg;
  __shared__ int s_ok;
  const int b = blockIdx.x;
  const double *q = a.params + (size_t)(a.p0 + b) * 14;
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  if (threadIdx.x < 2) {
    if (!load_var_rec64(q, a.type0, a.type1, threadIdx.x, s_rec)) atomicAnd(&s_ok, 0);
    // every later kernel of this set reads the varying potentials from here
    VarRecs &v = a.s.var[b];
    const double *w = q + 7 * threadIdx.x;
    make_rec32(threadIdx.x == 0 ? a.type0 : a.type1, w[3], w[2], w[4], w[5], w[6], v.r32[threadIdx.x]);
    const float xh = (float)w[0], yh = (float)w[1];
    v.cen[threadIdx.x][0] = xh;
    v.cen[threadIdx.x][1] = yh;
    v.cen[threadIdx.x][2] = (float)(w[0] - (double)xh);
    v.cen[threadIdx.x][3] = (float)(w[1] - (double)yh);
    make_recdf(threadIdx.x == 0 ? a.type0 : a.type1, w[0], w[1], w[3], w[2], w[4], w[5], w[6], v.rdf[threadIdx.x]);
    for (int k = 0; k < REC64; ++k) v.r64[threadIdx.x][k] = s_rec[threadIdx.x * REC64 + k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.s.valid[b] = s_ok;
    a.s.cnt[b] = 0;
    a.s.nuniq[b] = 0;
  }
  if (!s_ok) return;
  backtrace_set<SRC_THREADS>(stat, x, y, ratio, src_of, img_off, a.nimg, a.nsrc, s_rec, &a.s.var[b].rdf[0][0], s_beta,
                             nullptr, s_bary);
  for (int i = threadIdx.x; i < 2 * a.nsrc; i += SRC_THREADS) a.s.bary[(size_t)b * a.nsrc * 2 + i] = s_bary[i];
  for (int i = threadIdx.x; i < a.nsrc; i += SRC_THREADS)
    a.s.src32[(size_t)b * a.nsrc + i] = make_float2((float)s_bary[2 * i], (float)s_bary[2 * i + 1]);
}

// ----------------------------------------------------------------- 2. search
struct SearchArgs {
  const float *ax, *ay;  // static deflection planes [ny][nx]
  double xmin, ymin, dx, dy;
  float fdx, fdy, tiny;  // FP32 cell sizes; degenerate-triangle threshold on the doubled area
  int nx, ny;
  const int32_t *grp_off, *grp_src;
  const float *grp_r32;  // ratio of each group, FP32
  int ng;
};

#if !LENS_SEARCH_SUBTILE
__device__ __forceinline__ void tri_test(float2 A, float2 Bv, float2 Cv, float2 tA, float2 tB, float2 tC,
                                         const float2 *s_src, const int *list, int nlist, float tiny, int *cnt,
                                         Hit *hits, int cell) {
  const float lox = fminf(A.x, fminf(Bv.x, Cv.x)), hix = fmaxf(A.x, fmaxf(Bv.x, Cv.x));
  const float loy = fminf(A.y, fminf(Bv.y, Cv.y)), hiy = fmaxf(A.y, fmaxf(Bv.y, Cv.y));
  const float padx = BARY_TOL * (hix - lox) + 1e-6f, pady = BARY_TOL * (hiy - loy) + 1e-6f;
  const float e1x = Bv.x - A.x, e1y = Bv.y - A.y, e2x = Cv.x - A.x, e2y = Cv.y - A.y;
  const float area2 = e1x * e2y - e1y * e2x;
  if (!(fabsf(area2) > tiny)) return;
  const float inv = 1.f / area2;
  for (int k = 0; k < nlist; ++k) {
    const int src = list[k];
    const float2 P = s_src[src];
    if (P.x < lox - padx || P.x > hix + padx || P.y < loy - pady || P.y > hiy + pady) continue;
    const float px = P.x - A.x, py = P.y - A.y;
    const float wb = (px * e2y - py * e2x) * inv, wc = (e1x * py - e1y * px) * inv, wa = 1.f - wb - wc;
    if (wa < -BARY_TOL || wb < -BARY_TOL || wc < -BARY_TOL) continue;
    const int slot = atomicAdd(cnt, 1);
    if (slot < IMG_CAP) {
      Hit *h = hits + slot;
      h->src = src;
      h->cx = (tA.x + tB.x + tC.x) * (1.f / 3.f);
      h->cy = (tA.y + tB.y + tC.y) * (1.f / 3.f);
      h->cell = cell;
      h->status = ST_PENDING;
    }
  }
}

#else
// The same for the list entries whose bits are set in mask (entry k: bit k).
__device__ __forceinline__ void tri_test_mask(float2 A, float2 Bv, float2 Cv, float2 tA, float2 tB, float2 tC,
                                              const float2 *s_src, const int *list, unsigned mask, float tiny,
                                              int *cnt, Hit *hits, int cell) {
  const float lox = fminf(A.x, fminf(Bv.x, Cv.x)), hix = fmaxf(A.x, fmaxf(Bv.x, Cv.x));
  const float loy = fminf(A.y, fminf(Bv.y, Cv.y)), hiy = fmaxf(A.y, fmaxf(Bv.y, Cv.y));
  const float padx = BARY_TOL * (hix - lox) + 1e-6f, pady = BARY_TOL * (hiy - loy) + 1e-6f;
  const float e1x = Bv.x - A.x, e1y = Bv.y - A.y, e2x = Cv.x - A.x, e2y = Cv.y - A.y;
  const float area2 = e1x * e2y - e1y * e2x;
  if (!(fabsf(area2) > tiny)) return;
  const float inv = 1.f / area2;
  for (unsigned mm = mask; mm; mm &= mm - 1u) {
    const int src = list[__ffs(mm) - 1];
    const float2 P = s_src[src];
    if (P.x < lox - padx || P.x > hix + padx || P.y < loy - pady || P.y > hiy + pady) continue;
    const float px = P.x - A.x, py = P.y - A.y;
    const float wb = (px * e2y - py * e2x) * inv, wc = (e1x * py - e1y * px) * inv, wa = 1.f - wb - wc;
    if (wa < -BARY_TOL || wb < -BARY_TOL || wc < -BARY_TOL) continue;
    const int slot = atomicAdd(cnt, 1);
    if (slot < IMG_CAP) {
      Hit *h = hits + slot;
      h->src = src;
      h->cx = (tA.x + tB.x + tC.x) * (1.f / 3.f);
      h->cy = (tA.y + tB.y + tC.y) * (1.f / 3.f);
      h->cell = cell;
      h->status = ST_PENDING;
    }
  }
}
#endif

// Order-preserving map of floats to signed ints (and back: it is its own
// inverse), so that integer warp min/max reductions apply to floats.
__device__ __forceinline__ int f2ord(float f) {
  const int i = __float_as_int(f);
  return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i ^ ((i >> 31) & 0x7fffffff)); }

#ifndef LENS_SEARCH_PAIRED
#define LENS_SEARCH_PAIRED 0  // 1: two nodes per paired evaluation of the varying potentials (measured 1 % slower)
#endif
#ifndef LENS_SEARCH_MINB
#define LENS_SEARCH_MINB 4  // resident CTAs per SM the search is compiled for (64 registers: 4 % faster than 1, no spills; 5 spills)
#endif
__global__ void __launch_bounds__(SEARCH_THREADS, LENS_SEARCH_MINB) k_img_search(const SetArgs a, const SearchArgs g) {
  __shared__ __align__(16) float s_rec[2][REC32];
  __shared__ float2 s_off[2];  // tile origin minus each varying potential's centre
  __shared__ float s_T[2];     // tile origin
  __shared__ float2 s_al[NX_T * NY_T];
  __shared__ float2 s_src[MAX_SRC];
  __shared__ float s_box[SEARCH_GCH][4][SEARCH_WARPS];
  __shared__ int s_list[MAX_SRC];  // group q's sources inside the footprint, from s_list[grp_off[q]]
  __shared__ int s_nlist[SEARCH_GCH];
  const int b = blockIdx.z;
  if (!a.s.valid[b]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.x * CT_X, j0 = blockIdx.y * CT_Y;
  // positions in FP32 relative to the tile origin (the search only decides
  // which triangles seed a candidate; the refinement is exact); the few FP64
  // operations are done once per CTA
  const VarRecs &var = a.s.var[b];
  if (tid < 2) {
    const double T = tid == 0 ? g.xmin + i0 * g.dx : g.ymin + j0 * g.dy;
    s_T[tid] = (float)T;
    const double Tx = g.xmin + i0 * g.dx, Ty = g.ymin + j0 * g.dy;
    s_off[tid] = make_float2((float)(Tx - ((double)var.cen[tid][0] + (double)var.cen[tid][2])),
                             (float)(Ty - ((double)var.cen[tid][1] + (double)var.cen[tid][3])));
  }
  if (tid < 2 * REC32) s_rec[tid / REC32][tid % REC32] = var.r32[tid / REC32][tid % REC32];
  const float2 *src32 = a.s.src32 + (size_t)b * a.nsrc;
  for (int i = tid; i < a.nsrc; i += SEARCH_THREADS) s_src[i] = src32[i];
  __syncthreads();
  const float fdx = g.fdx, fdy = g.fdy, fTx = s_T[0], fTy = s_T[1];
#if LENS_SEARCH_PAIRED
  // the tile's nodes two at a time (n and n + SEARCH_THREADS) on the paired
  // FP32 path; past the end the second is a copy of the first, not stored
  for (int n = tid; n < NX_T * NY_T; n += 2 * SEARCH_THREADS) {
    const int n1 = n + SEARCH_THREADS < NX_T * NY_T ? n + SEARCH_THREADS : n;
    const int ia = min(i0 + n % NX_T, g.nx - 1), ja = min(j0 + n / NX_T, g.ny - 1);
    const int ib = min(i0 + n1 % NX_T, g.nx - 1), jb = min(j0 + n1 / NX_T, g.ny - 1);
    const size_t oa = (size_t)ja * g.nx + ia, ob = (size_t)jb * g.nx + ib;
    float2 tx = make_float2(g.ax[oa], g.ax[ob]), ty = make_float2(g.ay[oa], g.ay[ob]);
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const float2 dX2[1] = {make_float2(fmaf((float)(ia - i0), fdx, s_off[v].x), fmaf((float)(ib - i0), fdx, s_off[v].x))};
      const float2 dY2[1] = {make_float2(fmaf((float)(ja - j0), fdy, s_off[v].y), fmaf((float)(jb - j0), fdy, s_off[v].y))};
      Acc2<false, 1> acc;
      acc.zero();
      eval32x2_any<false, 1, false, true>(reinterpret_cast<const float4 *>(s_rec[v]), dX2, dY2, acc);
      tx = add2(tx, acc.ax[0]);
      ty = add2(ty, acc.ay[0]);
    }
    s_al[n] = make_float2(tx.x, ty.x);
    if (n1 != n) s_al[n1] = make_float2(tx.y, ty.y);
  }
#else
  for (int n = tid; n < NX_T * NY_T; n += SEARCH_THREADS) {
    const int li = n % NX_T, lj = n / NX_T;
    const int ii = min(i0 + li, g.nx - 1), jj = min(j0 + lj, g.ny - 1);
    const size_t o = (size_t)jj * g.nx + ii;
    float tx = g.ax[o], ty = g.ay[o];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      Acc<false, 1> acc;
      acc.zero();
      const float dX = fmaf((float)(ii - i0), fdx, s_off[v].x), dY[1] = {fmaf((float)(jj - j0), fdy, s_off[v].y)};
      eval32_any<false, 1, true>(reinterpret_cast<const float4 *>(s_rec[v]), dX, dY, acc);
      tx += acc.ax[0];
      ty += acc.ay[0];
    }
    s_al[n] = make_float2(tx, ty);
  }
#endif
  __syncthreads();
#if LENS_SEARCH_SUBTILE
  const int ci = lane;  // this thread's cells: column ci, rows warp SUB_R .. warp SUB_R + SUB_R - 1
#else
  const int ci = tid % CT_X, cj0 = tid / CT_X;  // this thread's cells: column ci, rows cj0, cj0 + CT_Y / CPT, ...
#endif
  const float tiny = g.tiny;
  int *cnt = a.s.cnt + b;
  Hit *hits = a.s.hits + (size_t)b * IMG_CAP;
  for (int q0 = 0; q0 < g.ng; q0 += SEARCH_GCH) {
    const int nq = min(SEARCH_GCH, g.ng - q0);
    // the tile's footprint in each ratio's source plane (bounding box of its
    // nodes): one pass over this thread's nodes for all groups of the chunk,
    // then one integer min/max reduction per warp and bound
    float lo[SEARCH_GCH][2], hi[SEARCH_GCH][2];
#pragma unroll
    for (int qq = 0; qq < SEARCH_GCH; ++qq) lo[qq][0] = lo[qq][1] = INFINITY, hi[qq][0] = hi[qq][1] = -INFINITY;
#if LENS_SEARCH_SUBTILE
    // warp w takes node rows w R .. w R + R (its own cells' rows and the row
    // below), so the bounds it reduces are its sub-tile's footprint
    for (int k = lane; k < (SUB_R + 1) * NX_T; k += 32) {
      const int n = warp * SUB_R * NX_T + k;
#else
    for (int n = tid; n < NX_T * NY_T; n += SEARCH_THREADS) {
#endif
      const int li = n % NX_T, lj = n / NX_T;
      if (i0 + li >= g.nx || j0 + lj >= g.ny) continue;
      const float X = fmaf((float)li, fdx, fTx), Y = fmaf((float)lj, fdy, fTy);
      const float2 al = s_al[n];
#pragma unroll
      for (int qq = 0; qq < SEARCH_GCH; ++qq) {
        if (qq >= nq) break;
        const float r = g.grp_r32[q0 + qq];
        const float bx = X - r * al.x, by = Y - r * al.y;
        lo[qq][0] = fminf(lo[qq][0], bx);
        hi[qq][0] = fmaxf(hi[qq][0], bx);
        lo[qq][1] = fminf(lo[qq][1], by);
        hi[qq][1] = fmaxf(hi[qq][1], by);
      }
    }
#pragma unroll
    for (int qq = 0; qq < SEARCH_GCH; ++qq) {
      if (qq >= nq) break;
      const int lx = __reduce_min_sync(0xffffffffu, f2ord(lo[qq][0])), hx = __reduce_max_sync(0xffffffffu, f2ord(hi[qq][0]));
      const int ly = __reduce_min_sync(0xffffffffu, f2ord(lo[qq][1])), hy = __reduce_max_sync(0xffffffffu, f2ord(hi[qq][1]));
      if (lane == 0) {
        s_box[qq][0][warp] = ord2f(lx);
        s_box[qq][1][warp] = ord2f(hx);
        s_box[qq][2][warp] = ord2f(ly);
        s_box[qq][3][warp] = ord2f(hy);
      }
    }
    __syncthreads();
    if (warp < nq) {
      // warp w: the sources of group q0 + w inside the footprint (+ the test's tolerance)
      float L = INFINITY, H = -INFINITY, Ly = INFINITY, Hy = -INFINITY;
      for (int w = 0; w < SEARCH_WARPS; ++w) {
        L = fminf(L, s_box[warp][0][w]);
        H = fmaxf(H, s_box[warp][1][w]);
        Ly = fminf(Ly, s_box[warp][2][w]);
        Hy = fmaxf(Hy, s_box[warp][3][w]);
      }
      const float px = BARY_TOL * (H - L) + 1e-5f, py = BARY_TOL * (Hy - Ly) + 1e-5f;
      const int g0 = g.grp_off[q0 + warp], g1 = g.grp_off[q0 + warp + 1];
      int base = 0;
      for (int k0 = g0; k0 < g1; k0 += 32) {
        const int k = k0 + lane;
        bool in = false;
        int src = 0;
        if (k < g1) {
          src = g.grp_src[k];
          const float2 P = s_src[src];
          in = P.x >= L - px && P.x <= H + px && P.y >= Ly - py && P.y <= Hy + py;
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) s_list[g0 + base + __popc(m & ((1u << lane) - 1u))] = src;
        base += __popc(m);
      }
      if (lane == 0) s_nlist[warp] = base;
    }
    __syncthreads();
    for (int qq = 0; qq < nq; ++qq) {
      const int nlist = s_nlist[qq];
      if (nlist == 0) continue;
      const float r = g.grp_r32[q0 + qq];
      const int *list = s_list + g.grp_off[q0 + qq];
#if LENS_SEARCH_SUBTILE
      // the list entries inside this warp's sub-tile footprint (padded as
      // the tile's, which covers every cell's padding), 32 at a time as bit
      // masks; a cell's box lies inside its sub-tile's
      const float sL = s_box[qq][0][warp], sH = s_box[qq][1][warp], sLy = s_box[qq][2][warp], sHy = s_box[qq][3][warp];
      const float spx = BARY_TOL * (sH - sL) + 1e-5f, spy = BARY_TOL * (sHy - sLy) + 1e-5f;
      for (int c0 = 0; c0 < nlist; c0 += 32) {
        bool in = false;
        if (c0 + lane < nlist) {
          const float2 P = s_src[list[c0 + lane]];
          in = P.x >= sL - spx && P.x <= sH + spx && P.y >= sLy - spy && P.y <= sHy + spy;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, in);
        if (mask == 0u) continue;  // uniform over the warp
#pragma unroll
        for (int rr = 0; rr < SUB_R; ++rr) {
          const int cj = warp * SUB_R + rr;
          const int gi = i0 + ci, gj = j0 + cj;
          if (gi >= g.nx - 1 || gj >= g.ny - 1) continue;
          const float X0 = fmaf((float)ci, fdx, fTx), X1 = fmaf((float)(ci + 1), fdx, fTx);
          const float Y0 = fmaf((float)cj, fdy, fTy), Y1 = fmaf((float)(cj + 1), fdy, fTy);
          const int n00 = cj * NX_T + ci;
          const float2 a00 = s_al[n00], a10 = s_al[n00 + 1], a01 = s_al[n00 + NX_T], a11 = s_al[n00 + NX_T + 1];
          const float2 t00 = make_float2(X0, Y0), t10 = make_float2(X1, Y0), t11 = make_float2(X1, Y1),
                       t01 = make_float2(X0, Y1);
          const float2 b00 = make_float2(X0 - r * a00.x, Y0 - r * a00.y),
                       b10 = make_float2(X1 - r * a10.x, Y0 - r * a10.y),
                       b11 = make_float2(X1 - r * a11.x, Y1 - r * a11.y),
                       b01 = make_float2(X0 - r * a01.x, Y1 - r * a01.y);
          const float qlx = fminf(fminf(b00.x, b10.x), fminf(b11.x, b01.x)),
                      qhx = fmaxf(fmaxf(b00.x, b10.x), fmaxf(b11.x, b01.x));
          const float qly = fminf(fminf(b00.y, b10.y), fminf(b11.y, b01.y)),
                      qhy = fmaxf(fmaxf(b00.y, b10.y), fmaxf(b11.y, b01.y));
          const float qpx = BARY_TOL * (qhx - qlx) + 1e-6f, qpy = BARY_TOL * (qhy - qly) + 1e-6f;
          bool any = false;
          for (unsigned mm = mask; mm && !any; mm &= mm - 1u) {
            const float2 P = s_src[list[c0 + __ffs(mm) - 1]];
            any = P.x >= qlx - qpx && P.x <= qhx + qpx && P.y >= qly - qpy && P.y <= qhy + qpy;
          }
          if (!any) continue;
          const int cell = 2 * (gj * (g.nx - 1) + gi);
          tri_test_mask(b00, b10, b11, t00, t10, t11, s_src, list + c0, mask, tiny, cnt, hits, cell);
          tri_test_mask(b00, b11, b01, t00, t11, t01, s_src, list + c0, mask, tiny, cnt, hits, cell + 1);
        }
      }
#else
#pragma unroll
      for (int half = 0; half < CPT; ++half) {
        const int cj = cj0 + half * (CT_Y / CPT);
        const int gi = i0 + ci, gj = j0 + cj;
        if (gi >= g.nx - 1 || gj >= g.ny - 1) continue;
        const float X0 = fmaf((float)ci, fdx, fTx), X1 = fmaf((float)(ci + 1), fdx, fTx);
        const float Y0 = fmaf((float)cj, fdy, fTy), Y1 = fmaf((float)(cj + 1), fdy, fTy);
        const int n00 = cj * NX_T + ci;
        const float2 a00 = s_al[n00], a10 = s_al[n00 + 1], a01 = s_al[n00 + NX_T], a11 = s_al[n00 + NX_T + 1];
        const float2 t00 = make_float2(X0, Y0), t10 = make_float2(X1, Y0), t11 = make_float2(X1, Y1),
                     t01 = make_float2(X0, Y1);
        const float2 b00 = make_float2(X0 - r * a00.x, Y0 - r * a00.y),
                     b10 = make_float2(X1 - r * a10.x, Y0 - r * a10.y),
                     b11 = make_float2(X1 - r * a11.x, Y1 - r * a11.y),
                     b01 = make_float2(X0 - r * a01.x, Y1 - r * a01.y);
        // the cell's padded bounding box contains both triangles' padded boxes
        const float qlx = fminf(fminf(b00.x, b10.x), fminf(b11.x, b01.x)),
                    qhx = fmaxf(fmaxf(b00.x, b10.x), fmaxf(b11.x, b01.x));
        const float qly = fminf(fminf(b00.y, b10.y), fminf(b11.y, b01.y)),
                    qhy = fmaxf(fmaxf(b00.y, b10.y), fmaxf(b11.y, b01.y));
        const float qpx = BARY_TOL * (qhx - qlx) + 1e-6f, qpy = BARY_TOL * (qhy - qly) + 1e-6f;
        bool any = false;
        for (int k = 0; k < nlist && !any; ++k) {
          const float2 P = s_src[list[k]];
          any = P.x >= qlx - qpx && P.x <= qhx + qpx && P.y >= qly - qpy && P.y <= qhy + qpy;
        }
        if (!any) continue;
        const int cell = 2 * (gj * (g.nx - 1) + gi);
        tri_test(b00, b10, b11, t00, t10, t11, s_src, list, nlist, tiny, cnt, hits, cell);
        tri_test(b00, b11, b01, t00, t11, t01, s_src, list, nlist, tiny, cnt, hits, cell + 1);
      }
#endif
    }
    __syncthreads();  // s_box, s_list and s_nlist are rewritten by the next chunk
  }
}

// ----------------------------------------------------------------- 3. Newton
struct NewtonArgs {
  const float *rec32, *cen32;  // static potentials on the FP32 path
  int n_light;
  int koff[5];                 // the FP32 ones by kind: Kind32 k occupies [koff[k], koff[k+1])
  const double *heavy;         // static potentials on the FP64 path
  const float2 *heavydf;       // the same in double-float, record-major (point-list refinement)
  int n_heavy;
  const double *all64;         // every static potential in FP64 (polish)
  const float2 *recdf;         // every static potential in double-float, field-major [RECDF][n_stat] (polish)
  int n_stat;
  const double *ratio;         // per source
  double xmin, ymin, dx, dy;   // search grid
  int nx;
  const float *gax, *gay;      // static deflection at the grid nodes [ny][nx] (D_ls/D_s = 1)
  int *err;                    // the context's error word
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int NW_THREADS = 256, NW_WARPS = NW_THREADS / 32;

// Barycentric weights of p in (a, b, c); false when degenerate.  The vertex
// offsets from p are formed in FP64 and the rest in FP32: the mapped vertices
// carry the FP32 sweep's error (~1e-7 of alpha), far above FP32 rounding of
// offsets of a (sub-)cell, and FP64 division is slow on this GPU.
__device__ __forceinline__ bool bary_w(const double *a, const double *b, const double *c, const double *p,
                                       double tiny, double w[3]) {
  const float ax = (float)(a[0] - p[0]), ay = (float)(a[1] - p[1]);
  const float bx = (float)(b[0] - p[0]), by = (float)(b[1] - p[1]);
  const float cx = (float)(c[0] - p[0]), cy = (float)(c[1] - p[1]);
  const float area2 = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
  if (!(fabs((double)area2) > tiny)) return false;
  const float inv = 1.f / area2;
  const float w0 = (bx * cy - by * cx) * inv, w1 = (cx * ay - cy * ax) * inv;
  w[0] = w0;
  w[1] = w1;
  w[2] = 1.0 - (double)w0 - (double)w1;
  return true;
}

// Vertex k of sub-triangle sb of a triangle (0, 1, 2) whose edge midpoints
// are 3 = (0,1), 4 = (1,2), 5 = (2,0): three corner triangles, then the middle.
__host__ __device__ constexpr int sub_vertex(int sb, int k) {
  return sb == 0   ? (k == 0 ? 0 : k == 1 ? 3 : 5)
         : sb == 1 ? (k == 0 ? 3 : k == 1 ? 1 : 4)
         : sb == 2 ? (k == 0 ? 5 : k == 1 ? 4 : 2)
                   : (k == 0 ? 3 : k == 1 ? 4 : 5);
}

// One candidate per group of RF_G threads.  Every evaluation is a sweep of
// the CTA over all static FP32 potentials, staged chunk by chunk in shared
// memory, each thread of a group taking every RF_G-th potential of a chunk
// with the compensated accumulation of the map kernel, plus the two varying
// potentials (FP32) and static cluster-scale ones (FP64, spread over the
// group); the group's partial sums are then combined by an xor butterfly,
// which gives every thread of the group the same bits (each level adds the
// same two values, and FP addition commutes).  Each thread evaluates NP
// points of its candidate per sweep.
// Newton steps: the two varying potentials in double-float, so the FP32 root
// is closer and the polish needs fewer full double-float evaluations
// (image-plane chi2, 1024^2 x 256 sets: 21.0 -> 19.6 ms)
#ifndef LENS_NEWTON_DFVAR
#define LENS_NEWTON_DFVAR 1
#endif
// FP32 Newton steps taken after the first step below NEWTON32_TOL (1 measured
// slower: the extra sweep costs more than the polish saves)
#ifndef LENS_NEWTON_EXTRA
#define LENS_NEWTON_EXTRA 0
#endif
#ifndef LENS_NEWTON_PAIRED
#define LENS_NEWTON_PAIRED 0
#endif
#ifndef LENS_RF_THREADS
#define LENS_RF_THREADS 128
#endif
#ifndef LENS_RF_G
#define LENS_RF_G 8
#endif
constexpr int RF_THREADS = LENS_RF_THREADS, RF_CH = 64, RF_G = LENS_RF_G, RF_CAND = RF_THREADS / RF_G;
constexpr int RF_STRIDE4 = REC32 / 4 + 1;  // float4 slots per staged record: the pad spreads a group's 8 records over all banks
static_assert(32 % RF_G == 0, "groups never straddle a warp");

// Point k of per-point sums or of pair sums.
template <int N>
__device__ __forceinline__ float pt_of(const float (&v)[N], int k) { return v[k]; }
template <int N>
__device__ __forceinline__ float pt_of(const float2 (&v)[N], int k) { return part2(v[k >> 1], k & 1); }

template <int NP, bool HESS>
__device__ __forceinline__ void sweep(const NewtonArgs &n, const VarRecs &var, float4 *s_rec, float4 *s_cen,
                                      const double (&px)[NP], const double (&py)[NP], double (&out)[NP][5]) {
  const int gl = threadIdx.x % RF_G;
  float hx[NP], lx[NP], hy[NP], ly[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    hx[k] = (float)px[k];
    lx[k] = (float)(px[k] - (double)hx[k]);
    hy[k] = (float)py[k];
    ly[k] = (float)(py[k] - (double)hy[k]);
  }
  // the NP points side by side (one range branch per potential); with
  // LENS_NEWTON_PAIRED, two or more points as pairs on the paired FP32 path
  // (an odd count padded with a copy of the last point, whose sums are not
  // used) -- measured slower: the padded fourth point and the registers of
  // the pairs (spills at 4 CTAs per SM) cost more than the pairing saves
  constexpr bool PAIRED = LENS_NEWTON_PAIRED && NP >= 2;
  constexpr int NPP = (NP + 1) / 2;
  using AccT = std::conditional_t<PAIRED, Acc2<HESS, NPP>, Acc<HESS, NP>>;
  AccT tot, cmp, part;
  tot.zero();
  cmp.zero();
  part.zero();
  auto fold_all = [&]() {
    if constexpr (PAIRED)
      fold2(tot, cmp, part);
    else
      fold(tot, cmp, part);
  };
  int seen = 0;
  const float4 *g_rec = reinterpret_cast<const float4 *>(n.rec32);
  const float4 *g_cen = reinterpret_cast<const float4 *>(n.cen32);
  for (int c0 = 0; c0 < n.n_light + 2; c0 += RF_CH) {
    const int cnt = min(RF_CH, n.n_light + 2 - c0);
    __syncthreads();  // the previous chunk has been used by every thread
    for (int i = threadIdx.x; i < cnt * (REC32 / 4); i += RF_THREADS) {
      const int hl = i / (REC32 / 4), hh = c0 + hl, q = i % (REC32 / 4);
      s_rec[hl * RF_STRIDE4 + q] = hh < n.n_light ? g_rec[(size_t)hh * (REC32 / 4) + q]
                                                  : reinterpret_cast<const float4 *>(var.r32[hh - n.n_light])[q];
    }
    for (int i = threadIdx.x; i < cnt; i += RF_THREADS) {
      const int hh = c0 + i;
      s_cen[i] = hh < n.n_light ? g_cen[hh]
                                : make_float4(var.cen[hh - n.n_light][0], var.cen[hh - n.n_light][1],
                                              var.cen[hh - n.n_light][2], var.cen[hh - n.n_light][3]);
    }
    __syncthreads();
    // kind-uniform runs of the chunk (the static potentials are sorted by
    // kind; the two varying ones at the end take the general dispatch)
    auto run = [&](auto kind_tag, int h0, int h1) {
      constexpr int KIND = decltype(kind_tag)::value;
      for (int h = h0 + gl; h < h1;) {
        // this thread's potentials up to the next fold (every 16 of them)
        const int hs = h, he = min(h1, h + (16 - seen) * RF_G);
        for (; h < he; h += RF_G) {
          const float4 *r4 = s_rec + h * RF_STRIDE4;
          const float4 c = s_cen[h];
          float dX[NP], dY[NP];
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            dX[k] = (hx[k] - c.x) + (lx[k] - c.z);
            dY[k] = (hy[k] - c.y) + (ly[k] - c.w);
          }
          if constexpr (PAIRED) {
            float2 dX2[NPP], dY2[NPP];
#pragma unroll
            for (int q = 0; q < NPP; ++q) {
              const int k1 = 2 * q + 1 < NP ? 2 * q + 1 : NP - 1;
              dX2[q] = make_float2(dX[2 * q], dX[k1]);
              dY2[q] = make_float2(dY[2 * q], dY[k1]);
            }
            if (KIND == K32_DPIE)
              dpie32x2<HESS, NPP, false, false>(r4, dX2, dY2, part);
            else if (KIND == K32_DPIE_SERIES)
              dpie32x2<HESS, NPP, true, false>(r4, dX2, dY2, part);
            else if (KIND == K32_SIS || KIND == K32_POINT)
              circ32x2<HESS, NPP, KIND == K32_POINT, false>(r4, dX2, dY2, part);
            else
              eval32x2_any<HESS, NPP, false>(r4, dX2, dY2, part);
          } else {
            if (KIND == K32_DPIE)
              dpie32<HESS, NP, false>(r4, dX, dY, part);
            else if (KIND == K32_DPIE_SERIES)
              dpie32<HESS, NP, true>(r4, dX, dY, part);
            else if (KIND == K32_SIS || KIND == K32_POINT)
              circ32<HESS, NP, KIND == K32_POINT>(r4, dX, dY, part);
            else
              eval32_any<HESS, NP>(r4, dX, dY, part);
          }
        }
        seen += (h - hs) / RF_G;
        if (seen == 16) {
          fold_all();
          seen = 0;
        }
      }
    };
    auto seg = [&](int lo, int hi, int &h0, int &h1) {
      h0 = max(lo - c0, 0);
      h1 = min(hi - c0, cnt);
    };
    int h0, h1;
    seg(n.koff[K32_DPIE], n.koff[K32_DPIE + 1], h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_DPIE>(), h0, h1);
    seg(n.koff[K32_DPIE_SERIES], n.koff[K32_DPIE_SERIES + 1], h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_DPIE_SERIES>(), h0, h1);
    seg(n.koff[K32_SIS], n.koff[K32_SIS + 1], h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_SIS>(), h0, h1);
    seg(n.koff[K32_POINT], n.koff[K32_POINT + 1], h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_POINT>(), h0, h1);
    if (!(HESS && LENS_NEWTON_DFVAR)) {
      seg(n.n_light, n.n_light + 2, h0, h1);
      if (h0 < h1) run(std::integral_constant<int, -1>(), h0, h1);
    }
  }
  constexpr int NC = HESS ? 5 : 2;
  fold_all();
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    // each thread's compensated sum tot - cmp as a float pair, combined over
    // the group in double-float (TwoSum gives both partners the same bits)
    float hi[5] = {pt_of(tot.ax, k), pt_of(tot.ay, k), HESS ? pt_of(tot.k, k) : 0.f, HESS ? pt_of(tot.g1, k) : 0.f,
                   HESS ? pt_of(tot.g2, k) : 0.f};
    float lo[5] = {-pt_of(cmp.ax, k), -pt_of(cmp.ay, k), HESS ? -pt_of(cmp.k, k) : 0.f,
                   HESS ? -pt_of(cmp.g1, k) : 0.f, HESS ? -pt_of(cmp.g2, k) : 0.f};
#pragma unroll
    for (int o = 1; o < RF_G; o <<= 1)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const float ph = __shfl_xor_sync(0xffffffffu, hi[q], o), pl = __shfl_xor_sync(0xffffffffu, lo[q], o);
        const df t = two_sum(hi[q], ph);
        const df u = fast_two_sum(t.hi, t.lo + (lo[q] + pl));
        hi[q] = u.hi;
        lo[q] = u.lo;
      }
#pragma unroll
    for (int q = 0; q < 5; ++q) out[k][q] = q < NC ? (double)hi[q] + (double)lo[q] : 0.0;
    if (n.n_heavy > 0) {  // static cluster-scale potentials: FP64, spread over the group
      double hv[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int j = gl; j < n.n_heavy; j += RF_G) {
        double e0, e1, e2 = 0, e3 = 0, e4 = 0;
        eval64<HESS>(n.heavy + (size_t)j * REC64, px[k], py[k], e0, e1, e2, e3, e4);
        hv[0] += e0;
        hv[1] += e1;
        hv[2] += e2;
        hv[3] += e3;
        hv[4] += e4;
      }
#pragma unroll
      for (int o = 1; o < RF_G; o <<= 1)
#pragma unroll
        for (int q = 0; q < NC; ++q) hv[q] += __shfl_xor_sync(0xffffffffu, hv[q], o);
#pragma unroll
      for (int q = 0; q < NC; ++q) out[k][q] += hv[q];
    }
    if (HESS && LENS_NEWTON_DFVAR) {
      // the two varying (cluster-scale) potentials in double-float, one on
      // each of the group's first two threads, broadcast to the group: their
      // FP32 error would otherwise set the Newton root's noise floor
      float vh[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, vl[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (gl < 2) {
        const float2 *rec = var.rdf[gl];
        const df X = df_from_double(px[k]), Y = df_from_double(py[k]);
        df ax, ay, h[3];
        bool ok = true;
        if (rec[F_U2].x < 0.f)
          circ_df<true>(rec, 1, X, Y, ax, ay, h);
        else
          ok = dpie_df<true, true>(rec, 1, X, Y, ax, ay, h);
        if (!ok) {
          double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
          eval64<true>(var.r64[gl], px[k], py[k], e[0], e[1], e[2], e[3], e[4]);
          ax = df_from_double(e[0]);
          ay = df_from_double(e[1]);
          h[0] = df_from_double(e[2]);
          h[1] = df_from_double(e[3]);
          h[2] = df_from_double(e[4]);
        }
        const df v[5] = {ax, ay, h[0], h[1], h[2]};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          vh[q] = v[q].hi;
          vl[q] = v[q].lo;
        }
      }
      const int g0 = (threadIdx.x & 31) & ~(RF_G - 1);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const float a0 = __shfl_sync(0xffffffffu, vh[q], g0), b0 = __shfl_sync(0xffffffffu, vl[q], g0);
        const float a1 = __shfl_sync(0xffffffffu, vh[q], g0 + 1), b1 = __shfl_sync(0xffffffffu, vl[q], g0 + 1);
        out[k][q] += ((double)a0 + (double)b0) + ((double)a1 + (double)b1);
      }
    }
  }
}

#ifndef LENS_NEWTON_MINB
#define LENS_NEWTON_MINB 4  // resident CTAs per SM the Newton kernel is compiled for
#endif
__global__ void __launch_bounds__(RF_THREADS, LENS_NEWTON_MINB) k_img_newton(const SetArgs a, const NewtonArgs n) {
  __shared__ float4 s_rec[RF_CH * RF_STRIDE4];
  __shared__ float4 s_cen[RF_CH];
  __shared__ VarRecs s_var;
  const int b = blockIdx.y;
  if (!a.s.valid[b]) return;
  const int ncand = min(a.s.cnt[b], IMG_CAP);
  if (blockIdx.x * RF_CAND >= ncand) return;  // both exits are uniform over the CTA
  {
    const float *f = reinterpret_cast<const float *>(&a.s.var[b]);
    float *d = reinterpret_cast<float *>(&s_var);
    for (int i = threadIdx.x; i < (int)(sizeof(VarRecs) / sizeof(float)); i += RF_THREADS) d[i] = f[i];
  }
  const int k = blockIdx.x * RF_CAND + threadIdx.x / RF_G;  // the group's candidate
  const bool mine = k < ncand, lead = threadIdx.x % RF_G == 0;
  Hit *h = a.s.hits + (size_t)b * IMG_CAP + (mine ? k : 0);
  const int src = mine ? h->src : 0;
  const double r = n.ratio[src];
  const double P[2] = {a.s.bary[((size_t)b * a.nsrc + src) * 2], a.s.bary[((size_t)b * a.nsrc + src) * 2 + 1]};
  const int cell = mine ? h->cell : 0, tri = cell & 1, ci = (cell >> 1) % (n.nx - 1), cj = (cell >> 1) / (n.nx - 1);
  // triangle 0: (i,j),(i+1,j),(i+1,j+1); triangle 1: (i,j),(i+1,j+1),(i,j+1)
  const int oi[2][3] = {{ci, ci + 1, ci + 1}, {ci, ci + 1, ci}}, oj[2][3] = {{cj, cj, cj + 1}, {cj, cj + 1, cj + 1}};
  double th[3][2], be[3][2];
  __syncthreads();  // s_var complete
  // the vertices are grid nodes: static deflection from the grid cache (the
  // search's values), the two varying potentials in FP32
  for (int q = 0; q < 3; ++q) {
    const int ii = oi[tri][q], jj = oj[tri][q];
    th[q][0] = n.xmin + ii * n.dx;
    th[q][1] = n.ymin + jj * n.dy;
    const size_t o = (size_t)jj * n.nx + ii;
    float ax = n.gax[o], ay = n.gay[o];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      Acc<false, 1> acc;
      acc.zero();
      const float dY[1] = {(float)(th[q][1] - ((double)s_var.cen[v][1] + (double)s_var.cen[v][3]))};
      eval32_any<false, 1>(reinterpret_cast<const float4 *>(s_var.r32[v]),
                           (float)(th[q][0] - ((double)s_var.cen[v][0] + (double)s_var.cen[v][2])), dY, acc);
      ax += acc.ax[0];
      ay += acc.ay[0];
    }
    be[q][0] = th[q][0] - r * ax;
    be[q][1] = th[q][1] - r * ay;
  }
  // subdivision: keep the sub-triangle that best contains the source; stop
  // when none does (map far from linear on this triangle)
  double tiny = 1e-14 * n.dx * n.dy, wgt[3] = {1.0 / 3, 1.0 / 3, 1.0 / 3};
  bool refining = mine;
  for (int lev = 0; lev < SUBDIV_LEVELS; ++lev) {
    if (!__syncthreads_or(refining)) break;
    double t6[6][2], mx[3], my[3], o[3][5];
    for (int q = 0; q < 3; ++q) {
      const int q1 = q == 2 ? 0 : q + 1;
      t6[q][0] = th[q][0];
      t6[q][1] = th[q][1];
      t6[3 + q][0] = mx[q] = 0.5 * (th[q][0] + th[q1][0]);
      t6[3 + q][1] = my[q] = 0.5 * (th[q][1] + th[q1][1]);
    }
    sweep<3, false>(n, s_var, s_rec, s_cen, mx, my, o);
    if (!refining) continue;
    double b6[6][2];
    for (int q = 0; q < 3; ++q) {
      b6[q][0] = be[q][0];
      b6[q][1] = be[q][1];
      b6[3 + q][0] = t6[3 + q][0] - r * o[q][0];
      b6[3 + q][1] = t6[3 + q][1] - r * o[q][1];
    }
    const double tiny_sub = 0.25 * tiny;
    int best = -1;
    double best_score = -INFINITY;
    // (every loop over sub-triangles is unrolled so the vertex tables index
    // registers with constants)
#pragma unroll
    for (int sb = 0; sb < 4; ++sb) {
      double ww[3];
      if (!bary_w(b6[sub_vertex(sb, 0)], b6[sub_vertex(sb, 1)], b6[sub_vertex(sb, 2)], P, tiny_sub, ww)) continue;
      const double score = fmin(ww[0], fmin(ww[1], ww[2]));
      if (score > best_score) {
        best_score = score;
        best = sb;
      }
    }
    if (best < 0 || best_score < -SUBDIV_TOL) {
      if (!bary_w(be[0], be[1], be[2], P, tiny, wgt)) wgt[0] = wgt[1] = wgt[2] = 1.0 / 3;
      refining = false;
      continue;
    }
    tiny = tiny_sub;
#pragma unroll
    for (int sb = 0; sb < 4; ++sb)
      if (sb == best)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          th[q][0] = t6[sub_vertex(sb, q)][0];
          th[q][1] = t6[sub_vertex(sb, q)][1];
          be[q][0] = b6[sub_vertex(sb, q)][0];
          be[q][1] = b6[sub_vertex(sb, q)][1];
        }
  }
  if (refining && !bary_w(be[0], be[1], be[2], P, tiny, wgt)) wgt[0] = wgt[1] = wgt[2] = 1.0 / 3;
  // FP32 Newton with steps limited to one cell
  double tx = wgt[0] * th[0][0] + wgt[1] * th[1][0] + wgt[2] * th[2][0];
  double ty = wgt[0] * th[0][1] + wgt[1] * th[1][1] + wgt[2] * th[2][1];
  const double step_max = fmax(n.dx, n.dy);
  int status = ST_FAILED, settled = 0;
  float h11 = 0.f, h22 = 0.f, h12 = 0.f;
  bool active = mine;
  for (int it = 0; it < NEWTON_MAXIT; ++it) {
    if (!__syncthreads_or(active)) break;
    double px[1] = {tx}, py[1] = {ty}, o[1][5];
    sweep<1, true>(n, s_var, s_rec, s_cen, px, py, o);
    if (!active) continue;
    const double fx = P[0] - (tx - r * o[0][0]), fy = P[1] - (ty - r * o[0][1]);
    const double m11 = r * (o[0][2] + o[0][3]), m22 = r * (o[0][2] - o[0][3]), m12 = r * o[0][4];
    const double a11 = 1.0 - m11, a22 = 1.0 - m22, a12 = -m12;
    const double det = a11 * a22 - a12 * a12;
    if (!(det != 0.0) || !isfinite(det)) {
      active = false;
      continue;
    }
    double dx = (a22 * fx - a12 * fy) / det, dy = (a11 * fy - a12 * fx) / det;
    const double len = sqrt(dx * dx + dy * dy);
    if (len > step_max) {
      dx *= step_max / len;
      dy *= step_max / len;
    }
    tx += dx;
    ty += dy;
    h11 = (float)m11;
    h22 = (float)m22;
    h12 = (float)m12;
    if (!isfinite(tx) || !isfinite(ty)) {
      active = false;
      continue;
    }
    if (len < NEWTON32_TOL && ++settled > LENS_NEWTON_EXTRA) {
      status = ST_NEWTON;
      active = false;
    }
  }
  // a root far from its triangle belongs to another triangle's search
  if (status == ST_NEWTON && hypot(tx - h->cx, ty - h->cy) > LOCAL_CELLS * fmax(n.dx, n.dy)) status = ST_FAR;
  if (mine && lead) {
    h->tx = tx;
    h->ty = ty;
    h->h11 = h11;
    h->h22 = h22;
    h->h12 = h12;
    h->status = status;
  }
}

// ---------------------------------------------- 3'. refinement, point lists
// Step 3 as a sequence of dense evaluations (LENS_REFINE_LISTS): every
// subdivision level evaluates the edge midpoints of all refining candidates
// of the batch in one launch, and every Newton round the Newton points of
// all active candidates, with the map kernel's structure -- one thread per
// KP points (two-point pairs on the paired FP32 path), the static FP32
// potentials streamed chunk by chunk into shared memory by bulk copies and
// read by every thread at once, Kahan folds every SUB potentials, the
// static cluster-scale potentials in FP64 and the two varying potentials
// per point; small kernels between the evaluations take the decisions per
// candidate (the same ones as k_img_newton) and append the next points.
// Candidates still iterating after NEWTON_ROUNDS Newton steps (0.9 % of them
// on the 1000-potential model) finish in k_ref_straggle, one CTA each.
#ifndef LENS_REFINE_LISTS
#define LENS_REFINE_LISTS 1
#endif
// The refinement's Newton steps solve their 2 x 2 systems in FP32 (1:
// 13.11 -> 12.93 ms per 256 sets, the stragglers' steps being chains of
// FP64 divisions and roots), the residual staying in FP64
#ifndef LENS_NEWTON_STEP32
#define LENS_NEWTON_STEP32 1
#endif
constexpr int PE_THREADS = 128, PE_CH = 64, PE_SUB = 16;
#ifndef LENS_PE_MINB_GRAD
#define LENS_PE_MINB_GRAD 4
#endif
#ifndef LENS_PE_MINB_HESS
#define LENS_PE_MINB_HESS 4
#endif
__host__ __device__ constexpr int pe_points(bool hess) { return PE_THREADS * (hess ? 2 : 4); }

// The compiler may not see through v: it has to keep it in registers.
__device__ __forceinline__ void opaque2(float2 &v) { asm volatile("" : "+f"(v.x), "+f"(v.y)); }

// Position of list entry e: an edge midpoint of the slot's current triangle
// or its Newton point.
__device__ __forceinline__ void entry_point(const Bufs &s, int e, double &X, double &Y) {
  const int slot = e >> 2, m = e & 3;
  if (m == 3) {
    X = s.hits[slot].tx;
    Y = s.hits[slot].ty;
  } else {
    const Ref &r = s.ref[slot];
    const int m1 = m == 2 ? 0 : m + 1;
    X = 0.5 * (r.th[m][0] + r.th[m1][0]);
    Y = 0.5 * (r.th[m][1] + r.th[m1][1]);
  }
}

template <bool HESS>
__global__ void __launch_bounds__(PE_THREADS, HESS ? LENS_PE_MINB_HESS : LENS_PE_MINB_GRAD)
    k_pts_eval(const SetArgs a, const NewtonArgs n, const int *__restrict__ lst, const int *__restrict__ count) {
  constexpr int KP = HESS ? 2 : 4, NP = KP / 2, NC = HESS ? 5 : 2;
  __shared__ __align__(128) float s_rec[2][PE_CH * REC32];
  __shared__ __align__(16) float4 s_cen[2][PE_CH];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ double s_hv[PE_THREADS][KP][NC];
  const int npts = *count, p0 = blockIdx.x * pe_points(HESS);
  if (p0 >= npts) return;  // uniform over the CTA
  const int tid = threadIdx.x;
  int ent[KP];
  bool live[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int p = p0 + k * PE_THREADS + tid;
    live[k] = p < npts;
    ent[k] = lst[live[k] ? p : p0];  // past the end: the tile's first point again, not stored
  }
  // hi/lo float pairs of the positions: (hi - centre hi) is exact next to a
  // centre (Sterbenz), as in k_img_newton's sweeps.  Made opaque, so that
  // the compiler keeps them rather than re-deriving them from the doubles
  // inside the potential loop (conversions run on the FP64 pipe, at 1/64 of
  // the FP32 rate: that re-derivation made the kernel FP64-bound).
  float2 hx[NP], lx[NP], hy[NP], ly[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double x, y;
      entry_point(a.s, ent[2 * j + h], x, y);
      const float fx = (float)x, fy = (float)y;
      part2(hx[j], h) = fx;
      part2(lx[j], h) = (float)(x - (double)fx);
      part2(hy[j], h) = fy;
      part2(ly[j], h) = (float)(y - (double)fy);
    }
    opaque2(hx[j]);
    opaque2(lx[j]);
    opaque2(hy[j]);
    opaque2(ly[j]);
  }
  // static cluster-scale potentials in double-float (FP64 where that
  // fails), before or after the FP32 sweep by tile parity.  Not FP64: at the
  // images these potentials mostly take the atan/atanh reductions, and in
  // FP64 (1/64 of the FP32 rate) that alone kept the FP64 pipe 84 % busy
  // for 2.5 times the sweep's FP32 time.
  auto heavy_pass = [&]() {
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      double X, Y;
      entry_point(a.s, ent[k], X, Y);
      for (int j = 0; j < n.n_heavy; ++j)
        add_potential_df<HESS>(n.heavydf + (size_t)j * RECDF, 1, n.heavy + (size_t)j * REC64, X, Y, v);
#pragma unroll
      for (int c = 0; c < NC; ++c) s_hv[tid][k][c] = v[c];
    }
  };
  const bool heavy_first = (blockIdx.x & 1) != 0;
  if (heavy_first) heavy_pass();

  Acc2<HESS, NP> tot, cmp, part;
  tot.zero();
  cmp.zero();
  part.zero();
  const int nl = n.n_light, nch = (nl + PE_CH - 1) / PE_CH;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int ch) {  // thread 0: chunk ch's records and centres into buffer ch & 1
    const int base = ch * PE_CH, cnt = min(PE_CH, nl - base), buf = ch & 1;
    mbar_expect_tx(&s_bar[buf], cnt * (REC32 * 4 + 16));
    bulk_g2s(&s_rec[buf][0], n.rec32 + (size_t)base * REC32, cnt * REC32 * 4, &s_bar[buf]);
    bulk_g2s(&s_cen[buf][0], n.cen32 + (size_t)base * 4, cnt * 16, &s_bar[buf]);
  };
  if (tid == 0 && nch > 0) issue(0);
  int seen = 0;
  for (int ch = 0; ch < nch; ++ch) {
    const int buf = ch & 1, base = ch * PE_CH, cnt = min(PE_CH, nl - base);
    const bool ok = mbar_wait_bounded(&s_bar[buf], (ch >> 1) & 1);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(n.err, ERRBIT_WAIT);
        mbar_wait_bounded(&s_bar[buf], (ch >> 1) & 1);  // let the copy in flight land before leaving
      }
      return;
    }
    if (tid == 0 && ch + 1 < nch) {
      fence_proxy_async();
      issue(ch + 1);
    }
    const float4 *recs = reinterpret_cast<const float4 *>(&s_rec[buf][0]);
    const float4 *cens = &s_cen[buf][0];
    auto run = [&](auto kind_tag, int h0, int h1) {
      constexpr int KIND = decltype(kind_tag)::value;
      for (int h = h0; h < h1;) {
        const int he = min(h + (PE_SUB - seen), h1);
        seen += he - h;
#pragma unroll 2
        for (; h < he; ++h) {
          const float4 *r4 = recs + h * (REC32 / 4);
          const float4 c = cens[h];
          float2 dX[NP], dY[NP];
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            dX[j] = add2(sub2(hx[j], dup2(c.x)), sub2(lx[j], dup2(c.z)));
            dY[j] = add2(sub2(hy[j], dup2(c.y)), sub2(ly[j], dup2(c.w)));
          }
          if (KIND == K32_DPIE)
            dpie32x2<HESS, NP, false, false>(r4, dX, dY, part);
          else if (KIND == K32_DPIE_SERIES)
            dpie32x2<HESS, NP, true, false>(r4, dX, dY, part);
          else
            circ32x2<HESS, NP, KIND == K32_POINT, false>(r4, dX, dY, part);
        }
        if (seen == PE_SUB) {
          fold2(tot, cmp, part);
          seen = 0;
        }
      }
    };
    auto seg = [&](int k, int &h0, int &h1) {
      h0 = max(n.koff[k] - base, 0);
      h1 = min(n.koff[k + 1] - base, cnt);
    };
    int h0, h1;
    seg(K32_DPIE, h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_DPIE>(), h0, h1);
    seg(K32_DPIE_SERIES, h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_DPIE_SERIES>(), h0, h1);
    seg(K32_SIS, h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_SIS>(), h0, h1);
    seg(K32_POINT, h0, h1);
    if (h0 < h1) run(std::integral_constant<int, K32_POINT>(), h0, h1);
  }
  fold2(tot, cmp, part);
  if (!heavy_first) heavy_pass();

  // the two varying potentials of each point's parameter set: FP32 in the
  // subdivision (as k_img_newton's sweeps), double-float with FP64 fallback
  // in the Newton steps
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int slot = ent[k] >> 2;
    const VarRecs &var = a.s.var[slot / IMG_CAP];
    double Xk, Yk;
    entry_point(a.s, ent[k], Xk, Yk);
    double o[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) o[c] = c < NC ? s_hv[tid][k][c] : 0.0;
    const float2 *tt[5] = {tot.ax, tot.ay, tot.k, tot.g1, tot.g2};
    const float2 *cc[5] = {cmp.ax, cmp.ay, cmp.k, cmp.g1, cmp.g2};
#pragma unroll
    for (int c = 0; c < NC; ++c) o[c] += (double)part2(tt[c][k >> 1], k & 1) - (double)part2(cc[c][k >> 1], k & 1);
    if (!HESS) {
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        Acc<false, 1> acc;
        acc.zero();
        const float dY[1] = {(float)(Yk - ((double)var.cen[v][1] + (double)var.cen[v][3]))};
        eval32_any<false, 1>(reinterpret_cast<const float4 *>(var.r32[v]),
                             (float)(Xk - ((double)var.cen[v][0] + (double)var.cen[v][2])), dY, acc);
        o[0] += acc.ax[0];
        o[1] += acc.ay[0];
      }
    } else {
      const df Xd = df_from_double(Xk), Yd = df_from_double(Yk);
#pragma unroll 1
      for (int v = 0; v < 2; ++v) {
        const float2 *rec = var.rdf[v];
        df ax, ay, hh[3];
        bool okv = true;
        if (rec[F_U2].x < 0.f)
          circ_df<true>(rec, 1, Xd, Yd, ax, ay, hh);
        else
          okv = dpie_df<true, true>(rec, 1, Xd, Yd, ax, ay, hh);
        if (okv) {
          o[0] += df_to_double(ax);
          o[1] += df_to_double(ay);
          o[2] += df_to_double(hh[0]);
          o[3] += df_to_double(hh[1]);
          o[4] += df_to_double(hh[2]);
        } else {
          double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
          eval64<true>(var.r64[v], Xk, Yk, e[0], e[1], e[2], e[3], e[4]);
#pragma unroll
          for (int c = 0; c < 5; ++c) o[c] += e[c];
        }
      }
    }
    if (!live[k]) continue;
    Ref &r = a.s.ref[slot];
    const int m = ent[k] & 3;
    if (m == 3) {
#pragma unroll
      for (int c = 0; c < NC; ++c) r.mo[c] = o[c];
    } else {
      r.mo[2 * m] = o[0];
      r.mo[2 * m + 1] = o[1];
    }
  }
}

// The source position, ratio and grid spacing a candidate's decisions use.
struct CandCtx {
  double P[2], r, tiny0, step_max, local;
};
__device__ __forceinline__ CandCtx cand_ctx(const SetArgs &a, const NewtonArgs &n, int slot) {
  CandCtx c;
  const int b = slot / IMG_CAP, src = a.s.hits[slot].src;
  c.r = n.ratio[src];
  c.P[0] = a.s.bary[((size_t)b * a.nsrc + src) * 2];
  c.P[1] = a.s.bary[((size_t)b * a.nsrc + src) * 2 + 1];
  c.tiny0 = 1e-14 * n.dx * n.dy;
  c.step_max = fmax(n.dx, n.dy);
  c.local = LOCAL_CELLS * fmax(n.dx, n.dy);
  return c;
}

// Newton start from the barycentric weights of P in the current triangle
// (the centroid where they are degenerate); the slot joins round 0.
__device__ __forceinline__ void newton_start(const SetArgs &a, int slot, const CandCtx &c, bool weigh, int *lst0,
                                             int *cnt0) {
  Ref &R = a.s.ref[slot];
  Hit &h = a.s.hits[slot];
  double wgt[3] = {1.0 / 3, 1.0 / 3, 1.0 / 3};
  if (weigh && !bary_w(R.be[0], R.be[1], R.be[2], c.P, R.tiny, wgt)) wgt[0] = wgt[1] = wgt[2] = 1.0 / 3;
  h.tx = wgt[0] * R.th[0][0] + wgt[1] * R.th[1][0] + wgt[2] * R.th[2][0];
  h.ty = wgt[0] * R.th[0][1] + wgt[1] * R.th[1][1] + wgt[2] * R.th[2][1];
  h.h11 = h.h22 = h.h12 = 0.f;
  h.status = ST_FAILED;
  R.nit = 0;
  R.settled = 0;
  lst0[atomicAdd(cnt0, 1)] = slot << 2 | 3;
}

constexpr int RL_THREADS = 128;

// Initial triangle of every candidate: vertices from the grid, their source
// images from the grid cache plus the varying potentials (FP32), as
// k_img_newton; the three edge midpoints join subdivision level 0.
__global__ void __launch_bounds__(RL_THREADS) k_ref_init(const SetArgs a, const NewtonArgs n) {
  const int b = blockIdx.y;
  if (!a.s.valid[b]) return;
  const int k = blockIdx.x * RL_THREADS + threadIdx.x;
  if (k >= min(a.s.cnt[b], IMG_CAP)) return;
  const int slot = b * IMG_CAP + k;
  const Hit &h = a.s.hits[slot];
  const CandCtx c = cand_ctx(a, n, slot);
  const VarRecs &var = a.s.var[b];
  const int cell = h.cell, tri = cell & 1, ci = (cell >> 1) % (n.nx - 1), cj = (cell >> 1) / (n.nx - 1);
  // triangle 0: (i,j),(i+1,j),(i+1,j+1); triangle 1: (i,j),(i+1,j+1),(i,j+1)
  const int oi[2][3] = {{ci, ci + 1, ci + 1}, {ci, ci + 1, ci}}, oj[2][3] = {{cj, cj, cj + 1}, {cj, cj + 1, cj + 1}};
  Ref &R = a.s.ref[slot];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int ii = oi[tri][q], jj = oj[tri][q];
    const double tx = n.xmin + ii * n.dx, ty = n.ymin + jj * n.dy;
    const size_t o = (size_t)jj * n.nx + ii;
    float ax = n.gax[o], ay = n.gay[o];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      Acc<false, 1> acc;
      acc.zero();
      const float dY[1] = {(float)(ty - ((double)var.cen[v][1] + (double)var.cen[v][3]))};
      eval32_any<false, 1>(reinterpret_cast<const float4 *>(var.r32[v]),
                           (float)(tx - ((double)var.cen[v][0] + (double)var.cen[v][2])), dY, acc);
      ax += acc.ax[0];
      ay += acc.ay[0];
    }
    R.th[q][0] = tx;
    R.th[q][1] = ty;
    R.be[q][0] = tx - c.r * ax;
    R.be[q][1] = ty - c.r * ay;
  }
  R.tiny = c.tiny0;
  int *cnt = a.s.lcnt;
  if (SUBDIV_LEVELS > 0) {
    const int base = atomicAdd(&cnt[0], 3);
#pragma unroll
    for (int m = 0; m < 3; ++m) a.s.lst[base + m] = slot << 2 | m;
  } else {
    const size_t N = (size_t)a.B * IMG_CAP;
    newton_start(a, slot, c, true, a.s.lst + 6 * N, &cnt[SUBDIV_LEVELS]);
  }
}

// Subdivision level `lev` after its midpoints were evaluated: keep the
// sub-triangle that best contains the source, or stop refining (k_img_newton's
// rule); the next level's midpoints, or the Newton start, are appended.
__global__ void __launch_bounds__(RL_THREADS) k_ref_level(const SetArgs a, const NewtonArgs n, int lev) {
  const size_t N = (size_t)a.B * IMG_CAP;
  const int *lst = a.s.lst + ((lev & 1) ? 3 * N : 0);
  int *nxt = a.s.lst + ((lev & 1) ? 0 : 3 * N);
  int *cnt = a.s.lcnt;
  const int npts = cnt[lev];
  for (int p = blockIdx.x * RL_THREADS + threadIdx.x; p < npts; p += gridDim.x * RL_THREADS) {
    const int e = lst[p];
    if ((e & 3) != 0) continue;  // one thread per candidate: its first midpoint's
    const int slot = e >> 2;
    const CandCtx c = cand_ctx(a, n, slot);
    Ref &R = a.s.ref[slot];
    double t6[6][2], b6[6][2];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int q1 = q == 2 ? 0 : q + 1;
      t6[q][0] = R.th[q][0];
      t6[q][1] = R.th[q][1];
      t6[3 + q][0] = 0.5 * (R.th[q][0] + R.th[q1][0]);
      t6[3 + q][1] = 0.5 * (R.th[q][1] + R.th[q1][1]);
      b6[q][0] = R.be[q][0];
      b6[q][1] = R.be[q][1];
      b6[3 + q][0] = t6[3 + q][0] - c.r * R.mo[2 * q];
      b6[3 + q][1] = t6[3 + q][1] - c.r * R.mo[2 * q + 1];
    }
    const double tiny_sub = 0.25 * R.tiny;
    int best = -1;
    double best_score = -INFINITY;
#pragma unroll
    for (int sb = 0; sb < 4; ++sb) {
      double ww[3];
      if (!bary_w(b6[sub_vertex(sb, 0)], b6[sub_vertex(sb, 1)], b6[sub_vertex(sb, 2)], c.P, tiny_sub, ww)) continue;
      const double score = fmin(ww[0], fmin(ww[1], ww[2]));
      if (score > best_score) {
        best_score = score;
        best = sb;
      }
    }
    if (best < 0 || best_score < -SUBDIV_TOL) {
      newton_start(a, slot, c, true, a.s.lst + 6 * N, &cnt[SUBDIV_LEVELS]);
      continue;
    }
    R.tiny = tiny_sub;
#pragma unroll
    for (int sb = 0; sb < 4; ++sb)
      if (sb == best)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          R.th[q][0] = t6[sub_vertex(sb, q)][0];
          R.th[q][1] = t6[sub_vertex(sb, q)][1];
          R.be[q][0] = b6[sub_vertex(sb, q)][0];
          R.be[q][1] = b6[sub_vertex(sb, q)][1];
        }
    if (lev + 1 < SUBDIV_LEVELS) {
      const int base = atomicAdd(&cnt[lev + 1], 3);
#pragma unroll
      for (int m = 0; m < 3; ++m) nxt[base + m] = slot << 2 | m;
    } else {
      newton_start(a, slot, c, true, a.s.lst + 6 * N, &cnt[SUBDIV_LEVELS]);
    }
  }
}

// One Newton step of a candidate from its evaluation o (alpha, kappa, gamma1,
// gamma2 at (tx, ty)): k_img_newton's step, limited to one cell; tx, ty
// and the step counters are the caller's (the hit receives the position,
// r H and, at the end, the status).  Returns true while the candidate
// iterates; otherwise its status is final.
__device__ __forceinline__ bool newton_step(const SetArgs &a, int slot, const CandCtx &c, const double *o, double &tx,
                                            double &ty, int &nit, int &settled) {
  Hit &h = a.s.hits[slot];
  int status = ST_FAILED;
  bool active = true;
  const double fx = c.P[0] - (tx - c.r * o[0]), fy = c.P[1] - (ty - c.r * o[1]);
#if LENS_NEWTON_STEP32
  // the residual in FP64 (it is a small difference of large numbers), the
  // 2 x 2 solve in FP32: the step needs only FP32's relative precision, and
  // a chain of FP64 divisions and roots is slow on this GPU's FP64 unit
  const float rf = (float)c.r, k = (float)o[2], g1 = (float)o[3], g2 = (float)o[4];
  const float m11 = rf * (k + g1), m22 = rf * (k - g1), m12 = rf * g2;
  const float a11 = 1.f - m11, a22 = 1.f - m22, a12 = -m12;
  const float det = a11 * a22 - a12 * a12;
  if (!(det != 0.f) || !isfinite(det)) {
    active = false;
  } else {
    const float fxf = (float)fx, fyf = (float)fy, idet = 1.f / det;
    float dx = (a22 * fxf - a12 * fyf) * idet, dy = (a11 * fyf - a12 * fxf) * idet;
    const float len = sqrtf(dx * dx + dy * dy), smax = (float)c.step_max;
    if (len > smax) {
      dx *= smax / len;
      dy *= smax / len;
    }
    tx += (double)dx;
    ty += (double)dy;
    h.tx = tx;
    h.ty = ty;
    h.h11 = m11;
    h.h22 = m22;
    h.h12 = m12;
    if (!isfinite(tx) || !isfinite(ty)) {
      active = false;
    } else if (len < (float)NEWTON32_TOL && ++settled > LENS_NEWTON_EXTRA) {
      status = ST_NEWTON;
      active = false;
    }
  }
  if (active && ++nit < NEWTON_MAXIT) return true;
  if (status == ST_NEWTON && hypotf((float)(tx - h.cx), (float)(ty - h.cy)) > (float)c.local) status = ST_FAR;
  h.status = status;
  return false;
#else
  const double m11 = c.r * (o[2] + o[3]), m22 = c.r * (o[2] - o[3]), m12 = c.r * o[4];
  const double a11 = 1.0 - m11, a22 = 1.0 - m22, a12 = -m12;
  const double det = a11 * a22 - a12 * a12;
  if (!(det != 0.0) || !isfinite(det)) {
    active = false;
  } else {
    double dx = (a22 * fx - a12 * fy) / det, dy = (a11 * fy - a12 * fx) / det;
    const double len = sqrt(dx * dx + dy * dy);
    if (len > c.step_max) {
      dx *= c.step_max / len;
      dy *= c.step_max / len;
    }
    tx += dx;
    ty += dy;
    h.tx = tx;
    h.ty = ty;
    h.h11 = (float)m11;
    h.h22 = (float)m22;
    h.h12 = (float)m12;
    if (!isfinite(tx) || !isfinite(ty)) {
      active = false;
    } else if (len < NEWTON32_TOL && ++settled > LENS_NEWTON_EXTRA) {
      status = ST_NEWTON;
      active = false;
    }
  }
  if (active && ++nit < NEWTON_MAXIT) return true;
  // a root far from its triangle belongs to another triangle's search
  if (status == ST_NEWTON && hypot(tx - h.cx, ty - h.cy) > c.local) status = ST_FAR;
  h.status = status;
  return false;
#endif
}

// Newton round `round` after its points were evaluated: a step per
// candidate; those still iterating join the next round, after the last
// round the stragglers.
__global__ void __launch_bounds__(RL_THREADS) k_ref_newton(const SetArgs a, const NewtonArgs n, int round) {
  const size_t N = (size_t)a.B * IMG_CAP;
  // rounds alternate between the lists at 6N and 7N; the stragglers' is at 8N
  const int *lst = a.s.lst + (6 + (round & 1)) * N;
  int *nxt = a.s.lst + (round + 1 < NEWTON_ROUNDS ? 6 + ((round + 1) & 1) : 8) * N;
  int *cnt = a.s.lcnt;
  int *ncnt = &cnt[round + 1 < NEWTON_ROUNDS ? SUBDIV_LEVELS + round + 1 : SUBDIV_LEVELS + NEWTON_ROUNDS];
  const int npts = cnt[SUBDIV_LEVELS + round];
  for (int p = blockIdx.x * RL_THREADS + threadIdx.x; p < npts; p += gridDim.x * RL_THREADS) {
    const int slot = lst[p] >> 2;
    const CandCtx c = cand_ctx(a, n, slot);
    Ref &R = a.s.ref[slot];
    double tx = a.s.hits[slot].tx, ty = a.s.hits[slot].ty;
    int nit = R.nit, settled = R.settled;
    const bool go = newton_step(a, slot, c, R.mo, tx, ty, nit, settled);
    R.nit = nit;
    R.settled = settled;
    if (go) nxt[atomicAdd(ncnt, 1)] = slot << 2 | 3;
  }
}

// The stragglers: RS_GROUPS groups of RS_GROUP threads per CTA, each group
// one candidate at a time, each evaluation a group-wide sweep -- the threads
// split the static FP32 potentials (records staged in shared memory once per
// CTA when they fit, else read from global memory), threads j < n_heavy take
// the static cluster-scale ones in double-float, the group's last two
// threads the varying ones in FP32 (here the step's latency matters more
// than the root's last digits: the polish refines it in double-float) -- a
// fixed-order group sum in FP64, then the same Newton step.  Its pace is the
// latency of a step times the steps of the group's candidates (~40 for one
// that never converges), so the CTA runs several groups side by side.
constexpr int RS_THREADS = 256, RS_GROUP = 128, RS_GROUPS = RS_THREADS / RS_GROUP, RS_GWARPS = RS_GROUP / 32;
constexpr size_t RS_SMEM_MAX = 200 * 1024;
__host__ __device__ constexpr size_t straggle_smem(int n_light) { return (size_t)n_light * (REC32 * 4 + 16); }
// barrier of group g (barrier 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(RS_GROUP) : "memory"); }

__global__ void __launch_bounds__(RS_THREADS) k_ref_straggle(const SetArgs a, const NewtonArgs n, int staged) {
  extern __shared__ __align__(16) float4 s_dyn[];
  __shared__ float2 s_red[RS_GROUPS][RS_GWARPS][5];
  __shared__ int s_go[RS_GROUPS], s_next[RS_GROUPS];
  __shared__ double s_pos[RS_GROUPS][2];                         // the candidate's position
  __shared__ __align__(16) float s_var[RS_GROUPS][2][REC32 + 4];  // its varying potentials' FP32 records + centres
  const size_t N = (size_t)a.B * IMG_CAP;
  const int *lst = a.s.lst + 8 * N;
  const int nst = a.s.lcnt[SUBDIV_LEVELS + NEWTON_ROUNDS];
  if ((int)blockIdx.x * RS_GROUPS >= nst) return;  // uniform over the CTA
  const int nl = n.n_light;
  const float4 *g_rec = reinterpret_cast<const float4 *>(n.rec32);
  const float4 *g_cen = reinterpret_cast<const float4 *>(n.cen32);
  if (staged) {
    float4 *sr = s_dyn, *sc = s_dyn + (size_t)nl * (REC32 / 4);
    for (int i = threadIdx.x; i < nl * (REC32 / 4); i += RS_THREADS) sr[i] = g_rec[i];
    for (int i = threadIdx.x; i < nl; i += RS_THREADS) sc[i] = g_cen[i];
    __syncthreads();
  }
  const int g = threadIdx.x / RS_GROUP, tid = threadIdx.x % RS_GROUP, lane = tid & 31, w = tid >> 5;
  int *next = &a.s.lcnt[LCNT - 1];  // the next straggler a group takes (groups that finish early take more)
  for (;;) {
    if (tid == 0) s_next[g] = atomicAdd(next, 1);
    group_sync(g);
    const int p = s_next[g];
    group_sync(g);  // s_next is rewritten by the group's next fetch
    if (p >= nst) break;  // uniform over the group
    const int slot = lst[p] >> 2;
    const CandCtx c = cand_ctx(a, n, slot);
    const VarRecs &var = a.s.var[slot / IMG_CAP];
    // the iteration state lives on chip: thread 0 keeps the counters, the
    // group reads the position and the varying records from shared memory
    double tx = 0.0, ty = 0.0;
    int nit = 0, settled = 0;
    if (tid == 0) {
      tx = a.s.hits[slot].tx;
      ty = a.s.hits[slot].ty;
      nit = a.s.ref[slot].nit;
      settled = a.s.ref[slot].settled;
      s_pos[g][0] = tx;
      s_pos[g][1] = ty;
    }
    for (int i = tid; i < 2 * (REC32 + 4); i += RS_GROUP) {
      const int v = i / (REC32 + 4), k = i % (REC32 + 4);
      s_var[g][v][k] = k < REC32 ? var.r32[v][k] : var.cen[v][k - REC32];
    }
    group_sync(g);
    for (;;) {
      const double X = s_pos[g][0], Y = s_pos[g][1];
      const float hx = (float)X, lx = (float)(X - (double)hx), hy = (float)Y, ly = (float)(Y - (double)hy);
      Acc<true, 1> tot, cmp, part;
      tot.zero();
      cmp.zero();
      part.zero();
      int seen = 0;
      // the static potentials: from the staged copy through shared-memory
      // loads (a pointer that may be either would compile to generic loads)
      auto sweep = [&](const float4 *rc, const float4 *cn) {
        for (int j = tid; j < nl; j += RS_GROUP) {
          const float4 cc = cn[j];
          const float dY[1] = {(hy - cc.y) + (ly - cc.w)};
          eval32_any<true, 1>(rc + (size_t)j * (REC32 / 4), (hx - cc.x) + (lx - cc.z), dY, part);
          if (++seen == PE_SUB) {
            fold(tot, cmp, part);
            seen = 0;
          }
        }
      };
      if (staged)
        sweep(s_dyn, s_dyn + (size_t)nl * (REC32 / 4));
      else
        sweep(g_rec, g_cen);
      if (tid >= RS_GROUP - 2) {  // the varying potentials join the FP32 sums
        const int vv = tid - (RS_GROUP - 2);
        const float *cv = &s_var[g][vv][REC32];
        const float dY[1] = {(float)(Y - ((double)cv[1] + (double)cv[3]))};
        eval32_any<true, 1>(reinterpret_cast<const float4 *>(&s_var[g][vv][0]),
                            (float)(X - ((double)cv[0] + (double)cv[2])), dY, part);
      }
      fold(tot, cmp, part);
      // each thread's compensated sum as a float pair, summed over the group
      // in double-float (FP32 pipe) in a fixed order: warp butterflies, then
      // the group's warps in order
      df v2[5] = {{tot.ax[0], -cmp.ax[0]}, {tot.ay[0], -cmp.ay[0]}, {tot.k[0], -cmp.k[0]},
                  {tot.g1[0], -cmp.g1[0]}, {tot.g2[0], -cmp.g2[0]}};
#pragma unroll
      for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const df t = {__shfl_xor_sync(0xffffffffu, v2[q].hi, o), __shfl_xor_sync(0xffffffffu, v2[q].lo, o)};
          v2[q] = df_add(v2[q], t);
        }
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 5; ++q) s_red[g][w][q] = make_float2(v2[q].hi, v2[q].lo);
      group_sync(g);
      if (tid == 0) {
        double v[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          df t = {s_red[g][0][q].x, s_red[g][0][q].y};
          for (int k = 1; k < RS_GWARPS; ++k) t = df_add(t, df{s_red[g][k][q].x, s_red[g][k][q].y});
          v[q] = df_to_double(t);
        }
        for (int j = 0; j < n.n_heavy; ++j)  // static cluster-scale potentials (double-float)
          add_potential_df<true>(n.heavydf + (size_t)j * RECDF, 1, n.heavy + (size_t)j * REC64, X, Y, v);
        const bool more = newton_step(a, slot, c, v, tx, ty, nit, settled);
        s_pos[g][0] = tx;
        s_pos[g][1] = ty;
        s_go[g] = more ? 1 : 0;
        if (!more) {
          a.s.ref[slot].nit = nit;
          a.s.ref[slot].settled = settled;
        }
      }
      group_sync(g);
      const bool go = s_go[g] != 0;
      group_sync(g);  // s_red, s_go and s_pos are rewritten by the next step
      if (!go) break;
    }
  }
}

// ------------------------------------------------------------------ 4. dedup
// The walk of one source's candidates in candidate order that keeps those
// not within DEDUP of a candidate it already kept (the definition's rule for
// the images it finds).  s_src[u] is candidate u's source (-1: not taken);
// pos(u, x, y) its position; kept candidates get s_flag[u] = 1.  Up to
// KW_LIST candidates are listed first (a scan of shared memory only); the
// first KW_KEEP kept positions are held in w.kx, w.ky, later ones re-read.
constexpr int KW_LIST = 128, KW_KEEP = 16;
struct KeepWalk {
  int lst[KW_LIST];
  double kx[KW_KEEP], ky[KW_KEEP];
  int nl, nc, nk;
  bool listed;
  __device__ __forceinline__ int cand(int k) const { return listed ? lst[k] : k; }
};
template <class Pos>
__device__ __forceinline__ void keep_walk(KeepWalk &w, int i, int n, const int *s_src, unsigned char *s_flag,
                                          Pos pos) {
  w.nl = 0;
  for (int u = 0; u < n; ++u)
    if (s_src[u] == i) {
      if (w.nl < KW_LIST) w.lst[w.nl] = u;
      ++w.nl;
    }
  w.listed = w.nl <= KW_LIST;
  w.nc = w.listed ? w.nl : n;  // candidates walked: the list, or every staged one
  w.nk = 0;
  for (int k = 0; k < w.nc; ++k) {
    const int u = w.cand(k);
    if (s_src[u] != i) continue;
    double tx, ty;
    pos(u, tx, ty);
    bool near = false;
    for (int q = 0; q < w.nk && q < KW_KEEP && !near; ++q) {
      const double ex = w.kx[q] - tx, ey = w.ky[q] - ty;
      near = ex * ex + ey * ey < DEDUP * DEDUP;
    }
    if (w.nk > KW_KEEP)  // kept candidates past the first KW_KEEP
      for (int q = 0, seen = 0; q < k && !near; ++q) {
        const int v = w.cand(q);
        if (s_src[v] != i || !s_flag[v] || ++seen <= KW_KEEP) continue;
        double vx, vy;
        pos(v, vx, vy);
        const double ex = vx - tx, ey = vy - ty;
        near = ex * ex + ey * ey < DEDUP * DEDUP;
      }
    if (near) continue;
    s_flag[u] = 1;
    if (w.nk < KW_KEEP) {
      w.kx[w.nk] = tx;
      w.ky[w.nk] = ty;
    }
    ++w.nk;
  }
}

constexpr int DD_THREADS = 256;

// Candidates that reached a root: a thread per source keeps, in candidate
// order, those not within DEDUP of one it kept (keep_walk); the kept ones'
// indices are then compacted in candidate order.
__global__ void __launch_bounds__(DD_THREADS) k_img_dedup(const SetArgs a) {
  __shared__ int s_scan[DD_THREADS];
  __shared__ int s_base;
  __shared__ int s_isrc[IMG_CAP];
  __shared__ unsigned char s_keep[IMG_CAP];
  const int b = blockIdx.x;
  if (!a.s.valid[b]) return;
  const int n = min(a.s.cnt[b], IMG_CAP);
  const Hit *hits = a.s.hits + (size_t)b * IMG_CAP;
  int *uniq = a.s.uniq + (size_t)b * IMG_CAP;
  for (int k = threadIdx.x; k < n; k += DD_THREADS) {
    s_isrc[k] = hits[k].status == ST_NEWTON ? hits[k].src : -1;
    s_keep[k] = 0;
  }
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < a.nsrc; i += DD_THREADS) {
    KeepWalk w;
    keep_walk(w, i, n, s_isrc, s_keep, [&](int u, double &x, double &y) {
      x = hits[u].tx;
      y = hits[u].ty;
    });
  }
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += DD_THREADS) {
    const int k = k0 + threadIdx.x;
    const int keep = k < n ? s_keep[k] : 0;
    // inclusive scan of keep flags (Hillis-Steele), keeps the candidates' order
    s_scan[threadIdx.x] = keep;
    __syncthreads();
    for (int o = 1; o < DD_THREADS; o <<= 1) {
      const int t = threadIdx.x >= o ? s_scan[threadIdx.x - o] : 0;
      __syncthreads();
      s_scan[threadIdx.x] += t;
      __syncthreads();
    }
    if (keep) uniq[s_base + s_scan[threadIdx.x] - 1] = k;
    __syncthreads();
    if (threadIdx.x == DD_THREADS - 1) s_base += s_scan[DD_THREADS - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.s.nuniq[b] = s_base;
}

// ----------------------------------------------------------------- 5. polish
#ifndef LENS_POLISH_MINB
#define LENS_POLISH_MINB 2  // resident CTAs per SM the polish is compiled for (3: same speed, spills)
#endif
__global__ void __launch_bounds__(NW_THREADS, LENS_POLISH_MINB) k_img_polish(const SetArgs a, const NewtonArgs n) {
  __shared__ double s_var[NW_WARPS][2 * REC64];
  __shared__ float2 s_vdf[NW_WARPS][2 * RECDF];
  __shared__ int s_q[NW_WARPS][64];  // potentials left to the FP64 evaluator
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * NW_WARPS;
  const int ntot = n.n_stat + 2;
  for (long long task = (long long)blockIdx.x * NW_WARPS + w; task < (long long)a.B * IMG_CAP; task += nwarps) {
    const int b = (int)(task / IMG_CAP), u = (int)(task % IMG_CAP);
    if (!a.s.valid[b] || u >= a.s.nuniq[b]) continue;
    Hit *h = a.s.hits + (size_t)b * IMG_CAP + a.s.uniq[(size_t)b * IMG_CAP + u];
    if (lane < 2 * REC64) s_var[w][lane] = a.s.var[b].r64[lane / REC64][lane % REC64];
    for (int i = lane; i < 2 * RECDF; i += 32) s_vdf[w][i] = a.s.var[b].rdf[i / RECDF][i % RECDF];
    __syncwarp();
    const int src = h->src;
    const double r = n.ratio[src];
    const double bx = a.s.bary[((size_t)b * a.nsrc + src) * 2], by = a.s.bary[((size_t)b * a.nsrc + src) * 2 + 1];
    const double a11 = 1.0 - h->h11, a22 = 1.0 - h->h22, a12 = -h->h12;
    const double det = a11 * a22 - a12 * a12, idet = 1.0 / det;
    // (steps compared squared: no FP64 root or division in the iteration,
    // whose FP64 tail is a serial chain on this GPU's narrow FP64 unit)
    double tx = h->tx, ty = h->ty, step2 = 1e60;
    for (int it = 0; it < POLISH_MAXIT && step2 >= POLISH_TOL * POLISH_TOL; ++it) {
      // alpha(tx, ty): dPIE terms inside the polynomial range in
      // double-float; the rest (cores: |w|^2 >= 0.16, SIS, point masses)
      // queued and evaluated 32 at a time, so the warp stays converged, by
      // the double-float reductions of atan/atanh (FP64 only if those fail)
      const df X = df_from_double(tx), Y = df_from_double(ty);
      df fx = {0.f, 0.f}, fy = {0.f, 0.f};
      double sx = 0.0, sy = 0.0;
      int nq = 0;
      auto queued = [&](int jj) {
        const bool stq = jj < n.n_stat;
        const float2 *rec = stq ? n.recdf + jj : s_vdf[w] + (jj - n.n_stat) * RECDF;
        const int stride = stq ? n.n_stat : 1;
        df gx, gy;
        if (rec[F_U2 * stride].x < 0.f) {
          circ_df(rec, stride, X, Y, gx, gy);
        } else if (!dpie_df<true>(rec, stride, X, Y, gx, gy)) {
          const double *r64 = stq ? n.all64 + (size_t)jj * REC64 : s_var[w] + (jj - n.n_stat) * REC64;
          double ex, ey, e2, e3, e4;
          eval64<false>(r64, tx, ty, ex, ey, e2, e3, e4);
          sx += ex;
          sy += ey;
          return;
        }
        fx = df_add(fx, gx);
        fy = df_add(fy, gy);
      };
      for (int base = 0; base < ntot; base += 32) {
        const int j = base + lane;
        bool need = false;
        if (j < ntot) {
          const bool st = j < n.n_stat;
          const float2 *rec = st ? n.recdf + j : s_vdf[w] + (j - n.n_stat) * RECDF;
          const int stride = st ? n.n_stat : 1;
          df gx, gy;
          if (rec[F_U2 * stride].x >= 0.f && dpie_df<false>(rec, stride, X, Y, gx, gy)) {
            // one-TwoSum accumulation: absolute error 2^-47 sum |alpha_i|,
            // a few 1e-13 arcsec over a cluster
            fx = df_add_ss(fx, gx);
            fy = df_add_ss(fy, gy);
          } else {
            need = true;
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (need) s_q[w][nq + __popc(m & ((1u << lane) - 1u))] = j;
        nq += __popc(m);
        if (nq >= 32) {
          __syncwarp();
          queued(s_q[w][nq - 32 + lane]);
          nq -= 32;
          __syncwarp();
        }
      }
      __syncwarp();
      if (lane < nq) queued(s_q[w][lane]);
      __syncwarp();
      sx = warp_sum(sx + df_to_double(fx));
      sy = warp_sum(sy + df_to_double(fy));
      const double fxr = bx - (tx - r * sx), fyr = by - (ty - r * sy);
      const double dx = (a22 * fxr - a12 * fyr) * idet, dy = (a11 * fyr - a12 * fxr) * idet;
      tx += dx;
      ty += dy;
      step2 = dx * dx + dy * dy;
    }
    if (lane == 0) {
      h->tx = tx;
      h->ty = ty;
      h->status = (step2 < ACCEPT_TOL * ACCEPT_TOL && isfinite(tx) && isfinite(ty)) ? ST_FINAL : ST_NO_POLISH;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------- 6. match, chi2
constexpr int C2_THREADS = 128;

__global__ void __launch_bounds__(C2_THREADS) k_img_chi2(const SetArgs a, const double *__restrict__ x,
                                                         const double *__restrict__ y,
                                                         const double *__restrict__ sigma,
                                                         const int32_t *__restrict__ img_off, double *chi2,
                                                         int32_t *nfound, int *err, double *images, int img_max,
                                                         int32_t *img_count) {
  __shared__ double s_red[C2_THREADS / 32];
  const int b = blockIdx.x, p = a.p0 + b;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (!a.s.valid[b]) {
    if (threadIdx.x == 0) {
      if (chi2) chi2[p] = nan;
      if (img_count) img_count[p] = 0;
    }
    if (nfound)
      for (int i = threadIdx.x; i < a.nsrc; i += C2_THREADS) nfound[(size_t)p * a.nsrc + i] = 0;
    return;
  }
  const bool overflow = a.s.cnt[b] > IMG_CAP;
  const Hit *hits = a.s.hits + (size_t)b * IMG_CAP;
  const int *uniq = a.s.uniq + (size_t)b * IMG_CAP;
  const int nu = a.s.nuniq[b];
  // Final images: polished, and not within DEDUP of an earlier final image of
  // the same source (candidates of one highly magnified image can end the
  // FP32 Newton further apart than DEDUP and meet only after the polish).
  // Each image's source is staged (-1: not polished); a thread per source
  // keeps its images (keep_walk: in candidate order, those not within DEDUP
  // of one already kept), counts them and matches its constraints to them.
  __shared__ unsigned char s_use[IMG_CAP];
  __shared__ int s_isrc[IMG_CAP];
  for (int u = threadIdx.x; u < nu; u += C2_THREADS) {
    const Hit &h = hits[uniq[u]];
    s_isrc[u] = h.status == ST_FINAL ? h.src : -1;
    s_use[u] = 0;
  }
  __syncthreads();
  double acc[1] = {0.0};
  auto pos = [&](int u, double &x, double &y) {
    x = hits[uniq[u]].tx;
    y = hits[uniq[u]].ty;
  };
  for (int i = threadIdx.x; i < a.nsrc; i += C2_THREADS) {
    KeepWalk w;
    keep_walk(w, i, nu, s_isrc, s_use, pos);
    if (nfound) nfound[(size_t)p * a.nsrc + i] = overflow ? -1 : w.nk;
    // each constraint of the source: the nearest kept image (ties: lower y,
    // then lower x)
    for (int j = img_off[i]; j < img_off[i + 1]; ++j) {
      double best = INFINITY, bx = 0.0, by = 0.0;
      auto consider = [&](double tx, double ty) {
        const double ex = x[j] - tx, ey = y[j] - ty, d2 = ex * ex + ey * ey;
        if (d2 < best || (d2 == best && (ty < by || (ty == by && tx < bx)))) {
          best = d2;
          bx = tx;
          by = ty;
        }
      };
      for (int k = 0; k < w.nk && k < KW_KEEP; ++k) consider(w.kx[k], w.ky[k]);
      if (w.nk > KW_KEEP)
        for (int k = 0, seen = 0; k < w.nc; ++k) {
          const int v = w.cand(k);
          if (s_isrc[v] != i || !s_use[v] || ++seen <= KW_KEEP) continue;
          double vx, vy;
          pos(v, vx, vy);
          consider(vx, vy);
        }
      acc[0] += best / (sigma[j] * sigma[j]);  // no image of this source: +inf -> NaN below
    }
  }
  __syncthreads();  // s_use complete
  if (images && threadIdx.x == 0) {  // predicted images, in candidate order
    int c = 0;
    for (int u = 0; u < nu; ++u) {
      if (!s_use[u]) continue;
      if (c < img_max) {
        const Hit &h = hits[uniq[u]];
        double *o = images + ((size_t)p * img_max + c) * 3;
        o[0] = h.tx;
        o[1] = h.ty;
        o[2] = (double)h.src;
      }
      ++c;
    }
    img_count[p] = overflow ? -1 : c;
  }
  block_sum<1, C2_THREADS>(acc, s_red);
  if (threadIdx.x == 0) {
    if (chi2) chi2[p] = (overflow || !isfinite(acc[0])) ? nan : acc[0];
    if (overflow) atomicOr(err, ERRBIT_CAPACITY);
  }
}

}  // namespace

size_t chi2_image_scratch_bytes(const CSet *c, int32_t batch, bool lists) {
  return layout(batch, c->nsrc, lists).total;
}

int run_chi2_image(lens_ctx *ctx, CSet *c, const GridCache *gc, const double *d_params, int32_t P, double *d_chi2,
                   int32_t *d_nfound, void *scratch, int32_t batch, cudaStream_t st, double *d_images,
                   int32_t img_max, int32_t *d_img_count, bool lists) {
  {
    // every caller (the entry points, the request loop, the allocation-free
    // path) passes through here: refuse what the kernels' fixed shared
    // arrays cannot hold before anything is launched
    lens_grid g;
    g.xmin = gc->xmin;
    g.xmax = gc->xmax;
    g.ymin = gc->ymin;
    g.ymax = gc->ymax;
    g.nx = gc->nx;
    g.ny = gc->ny;
    const int lim = check_chi2_image_limits(c, &g);
    if (lim) return lim;
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  const Model *sm = c->stat_model;
  NewtonArgs n;
  n.rec32 = sm->rec32;
  n.cen32 = sm->cen32;
  n.n_light = sm->n_light;
  for (int k = 0; k < 5; ++k) n.koff[k] = sm->koff[k];
  n.heavy = sm->heavy;
  n.heavydf = sm->heavydf;
  n.n_heavy = sm->n_heavy;
  n.all64 = sm->all64;
  n.recdf = sm->recdf;
  n.n_stat = sm->n;
  n.ratio = c->ratio;
  n.xmin = gc->xmin;
  n.ymin = gc->ymin;
  n.dx = (gc->xmax - gc->xmin) / (gc->nx - 1);
  n.dy = (gc->ymax - gc->ymin) / (gc->ny - 1);
  n.nx = gc->nx;
  n.gax = gc->alpha32;
  n.gay = gc->alpha32 + (size_t)gc->nx * gc->ny;
  n.err = ctx->d_err;
  SearchArgs g;
  g.ax = gc->alpha32;
  g.ay = gc->alpha32 + (size_t)gc->nx * gc->ny;
  g.xmin = gc->xmin;
  g.ymin = gc->ymin;
  g.dx = (gc->xmax - gc->xmin) / (gc->nx - 1);
  g.dy = (gc->ymax - gc->ymin) / (gc->ny - 1);
  g.nx = gc->nx;
  g.ny = gc->ny;
  g.grp_off = c->grp_off;
  g.grp_src = c->grp_src;
  g.grp_r32 = c->grp_ratio32;
  g.ng = c->ng;
  g.fdx = (float)g.dx;
  g.fdy = (float)g.dy;
  g.tiny = (float)(1e-10 * g.dx * g.dy);
  const size_t src_smem = sizeof(double) * (2 * REC64 + 2 * (size_t)c->nimg + 2 * (size_t)c->nsrc);
  cudaFuncSetAttribute(k_img_sources, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)IMG_SRC_SMEM_MAX);
  for (int32_t p0 = 0; p0 < P; p0 += batch) {
    SetArgs a;
    a.params = d_params;
    a.p0 = p0;
    a.B = std::min(batch, P - p0);
    a.type0 = c->var_type[0];
    a.type1 = c->var_type[1];
    a.nsrc = c->nsrc;
    a.nimg = c->nimg;
    a.s = bufs(scratch, batch, c->nsrc, lists);
    k_img_sources<<<a.B, SRC_THREADS, src_smem, st>>>(a, c->stat, c->x, c->y, c->ratio, c->src_of, c->img_off);
    dim3 sg((gc->nx - 1 + CT_X - 1) / CT_X, (gc->ny - 1 + CT_Y - 1) / CT_Y, a.B);
    k_img_search<<<sg, SEARCH_THREADS, 0, st>>>(a, g);
    if (LENS_REFINE_LISTS && lists) {
      // step 3 as point lists: the list counters, the initial triangles,
      // one evaluation + decision pair per subdivision level and Newton
      // round (the grids of the evaluations cover the largest lists; CTAs
      // past a list's end return at once), the stragglers
      if (cudaMemsetAsync(a.s.lcnt, 0, LCNT * sizeof(int), st) != cudaSuccess)
        return fail(LENS_ECUDA, "cudaMemsetAsync failed");
      k_ref_init<<<dim3((IMG_CAP + RL_THREADS - 1) / RL_THREADS, a.B), RL_THREADS, 0, st>>>(a, n);
      const size_t N = (size_t)a.B * IMG_CAP;
      const unsigned gsub = (unsigned)((3 * N + pe_points(false) - 1) / pe_points(false));
      const unsigned gnew = (unsigned)((N + pe_points(true) - 1) / pe_points(true));
      for (int lev = 0; lev < SUBDIV_LEVELS; ++lev) {
        k_pts_eval<false><<<gsub, PE_THREADS, 0, st>>>(a, n, a.s.lst + ((lev & 1) ? 3 * N : 0), a.s.lcnt + lev);
        k_ref_level<<<4 * nsm, RL_THREADS, 0, st>>>(a, n, lev);
      }
      for (int r = 0; r < NEWTON_ROUNDS; ++r) {
        k_pts_eval<true><<<gnew, PE_THREADS, 0, st>>>(a, n, a.s.lst + (6 + (r & 1)) * N,
                                                      a.s.lcnt + SUBDIV_LEVELS + r);
        k_ref_newton<<<4 * nsm, RL_THREADS, 0, st>>>(a, n, r);
      }
      const size_t rs_smem = straggle_smem(sm->n_light);
      const int staged = rs_smem <= RS_SMEM_MAX;
      if (staged) cudaFuncSetAttribute(k_ref_straggle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SMEM_MAX);
      k_ref_straggle<<<nsm, RS_THREADS, staged ? rs_smem : 0, st>>>(a, n, staged);
    } else {
      k_img_newton<<<dim3(IMG_CAP / RF_CAND, a.B), RF_THREADS, 0, st>>>(a, n);
    }
    k_img_dedup<<<a.B, DD_THREADS, 0, st>>>(a);
    k_img_polish<<<nsm * 8, NW_THREADS, 0, st>>>(a, n);
    k_img_chi2<<<a.B, C2_THREADS, 0, st>>>(a, c->x, c->y, c->sigma, c->img_off, d_chi2, d_nfound, ctx->d_err,
                                           d_images, img_max, d_img_count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LENS_ECUDA, "image-plane chi2 launch: %s", cudaGetErrorString(e));
  }
  return LENS_OK;
}

const GridCache *find_grid_cache(const CSet *c, const lens_grid *g) {
  for (auto &x : c->grids)
    if (x.xmin == g->xmin && x.xmax == g->xmax && x.ymin == g->ymin && x.ymax == g->ymax && x.nx == g->nx &&
        x.ny == g->ny)
      return &x;
  return nullptr;
}

// Static deflection of the constraint set's model on grid g (LENS_MIXED map
// of the static potentials, D_ls/D_s = 1), enqueued on st and kept with the
// constraint set.
int build_grid_cache(lens_ctx *ctx, CSet *c, const lens_grid *g, cudaStream_t st) {
  GridCache n;
  n.xmin = g->xmin;
  n.xmax = g->xmax;
  n.ymin = g->ymin;
  n.ymax = g->ymax;
  n.nx = g->nx;
  n.ny = g->ny;
  n.bytes = 2 * sizeof(float) * (size_t)g->nx * g->ny;
  int rc = dev_alloc(ctx, (void **)&n.alpha32, n.bytes);
  if (rc) return rc;
  if (c->stat_model->n > 0)
    rc = launch_map_mixed(ctx, c->stat_model, g, 1.0, false, n.alpha32, st, 0, -1, false);
  else
    rc = cudaMemsetAsync(n.alpha32, 0, n.bytes, st) == cudaSuccess ? LENS_OK : fail(LENS_ECUDA, "memset failed");
  if (rc) {
    dev_free(ctx, n.alpha32, n.bytes);
    return rc;
  }
  c->grids.push_back(n);
  return LENS_OK;
}

int check_chi2_image_limits(const CSet *c, const lens_grid *g) {
  if (c->nsrc > MAX_SRC) return fail(LENS_EINVAL, "image-plane chi2 supports at most %d sources", MAX_SRC);
  const size_t src_smem = sizeof(double) * (2 * REC64 + 2 * (size_t)c->nimg + 2 * (size_t)c->nsrc);
  if (src_smem > IMG_SRC_SMEM_MAX)
    return fail(LENS_EINVAL, "constraint set too large for one CTA (%d images)", c->nimg);
  if ((long long)(g->nx - 1) * (g->ny - 1) > (1ll << 30)) return fail(LENS_EINVAL, "grid too large");
  return LENS_OK;
}

int launch_chi2_image(lens_ctx *ctx, const Model *m, CSet *c, const lens_grid *g, const double *d_params, int32_t P,
                      double *d_chi2, int32_t *d_nfound, cudaStream_t st, double *d_images, int32_t img_max,
                      int32_t *d_img_count) {
  (void)m;
  int lim = check_chi2_image_limits(c, g);
  if (lim) return lim;
  const GridCache *gc = find_grid_cache(c, g);
  if (!gc) {
    int rc = build_grid_cache(ctx, c, g, st);
    if (rc) return rc;
    gc = find_grid_cache(c, g);
  }
  const int32_t batch = std::min<int32_t>(IMG_BATCH, P);
  CallScratch scratch(ctx, st);  // this call's candidate buffers, on its own stream
  const int rc = scratch.alloc(chi2_image_scratch_bytes(c, batch));
  if (rc) return rc;
  return run_chi2_image(ctx, c, gc, d_params, P, d_chi2, d_nfound, scratch.p, batch, st, d_images, img_max,
                        d_img_count);
}

}  // namespace lens
