// Map kernels: deflection (Sec. 4.1, Eq. 10) and deflection + Hessian maps
// (Sec. 2.4, Eqs. 7-9; magnification Sec. 2.1, Eqs. 4-5) over a rectangular
// grid with inclusive corners.
//
// LENS_MIXED kernel (the hot path):
//   - CTA = 128 threads = 4 warps over a 32 x (4 KP) point tile; lane l owns
//     column i0 + l, warp w owns rows j0 + w KP .. + KP-1, so every store of
//     one row is 32 consecutive elements (one 128-byte segment per warp).
//   - Potentials evaluated in FP32 are streamed through shared memory in
//     chunks of CH packed 128-byte records by 1-D bulk copies (TMA,
//     cp.async.bulk + mbarrier), double-buffered: the copy of chunk c+1 is in
//     flight while chunk c is evaluated.  Every thread reads the same record
//     at the same time (shared-memory broadcast).
//   - Point positions relative to each potential: per (tile, potential), the
//     tile origin's X - x0 and Y - y0 in FP64, kept as hi/lo float pairs; a
//     lane adds its column offset (also a hi/lo pair) to the first, and the
//     staging adds each row's offset to the second, so (hi + offset) is
//     exact next to a potential's centre (Sterbenz) and dX, dY keep FP32
//     relative precision there, before rotating into its frame.
//   - FP32 contributions go into naive partial sums that are folded every
//     SUB potentials into a Kahan-compensated total.
//   - Potentials at or above the FP64 threshold (cluster-scale halos) are
//     evaluated in FP64; the final sum, scaling by D_ls/D_s and the derived
//     kappa/gamma/mu are formed in FP64 per point and stored as FP32.
// LENS_FP64 kernel: one point per thread, every potential in FP64.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "lens_device.cuh"

namespace lens {
namespace {

// Launch shape (overridable at build time for tuning): CTAs per SM the
// register budget targets, and points per thread of the Hessian and
// deflection-only kernels.
#ifndef LENS_MAP_MINB
#define LENS_MAP_MINB 4     // Hessian kernel (128-thread CTAs)
#endif
#ifndef LENS_MAP_MINB_GRAD
#define LENS_MAP_MINB_GRAD 6  // deflection-only kernel (128-thread CTAs)
#endif
#ifndef LENS_MAP_MINB_POT
#define LENS_MAP_MINB_POT 4  // potential kernel (126 registers; 6 CTAs/SM at 80: 8.37 against 7.98 ms)
#endif
#ifndef LENS_MAP_SEGMENTS
#define LENS_MAP_SEGMENTS 1  // kind-uniform loops over each chunk's potentials
#endif
#ifndef LENS_MAP_SEGMENTS_GRAD
#define LENS_MAP_SEGMENTS_GRAD 0  // the same in the deflection-only kernel (measured slower: it spills)
#endif
#ifndef LENS_POT_PAIRED
#define LENS_POT_PAIRED 1  // potential map on the paired FP32 path
#endif
#ifndef LENS_MAP_UNROLL
#define LENS_MAP_UNROLL 2  // potentials per iteration of those loops (2: 0.6 % faster than 4 at 128 threads)
#endif
#ifndef LENS_KP_HESS
#define LENS_KP_HESS 2
#endif
#ifndef LENS_KP_GRAD
#define LENS_KP_GRAD 4
#endif
// threads per CTA, one warp per KP rows of the tile (128 measured 3 % faster
// than 256 for both kernels at the same warps per SM, 64 slower)
#ifndef LENS_MAP_THREADS_HESS
#define LENS_MAP_THREADS_HESS 128
#endif
#ifndef LENS_MAP_THREADS_GRAD
#define LENS_MAP_THREADS_GRAD 128
#endif
__host__ __device__ constexpr int map_threads(bool hess) { return hess ? LENS_MAP_THREADS_HESS : LENS_MAP_THREADS_GRAD; }
static_assert(map_threads(true) >= 64 && map_threads(false) >= 64 && map_threads(true) % 32 == 0 &&
                  map_threads(false) % 32 == 0,
              "the chunk staging uses 64 threads");
constexpr int MAP_UNROLL = LENS_MAP_UNROLL;
constexpr int CH = 64;   // potentials per staged chunk (8 KB of records)
#ifndef LENS_MAP_SUB
#define LENS_MAP_SUB 16
#endif
constexpr int SUB = LENS_MAP_SUB;  // partial sums folded into the compensated total every SUB potentials
// Repair of the Hessian maps' det = 1/mu: the FP32 terms' relative error
// (measured below 2e-7 of each term) and the det error above which a node is
// recomputed in double-float (a third of the 3e-5 the maps are held to)
constexpr double DET_TERM_ERR = 2e-7, DET_REPAIR_ABS = 1e-5;

struct MapArgs {
  const float *rec32;
  const double *pos64;
  int n_light;
  int koff[5];  // light potentials of kind k (Kind32 order) are [koff[k], koff[k+1])
  const double *heavy;
  const float2 *heavydf;  // the same in double-float, record-major
  int n_heavy;
  int heavy_df;           // evaluate them in double-float instead of FP64 (deflection / Hessian maps)
  double xmin, ymin, dx, dy;
  int nx, ny;   // ny: rows computed by this launch
  int row0;     // grid row of the launch's first row (row bands of one grid)
  double dls;
  float *out;   // [planes][ny][nx] for the launch's rows
  long long plane;
  int *err;
  int tau;          // potential map: also the Fermat potential about (bx, by)
  double bx, by;
  double *out64;    // potential map: [1 or 2][ny][nx] doubles
  // deflection / Hessian maps: nodes where |alpha| < repair * (summed
  // magnitude of the FP32 terms) are appended to rep_list (count in
  // *rep_count) for the double-float repair pass; repair = 0: none
  double repair;
  float repair_f;  // 2 * repair (mag holds half the magnitude sum)
  int *rep_count, *rep_list;
};

// What a map computes: deflection, deflection + Hessian, or the potential.
enum MapMode : int { MAP_GRAD = 0, MAP_HESS = 1, MAP_POT = 2 };

// Point k of a thread's sums: plain per-point arrays (the potential map) or
// point pairs (the paired deflection / Hessian maps).
template <int N>
__device__ __forceinline__ float pt(const float (&v)[N], int k) { return v[k]; }
template <int N>
__device__ __forceinline__ float pt(const float2 (&v)[N], int k) { return part2(v[k >> 1], k & 1); }

template <int MODE, int KP>
__global__ void __launch_bounds__(map_threads(MODE == MAP_HESS), MODE == MAP_HESS  ? LENS_MAP_MINB
                                                                  : MODE == MAP_POT ? LENS_MAP_MINB_POT
                                                                                    : LENS_MAP_MINB_GRAD)
    k_map_mixed(const MapArgs a) {
  constexpr bool HESS = MODE == MAP_HESS, POT = MODE == MAP_POT;
  constexpr int MAP_THREADS = map_threads(HESS), MAP_WARPS = MAP_THREADS / 32;
  __shared__ __align__(128) float s_rec[2][CH * REC32];
  // Offsets of the tile from each staged potential's centre: X - x0 at the
  // tile's first column as a hi/lo float pair (a lane adds its column
  // offset), Y - y0 of every row of the tile rounded to float (rows are
  // per warp, so no per-thread work).  KP = 2: one float4 per (warp,
  // potential) = (x hi, x lo, y row 0, y row 1); KP = 4: the x pair per
  // potential and one float4 of rows per (warp, potential).
  static_assert(KP == 2 || KP == 4, "offset staging layout");
  constexpr int ROWS = MAP_WARPS * KP;
  __shared__ __align__(16) float4 s_offy[2][MAP_WARPS][CH];
  __shared__ __align__(8) float2 s_offx[2][KP == 2 ? 1 : CH];
  __shared__ float2 s_ly[ROWS];  // row r's offset r dy inside the tile, hi/lo
  __shared__ __align__(8) uint64_t s_bar[2];
  constexpr int NC = HESS ? 5 : POT ? 1 : 2;
  __shared__ double s_hv[MAP_THREADS][KP][NC];  // FP64 potentials' sums per point

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * (MAP_WARPS * KP);
  const double Tx = a.xmin + i0 * a.dx, Ty = a.ymin + (a.row0 + j0) * a.dy;
  // the point's offset inside the tile as a hi/lo float pair: (hi_off + hi_L)
  // is exact when the point is near the potential's centre (Sterbenz), so
  // dX, dY keep full relative precision where the profile is steepest
  const double lx = lane * a.dx;
  const float Lxh = (float)lx, Lxl = (float)(lx - (double)Lxh);
  if (tid < ROWS) {
    const double ly = tid * a.dy;
    const float h = (float)ly;
    s_ly[tid] = make_float2(h, (float)(ly - (double)h));
  }

  // deflection / Hessian: the thread's points as KP/2 pairs on the paired
  // FP32 path; the potential map: per point (POT: the potential in .k)
  constexpr int NP = KP / 2;
  constexpr bool POT1 = POT && !LENS_POT_PAIRED;  // the potential point by point
  using AccT = std::conditional_t<POT1, Acc<true, KP>, Acc2<HESS, NP>>;
  AccT tot, cmp, part;
  tot.zero();
  cmp.zero();
  part.zero();
  auto fold_all = [&]() {
    if constexpr (POT1)
      fold(tot, cmp, part);
    else if constexpr (POT)
      fold2_pot(tot, cmp, part);
    else
      fold2(tot, cmp, part);
  };

  // FP64 potentials (cluster scale), in FP64 or, when the model has few FP32
  // potentials per FP64 one, in double-float.  Half of the tiles evaluate
  // them before the FP32 loop, half after, so the CTAs sharing an SM rarely
  // load the FP64 pipe at the same time.
  auto heavy_pass = [&]() {
    const double X = a.xmin + (i0 + lane) * a.dx;
    if constexpr (!POT) {
      if (a.heavy_df) {
        // in double-float on the FP32 pipe (FP64 where that fails)
        const df Xd = df_from_double(X);
#pragma unroll 1
        for (int k = 0; k < KP; ++k) {
          const double Y = a.ymin + (a.row0 + j0 + warp * KP + k) * a.dy;
          const df Yd = df_from_double(Y);
          df sum[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
          for (int h = 0; h < a.n_heavy; ++h)
            add_potential_dfs<HESS>(a.heavydf + (size_t)h * RECDF, 1, a.heavy + (size_t)h * REC64, X, Y, Xd, Yd,
                                    sum);
#pragma unroll
          for (int c = 0; c < NC; ++c) s_hv[tid][k][c] = df_to_double(sum[c]);
        }
        return;
      }
    }
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const double Y = a.ymin + (a.row0 + j0 + warp * KP + k) * a.dy;
      double v[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = 0.0;
      for (int h = 0; h < a.n_heavy; ++h) {
        if constexpr (POT) {
          v[0] += pot64(a.heavy + (size_t)h * REC64, X, Y);
          continue;
        }
        double ax, ay, kk = 0, q1 = 0, q2 = 0;
        eval64<HESS>(a.heavy + (size_t)h * REC64, X, Y, ax, ay, kk, q1, q2);
        v[0] += ax;
        v[NC > 1 ? 1 : 0] += ay;
        if (HESS) {
          v[NC > 2 ? 2 : 0] += kk;
          v[NC > 3 ? 3 : 0] += q1;
          v[NC > 4 ? 4 : 0] += q2;
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) s_hv[tid][k][c] = v[c];
    }
  };
  const bool heavy_first = ((blockIdx.x + blockIdx.y) & 1) != 0;
  if (heavy_first) heavy_pass();

  const int nch = (a.n_light + CH - 1) / CH;
  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && nch > 0) {
    const int cnt = min(CH, a.n_light);
    mbar_expect_tx(&s_bar[0], cnt * REC32 * 4);
    bulk_g2s(&s_rec[0][0], a.rec32, cnt * REC32 * 4, &s_bar[0]);
  }
  // FP64 centre of the potential this thread stages in the next chunk,
  // prefetched into registers (threads hs and hs + CH stage the same one)
  const int hs = tid % CH, spart = tid / CH;
  constexpr int PARTS = MAP_THREADS / CH;
  static_assert(MAP_THREADS % CH == 0 && PARTS >= 2, "staging threads");
  double2 pxy = make_double2(0, 0);
  if (hs < a.n_light) pxy = reinterpret_cast<const double2 *>(a.pos64)[2 * hs];

  // (X - x0, Y - y0) of this thread's KP points: the column offset added to
  // the staged hi/lo pair ((hi + Lxh) is exact next to the centre, by
  // Sterbenz), the rows as staged
  auto tile_offsets = [&](int buf, int h, float &dX, float (&dY)[KP]) {
    const float4 oy = s_offy[buf][warp][h];
    if constexpr (KP == 2) {
      dX = (oy.x + Lxh) + (oy.y + Lxl);
      dY[0] = oy.z;
      dY[1] = oy.w;
    } else {
      const float2 ox = s_offx[buf][KP == 2 ? 0 : h];
      dX = (ox.x + Lxh) + (ox.y + Lxl);
      dY[0] = oy.x;
      dY[1] = oy.y;
      dY[2] = oy.z;
      dY[3] = oy.w;
    }
  };

  int seen = 0;
  for (int ch = 0; ch < nch; ++ch) {
    const int buf = ch & 1;
    const int base = ch * CH, cnt = min(CH, a.n_light - base);
    if (hs < cnt) {
      // offsets from the potential's centre: one staging thread forms X - x0,
      // the other Y - y0 (FP64, kept as hi/lo float pairs), from which it
      // adds each row's offset inside the tile as a hi/lo pair too
      if (spart == 0) {
        const double dX = Tx - pxy.x;
        const float hx = (float)dX, lx = (float)(dX - (double)hx);
        if constexpr (KP == 2) {
#pragma unroll
          for (int w = 0; w < MAP_WARPS; ++w) {
            s_offy[buf][w][hs].x = hx;
            s_offy[buf][w][hs].y = lx;
          }
        } else {
          s_offx[buf][KP == 2 ? 0 : hs] = make_float2(hx, lx);
        }
      } else if (spart == 1) {
        const double dY = Ty - pxy.y;
        const float hy = (float)dY, ly = (float)(dY - (double)hy);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const float2 L = s_ly[r];
          reinterpret_cast<float *>(&s_offy[buf][r / KP][hs])[(KP == 2 ? 2 : 0) + r % KP] = (hy + L.x) + (ly + L.y);
        }
      }
    }
    const bool ok = mbar_wait_bounded(&s_bar[buf], (ch >> 1) & 1);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(a.err, ERRBIT_WAIT);
        mbar_wait_bounded(&s_bar[buf], (ch >> 1) & 1);  // let the copy in flight land before leaving
      }
      return;
    }
    if (ch + 1 < nch) {
      if (tid == 0) {
        fence_proxy_async();
        const int ncnt = min(CH, a.n_light - base - CH);
        mbar_expect_tx(&s_bar[buf ^ 1], ncnt * REC32 * 4);
        bulk_g2s(&s_rec[buf ^ 1][0], a.rec32 + (size_t)(base + CH) * REC32, ncnt * REC32 * 4, &s_bar[buf ^ 1]);
      }
      if (base + CH + hs < a.n_light) pxy = reinterpret_cast<const double2 *>(a.pos64)[2 * (base + CH + hs)];
    }
    const float4 *recs = reinterpret_cast<const float4 *>(&s_rec[buf][0]);
    if constexpr (HESS ? LENS_MAP_SEGMENTS : (POT || LENS_MAP_SEGMENTS_GRAD)) {
      // the potentials are sorted by kind: each kind's run inside this chunk is
      // a loop without a per-potential dispatch (Hessian kernel: 6 % faster;
      // the deflection-only kernel spills with it and keeps the plain loop)
      auto run = [&](auto kind_tag, int h0, int h1) {
        constexpr int KIND = decltype(kind_tag)::value;
        for (int h = h0; h < h1;) {
          // up to the next fold: no per-potential counter in the inner loop
          const int he = min(h + (SUB - seen), h1);
          seen += he - h;
#pragma unroll MAP_UNROLL
          for (; h < he; ++h) {
            const float4 *r4 = recs + h * (REC32 / 4);
            float dX, dY[KP];
            tile_offsets(buf, h, dX, dY);
            if constexpr (POT1) {
              if (KIND == K32_DPIE)
                dpie32<false, KP, false, false, true>(r4, dX, dY, part);
              else if (KIND == K32_DPIE_SERIES)
                dpie32<false, KP, true, false, true>(r4, dX, dY, part);
              else
                circ32<false, KP, KIND == K32_POINT, true>(r4, dX, dY, part);
            } else {
              float2 dY2[NP];
#pragma unroll
              for (int j = 0; j < NP; ++j) dY2[j] = make_float2(dY[2 * j], dY[2 * j + 1]);
              if (KIND == K32_DPIE)
                dpie32x2<HESS, NP, false, !POT, false, POT>(r4, dX, dY2, part);
              else if (KIND == K32_DPIE_SERIES)
                dpie32x2<HESS, NP, true, !POT, false, POT>(r4, dX, dY2, part);
              else
                circ32x2<HESS, NP, KIND == K32_POINT, !POT, POT>(r4, dX, dY2, part);
            }
          }
          if (seen == SUB) {
            fold_all();
            seen = 0;
          }
        }
      };
      auto seg = [&](int k, int &h0, int &h1) {
        h0 = max(a.koff[k] - base, 0);
        h1 = min(a.koff[k + 1] - base, cnt);
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
    } else if constexpr (!POT) {
      for (int h = 0; h < cnt;) {
        const int he = min(h + (SUB - seen), cnt);
        seen += he - h;
        for (; h < he; ++h) {
          const float4 *r4 = recs + h * (REC32 / 4);
          float dX, dY[KP];
          tile_offsets(buf, h, dX, dY);
          float2 dY2[NP];
#pragma unroll
          for (int j = 0; j < NP; ++j) dY2[j] = make_float2(dY[2 * j], dY[2 * j + 1]);
          eval32x2_any<HESS, NP>(r4, dX, dY2, part);
        }
        if (seen == SUB) {
          fold_all();
          seen = 0;
        }
      }
    }
  }
  fold_all();
  if (!heavy_first) heavy_pass();

  // per-point epilogue: FP32 totals + FP64 sums, scaled, derived maps
  const int i = i0 + lane;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int j = j0 + warp * KP + k;
    if constexpr (POT) {
      if (i < a.nx && j < a.ny) {
        const long long o = (long long)j * a.nx + i;
        const double phi = a.dls * ((double)pt(tot.k, k) - (double)pt(cmp.k, k) + s_hv[tid][k][0]);
        a.out64[o] = phi;
        if (a.tau) {
          const double X = a.xmin + i * a.dx - a.bx, Y = a.ymin + (a.row0 + j) * a.dy - a.by;
          a.out64[a.plane + o] = 0.5 * (X * X + Y * Y) - phi;
        }
      }
      continue;
    }
    const double AX = (double)pt(tot.ax, k) - (double)pt(cmp.ax, k) + s_hv[tid][k][0];
    const double AY = (double)pt(tot.ay, k) - (double)pt(cmp.ay, k) + s_hv[tid][k][NC > 1 ? 1 : 0];
    double KA = 0, G1 = 0, G2 = 0;
    if (HESS) {
      KA = (double)pt(tot.k, k) - (double)pt(cmp.k, k) + s_hv[tid][k][NC > 2 ? 2 : 0];
      G1 = (double)pt(tot.g1, k) - (double)pt(cmp.g1, k) + s_hv[tid][k][NC > 3 ? 3 : 0];
      G2 = (double)pt(tot.g2, k) - (double)pt(cmp.g2, k) + s_hv[tid][k][NC > 4 ? 4 : 0];
    }
    if constexpr (!POT) {
      // FP32 cancellation: the rounding error of the FP32 terms is ~1e-7 of
      // their summed magnitude; where that is not well below 1e-6 |alpha|
      // the node is recomputed in double-float (k_map_repair)
      // (the decisions in FP32: they only need a few significant digits)
      const float S = a.repair_f * pt(tot.mag, k), fax = (float)AX, fay = (float)AY;
      const bool rep = i < a.nx && j < a.ny && fmaf(fax, fax, fay * fay) < S * S;
      bool rep_h = false;  // det's error: the Hessian planes need the repair as well
      if (HESS && a.repair > 0.0) {
        // det = (1 - kappa)^2 - gamma^2 carries 2 |1 - kappa| dkappa + 2 |gamma| dgamma;
        // the FP32 terms' kappa are positive, so their sum bounds their
        // magnitude, and their gamma's by that sum plus |gamma| of their sum
        const float d = (float)a.dls;
        const float kl = d * pt(tot.k, k), g1l = d * pt(tot.g1, k), g2l = d * pt(tot.g2, k);
        const float kap = d * (float)KA, g1 = d * (float)G1, g2 = d * (float)G2;
        const float gm = sqrtf(fmaf(g1, g1, g2 * g2)), gl = sqrtf(fmaf(g1l, g1l, g2l * g2l));
        rep_h = i < a.nx && j < a.ny &&
                (float)(2.0 * DET_TERM_ERR) * (fabsf(1.f - kap) * fabsf(kl) + gm * (fabsf(kl) + gl)) >
                    (float)DET_REPAIR_ABS;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, rep || rep_h);
      if (mask) {
        int first = 0;
        if (lane == __ffs(mask) - 1) first = atomicAdd(a.rep_count, __popc(mask));
        first = __shfl_sync(0xffffffffu, first, __ffs(mask) - 1);
        // bit 31: the Hessian planes too (else the deflection alone)
        if (rep || rep_h)
          a.rep_list[first + __popc(mask & ((1u << lane) - 1u))] = (j * a.nx + i) | (rep_h ? (int)0x80000000u : 0);
      }
    }
    if (i < a.nx && j < a.ny) {
      const long long o = (long long)j * a.nx + i;
      a.out[o] = (float)(a.dls * AX);
      a.out[a.plane + o] = (float)(a.dls * AY);
      if (HESS) {
        const double kap = a.dls * KA, g1 = a.dls * G1, g2 = a.dls * G2;
        const double det = (1.0 - kap) * (1.0 - kap) - g1 * g1 - g2 * g2;
        a.out[2 * a.plane + o] = (float)kap;
        a.out[3 * a.plane + o] = (float)g1;
        a.out[4 * a.plane + o] = (float)g2;
        a.out[5 * a.plane + o] = (float)(1.0 / det);
      }
    }
  }
}

// Double-float repair of the nodes the mixed map kernel listed: a CTA of
// REP_WARPS warps takes REP_WARPS nodes, one per warp; the potentials' double-
// float records are staged in shared memory 32 at a time (field-major, read
// by all the CTA's warps) and lane l evaluates potential h0 + l of each chunk
// at its warp's node (FP64 where double-float fails); a warp sum in FP64 and
// the node's deflection planes -- and, for an entry with bit 31 set, its
// Hessian planes too -- rewritten as the map kernel writes them.  A node
// listed for its deflection alone keeps the map kernel's kappa, gamma and mu
// (their FP32 errors are far inside their tolerances there).
struct RepairArgs {
  const float2 *recdf;
  const double *all64;
  int n;
  double xmin, ymin, dx, dy;
  int nx, row0;
  double dls;
  float *out;
  long long plane;
  const int *count, *list;
};

// LENS_REPAIR_DFSUM: each lane sums its terms in double-float and converts
// once (0: every term converted and added in FP64, 20 FP64-pipe operations
// per term with the Hessian)
#ifndef LENS_REPAIR_DFSUM
#define LENS_REPAIR_DFSUM 1
#endif
constexpr int REP_WARPS = 8, REP_THREADS = 32 * REP_WARPS, REP_CH = 32;  // potentials per staged chunk (one per lane)

template <bool HESS>
__global__ void __launch_bounds__(REP_THREADS) k_map_repair(const RepairArgs a) {
  __shared__ float2 s_rdf[RECDF][REP_CH];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int total = *a.count;
  for (int e0 = blockIdx.x * REP_WARPS; e0 < total; e0 += gridDim.x * REP_WARPS) {  // uniform over the CTA
    const int e = e0 + warp;
    const bool have = e < total;
    const int entry = have ? a.list[e] : 0;
    const int o = entry & 0x7fffffff;
    const bool full = HESS && entry < 0;  // warp-uniform
    const int i = o % a.nx, j = o / a.nx;
    const double X = a.xmin + i * a.dx, Y = a.ymin + (a.row0 + j) * a.dy;
#if LENS_REPAIR_DFSUM
    const df Xd = df_from_double(X), Yd = df_from_double(Y);
    df sum[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#endif
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int h0 = 0; h0 < a.n; h0 += REP_CH) {
      __syncthreads();  // the previous chunk has been used
      for (int t = threadIdx.x; t < RECDF * REP_CH; t += REP_THREADS) {
        const int f = t / REP_CH, h = h0 + t % REP_CH;
        s_rdf[f][t % REP_CH] = h < a.n ? a.recdf[(size_t)f * a.n + h] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const int h = h0 + lane;
      if (have && h < a.n) {
#if LENS_REPAIR_DFSUM
        if (full)
          add_potential_dfs<true>(&s_rdf[0][lane], REP_CH, a.all64 + (size_t)h * REC64, X, Y, Xd, Yd, sum);
        else
          add_potential_dfs<false>(&s_rdf[0][lane], REP_CH, a.all64 + (size_t)h * REC64, X, Y, Xd, Yd, sum);
#else
        if (full)
          add_potential_df<true>(&s_rdf[0][lane], REP_CH, a.all64 + (size_t)h * REC64, X, Y, acc);
        else
          add_potential_df<false>(&s_rdf[0][lane], REP_CH, a.all64 + (size_t)h * REC64, X, Y, acc);
#endif
      }
    }
#if LENS_REPAIR_DFSUM
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[c] = df_to_double(sum[c]);
#endif
#pragma unroll
    for (int c = 0; c < (HESS ? 5 : 2); ++c)
#pragma unroll
      for (int off = 16; off; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
    if (have && lane == 0) {
      a.out[o] = (float)(a.dls * acc[0]);
      a.out[a.plane + o] = (float)(a.dls * acc[1]);
      if (full) {
        const double kap = a.dls * acc[2], g1 = a.dls * acc[3], g2 = a.dls * acc[4];
        const double det = (1.0 - kap) * (1.0 - kap) - g1 * g1 - g2 * g2;
        a.out[2 * a.plane + o] = (float)kap;
        a.out[3 * a.plane + o] = (float)g1;
        a.out[4 * a.plane + o] = (float)g2;
        a.out[5 * a.plane + o] = (float)(1.0 / det);
      }
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_map_fp64(const double *__restrict__ all64, int n, double xmin, double ymin,
                                                  double dx, double dy, int nx, int row0, double dls,
                                                  double *__restrict__ out, long long plane, int tau = 0,
                                                  double bx = 0.0, double by = 0.0) {
  constexpr bool HESS = MODE == MAP_HESS;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= plane) return;
  const int i = (int)(p % nx), j = (int)(p / nx);
  const double X = xmin + i * dx, Y = ymin + (row0 + j) * dy;
  if constexpr (MODE == MAP_POT) {
    double PHI = 0;
    for (int h = 0; h < n; ++h) PHI += pot64(all64 + (size_t)h * REC64, X, Y);
    const double phi = dls * PHI;
    out[p] = phi;
    if (tau) out[plane + p] = 0.5 * ((X - bx) * (X - bx) + (Y - by) * (Y - by)) - phi;
    return;
  }
  double AX = 0, AY = 0, KA = 0, G1 = 0, G2 = 0;
  for (int h = 0; h < n; ++h) {
    double ax, ay, kk = 0, q1 = 0, q2 = 0;
    eval64<HESS>(all64 + (size_t)h * REC64, X, Y, ax, ay, kk, q1, q2);
    AX += ax;
    AY += ay;
    if (HESS) {
      KA += kk;
      G1 += q1;
      G2 += q2;
    }
  }
  out[p] = dls * AX;
  out[plane + p] = dls * AY;
  if (HESS) {
    const double kap = dls * KA, g1 = dls * G1, g2 = dls * G2;
    out[2 * plane + p] = kap;
    out[3 * plane + p] = g1;
    out[4 * plane + p] = g2;
    out[5 * plane + p] = 1.0 / ((1.0 - kap) * (1.0 - kap) - g1 * g1 - g2 * g2);
  }
}

// The bounded-wait failure path on its own: one thread waits on an mbarrier
// that nothing completes, gives up after `polls` tries, and reports it the way
// the map kernel would (ERRBIT_WAIT in the context's error word).
__global__ void k_wait_selftest(int *err, unsigned polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0, polls)) atomicOr(err, ERRBIT_WAIT);
  }
}

// The FP64 reciprocal and reciprocal square root of the evaluators next to
// CUDA's division and rsqrt: out[0..3][i] = rcp64, 1/x, rsqrt64, rsqrt.
__global__ void k_math_selftest(const double *__restrict__ x, int n, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  out[i] = rcp64(v);
  out[n + i] = 1.0 / v;
  out[2 * n + i] = rsqrt64(v);
  out[3 * n + i] = rsqrt(v);
}

}  // namespace

int launch_math_selftest(const double *x, int n, double *out, cudaStream_t st) {
  if (n > 0) k_math_selftest<<<(n + 255) / 256, 256, 0, st>>>(x, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "self-test launch: %s", cudaGetErrorString(e));
  return LENS_OK;
}

int launch_wait_selftest(lens_ctx *ctx, unsigned polls, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(ctx->d_err, polls);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "self-test launch: %s", cudaGetErrorString(e));
  return LENS_OK;
}

// The FP64 pipe runs at 1/64 of the FP32 rate: with few FP32 potentials per
// FP64 one the cluster-scale potentials' FP64 work outlasts the FP32 sweep
// it overlaps, and their double-float evaluation on the FP32 pipe is faster
// (2 cluster-scale + 215 members: 13.85 -> 9.94 ms per 5000^2 deflection
// map; 2 + 998: 10.00 against 10.17 ms per 2048^2 Hessian map in FP64).
#ifndef LENS_HEAVY_DF_RATIO
#define LENS_HEAVY_DF_RATIO 400
#endif
static int heavy_in_df(const Model *m) {
  return m->n_heavy > 0 && (long long)m->n_light < (long long)LENS_HEAVY_DF_RATIO * m->n_heavy;
}

int map_tile_rows(bool hess) { return map_threads(hess) / 32 * (hess ? LENS_KP_HESS : LENS_KP_GRAD); }

size_t map_repair_bytes(const lens_grid *g, int rows) {
  return sizeof(int) * ((size_t)g->nx * (size_t)(rows < 0 ? g->ny : rows) + 1);
}

int launch_map_mixed(lens_ctx *ctx, const Model *m, const lens_grid *g, double dls, bool hess, void *out,
                     cudaStream_t st, int row0, int rows, bool repair, void *repair_mem) {
  if (rows < 0) rows = g->ny - row0;
  const long long nodes = (long long)g->nx * rows;
  if (nodes > INT32_MAX) return fail(LENS_EINVAL, "map launch of more than 2^31 points");
  repair = repair && ctx->repair_ratio > 0.0 && m->n_light > 0;
  CallScratch rs(ctx, st);  // repair list: a count and up to one entry per node
  if (repair) {
    if (repair_mem) {
      rs.p = nullptr;  // the caller's memory (the request loop's arena)
    } else {
      int rc = rs.alloc(map_repair_bytes(g, rows));
      if (rc) return rc;
      repair_mem = rs.p;
    }
    if (cudaMemsetAsync(repair_mem, 0, sizeof(int), st) != cudaSuccess)
      return fail(LENS_ECUDA, "cudaMemsetAsync failed");
  }
  MapArgs a;
  a.rec32 = m->rec32;
  a.pos64 = m->pos64;
  a.n_light = m->n_light;
  for (int k = 0; k < 5; ++k) a.koff[k] = m->koff[k];
  a.heavy = m->heavy;
  a.heavydf = m->heavydf;
  a.n_heavy = m->n_heavy;
  a.heavy_df = heavy_in_df(m);
  a.xmin = g->xmin;
  a.ymin = g->ymin;
  a.dx = (g->xmax - g->xmin) / (g->nx - 1);
  a.dy = (g->ymax - g->ymin) / (g->ny - 1);
  a.nx = g->nx;
  a.ny = rows;
  a.row0 = row0;
  a.dls = dls;
  a.out = (float *)out;
  a.plane = (long long)g->nx * rows;
  a.err = ctx->d_err;
  a.tau = 0;
  a.bx = a.by = 0.0;
  a.out64 = nullptr;
  a.repair = repair ? ctx->repair_ratio : 0.0;
  a.repair_f = (float)(2.0 * a.repair);
  a.rep_count = repair ? (int *)repair_mem : nullptr;
  a.rep_list = repair ? (int *)repair_mem + 1 : nullptr;
  constexpr int KPG = LENS_KP_GRAD, KPH = LENS_KP_HESS;
  if (hess) {
    const int th = map_tile_rows(true);
    dim3 grid((g->nx + 31) / 32, (rows + th - 1) / th);
    k_map_mixed<MAP_HESS, KPH><<<grid, map_threads(true), 0, st>>>(a);
  } else {
    const int th = map_tile_rows(false);
    dim3 grid((g->nx + 31) / 32, (rows + th - 1) / th);
    k_map_mixed<MAP_GRAD, KPG><<<grid, map_threads(false), 0, st>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "map kernel launch: %s", cudaGetErrorString(e));
  if (repair) {
    RepairArgs r;
    r.recdf = m->recdf;
    r.all64 = m->all64;
    r.n = m->n;
    r.xmin = a.xmin;
    r.ymin = a.ymin;
    r.dx = a.dx;
    r.dy = a.dy;
    r.nx = a.nx;
    r.row0 = row0;
    r.dls = dls;
    r.out = (float *)out;
    r.plane = a.plane;
    r.count = a.rep_count;
    r.list = a.rep_list;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    const int blocks = std::max(1, 4 * nsm);  // CTAs loop over the list: any count covers it
    if (hess)
      k_map_repair<true><<<blocks, REP_THREADS, 0, st>>>(r);
    else
      k_map_repair<false><<<blocks, REP_THREADS, 0, st>>>(r);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LENS_ECUDA, "map repair launch: %s", cudaGetErrorString(e));
  }
  return LENS_OK;
}


int launch_map_fp64(lens_ctx *ctx, const Model *m, const lens_grid *g, double dls, bool hess, void *out,
                    cudaStream_t st, int row0, int rows) {
  (void)ctx;
  if (rows < 0) rows = g->ny - row0;
  const long long plane = (long long)g->nx * rows;
  const double dx = (g->xmax - g->xmin) / (g->nx - 1), dy = (g->ymax - g->ymin) / (g->ny - 1);
  const unsigned blocks = (unsigned)((plane + 255) / 256);
  if (hess)
    k_map_fp64<MAP_HESS><<<blocks, 256, 0, st>>>(m->all64, m->n, g->xmin, g->ymin, dx, dy, g->nx, row0, dls,
                                              (double *)out, plane);
  else
    k_map_fp64<MAP_GRAD><<<blocks, 256, 0, st>>>(m->all64, m->n, g->xmin, g->ymin, dx, dy, g->nx, row0, dls,
                                               (double *)out, plane);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "FP64 map kernel launch: %s", cudaGetErrorString(e));
  return LENS_OK;
}

int launch_pot_map(lens_ctx *ctx, const Model *m, const lens_grid *g, double dls, int32_t precision,
                   const double *beta, void *out, cudaStream_t st) {
  const int rows = g->ny;
  const double dx = (g->xmax - g->xmin) / (g->nx - 1), dy = (g->ymax - g->ymin) / (g->ny - 1);
  const long long plane = (long long)g->nx * rows;
  if (precision == LENS_FP64) {
    const unsigned blocks = (unsigned)((plane + 255) / 256);
    k_map_fp64<MAP_POT><<<blocks, 256, 0, st>>>(m->all64, m->n, g->xmin, g->ymin, dx, dy, g->nx, 0, dls,
                                                 (double *)out, plane, beta != nullptr, beta ? beta[0] : 0.0,
                                                 beta ? beta[1] : 0.0);
  } else {
    MapArgs a;
    a.rec32 = m->rec32;
    a.pos64 = m->pos64;
    a.n_light = m->n_light;
    for (int k = 0; k < 5; ++k) a.koff[k] = m->koff[k];
    a.heavy = m->heavy;
    a.heavydf = m->heavydf;
    a.n_heavy = m->n_heavy;
    a.heavy_df = 0;  // the potential kernel keeps them in FP64 (no double-float potential form)
    a.xmin = g->xmin;
    a.ymin = g->ymin;
    a.dx = dx;
    a.dy = dy;
    a.nx = g->nx;
    a.ny = rows;
    a.row0 = 0;
    a.dls = dls;
    a.out = nullptr;
    a.out64 = (double *)out;
    a.plane = plane;
    a.err = ctx->d_err;
    a.tau = beta != nullptr;
    a.bx = beta ? beta[0] : 0.0;
    a.by = beta ? beta[1] : 0.0;
    a.repair = 0.0;
    a.repair_f = 0.f;
    a.rep_count = a.rep_list = nullptr;
    constexpr int KPG = LENS_KP_GRAD;
    const int th = map_tile_rows(false);
    dim3 grid((g->nx + 31) / 32, (rows + th - 1) / th);
    k_map_mixed<MAP_POT, KPG><<<grid, map_threads(false), 0, st>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LENS_ECUDA, "potential map launch: %s", cudaGetErrorString(e));
  return LENS_OK;
}

}  // namespace lens
