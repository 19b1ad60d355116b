// Device-side building blocks shared by the map and chi2 kernels:
// approximate MUFU reciprocals, mbarrier + 1-D bulk-copy (TMA) helpers with
// bounded waits, and the FP64 evaluation of one potential.
#pragma once

#include "lens_internal.cuh"

namespace lens {

// Bound on any spin on an mbarrier: ~2^24 try_wait polls (seconds), after
// which the kernel sets ERRBIT_WAIT in the context's error word and leaves
// instead of hanging.
constexpr unsigned WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ float rcp_a(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_a(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// FP64 reciprocal and reciprocal square root for positive normal arguments:
// the MUFU approximations refined by two Newton-Raphson steps each (the
// iterations y <- y + y (1 - b y) and y <- y + (y/2)(1 - a y^2), quadratic
// convergence; Muller, "Elementary Functions", ch. 2), about 1 ulp, in 5
// FP64 operations instead of a correctly rounded division or square root.
__device__ __forceinline__ double rcp64(double b) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(b));
  double e = fma(-b, y, 1.0);
  y = fma(y, e, y);
  e = fma(-b, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ double rsqrt64(double a) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  double e = fma(-a * y, y, 1.0);
  y = fma(0.5 * y, e, y);
  e = fma(-a * y, y, 1.0);
  return fma(0.5 * y, e, y);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (TMA), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit = WAIT_LIMIT) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// FP64 counterparts (degree 11, same interval): interpolants at the
// Chebyshev nodes of [0, 0.16] computed in 60-digit arithmetic
// (csrc/fit_series.py); interpolation error below 4e-18 relative.
__device__ __forceinline__ double atan_over_w64(double t) {
  double p = -1.88510462903004675e-02;
  p = fma(p, t, 3.88765647477774812e-02);
  p = fma(p, t, -5.06934062578019290e-02);
  p = fma(p, t, 5.85413360654678111e-02);
  p = fma(p, t, -6.66390440659186400e-02);
  p = fma(p, t, 7.69212547783340445e-02);
  p = fma(p, t, -9.09090112754652180e-02);
  p = fma(p, t, 1.11111108895220217e-01);
  p = fma(p, t, -1.42857142820646682e-01);
  p = fma(p, t, 1.99999999999688677e-01);
  p = fma(p, t, -3.33333333333332316e-01);
  return fma(p, t, 1.0);
}
__device__ __forceinline__ double atanh_over_w64(double t) {
  double p = 1.11279998802890107e-01;
  p = fma(p, t, 1.42027510153455820e-02);
  p = fma(p, t, 6.13504335260846093e-02);
  p = fma(p, t, 5.74260884066186833e-02);
  p = fma(p, t, 6.68122440454864269e-02);
  p = fma(p, t, 7.69130553539208311e-02);
  p = fma(p, t, 9.09095422594738550e-02);
  p = fma(p, t, 1.11111098280666135e-01);
  p = fma(p, t, 1.42857143071626003e-01);
  p = fma(p, t, 1.99999999998152628e-01);
  p = fma(p, t, 3.33333333333339532e-01);
  return fma(p, t, 1.0);
}
constexpr double T_SERIES64 = 0.16;

// FP64 atan and atanh for every argument, by argument reduction into the
// interval of the degree-11 interpolants (|v| <= 0.4) with the addition
// formulas (table-based reduction, as in Muller, "Elementary Functions",
// ch. 6): atan folds |w| > 1 to pi/2 - atan(1/|w|) and shifts [0.4, 1] about
// c = 11/16; atanh shifts about the nearest c_k = tanh(0.8 k) (rounded to
// double; ATANH_A[k] = atanh of that double, 60-digit value), k from a
// single-precision estimate of atanh.  Reduced arguments stay within
// |v| < 0.4; the only FP64 divisions are the one of the shift and, for
// |w| > 1, the reciprocal.  Tables: csrc/fit_series.py.
constexpr double ATAN_11_16 = 0.6022873461349642;  // atan(11/16)
constexpr double PI_2_HI = 1.5707963267948966, PI_2_LO = 6.123233995736766e-17;
constexpr int ATANH_K = 22;
__device__ __constant__ const double ATANH_C[23] = {
    0.0, 0.664036770267849, 0.9216685544064713, 0.9836748576936802,
    0.9966823978396512, 0.999329299739067, 0.9998645517007605, 0.9999726519818308,
    0.9999944784700996, 0.9999988852198828, 0.9999997749296758, 0.9999999545590812,
    0.9999999908256365, 0.999999998147728, 0.9999999996260327, 0.9999999999244973,
    0.9999999999847563, 0.9999999999969224, 0.9999999999993786, 0.9999999999998745,
    0.9999999999999747, 0.9999999999999949, 0.999999999999999};
__device__ __constant__ const double ATANH_A[23] = {
    0.0, 0.8, 1.6000000000000003, 2.400000000000001,
    3.2000000000000037, 3.999999999999993, 4.800000000000132, 5.60000000000052,
    6.399999999997866, 7.199999999979319, 7.999999999898783, 8.800000000192549,
    9.599999997824579, 10.400000010784895, 11.199999965832989, 11.999999839023337,
    12.800001154374243, 13.60000111127314, 14.399980865672688, 15.199987419265298,
    16.000301060641295, 16.800653176873976, 17.616361586450413};

__device__ __forceinline__ double atan64(double w) {
  const double a = fabs(w);
  const bool inv = a > 1.0;
  double v = inv ? rcp64(a) : a, base = 0.0;
  if (v > 0.4) {
    v = (v - 0.6875) * rcp64(fma(v, 0.6875, 1.0));
    base = ATAN_11_16;
  }
  double r = fma(v, atan_over_w64(v * v), base);
  if (inv) r = (PI_2_HI - r) + PI_2_LO;
  return copysign(r, w);
}

__device__ __forceinline__ double atanh64(double w) {
  const double a = fabs(w);
  if (a <= 0.4) return w * atanh_over_w64(w * w);
  // hyperbolic angle estimate 0.5 ln((1+a)/(1-a)); 1-a is exact for a >= 0.5
  const float est = 0.5f * (__logf((float)(1.0 + a)) - __logf((float)(1.0 - a)));
  const int k = __float2int_rn(est * 1.25f);
  if (!(a < 1.0) || k > ATANH_K) return atanh(w);  // |w| >= 1 or within 1e-15 of it
  const int kk = k < 1 ? 1 : k;
  const double c = ATANH_C[kk];
  const double v = (a - c) * rcp64(fma(-a, c, 1.0));
  return copysign(fma(v, atanh_over_w64(v * v), ATANH_A[kk]), w);
}
// The same coefficients as float pairs (hi, lo) for the double-float path.
__device__ __constant__ const float C_ATAN_DF[12][2] = {
    {1.000000000e+00f, 0.000000000e+00f}, {-3.333333433e-01f, 9.934108647e-09f}, {2.000000030e-01f, -2.980543590e-09f},
    {-1.428571492e-01f, 6.422708143e-09f}, {1.111111119e-01f, -3.043733265e-09f}, {-9.090901166e-02f, 3.865411602e-10f},
    {7.692125440e-02f, 3.818954597e-10f}, {-6.663904339e-02f, -6.751677550e-10f}, {5.854133517e-02f, 8.999671564e-10f},
    {-5.069340765e-02f, 1.396960325e-09f}, {3.887656331e-02f, 1.437154284e-09f}, {-1.885104552e-02f, -7.711869476e-10f}};
__device__ __constant__ const float C_ATANH_DF[12][2] = {
    {1.000000000e+00f, 0.000000000e+00f}, {3.333333433e-01f, -9.934101541e-09f}, {2.000000030e-01f, -2.982079694e-09f},
    {1.428571492e-01f, -6.171728906e-09f}, {1.111110970e-01f, 1.242873915e-09f}, {9.090954065e-02f, 1.606245137e-09f},
    {7.691305876e-02f, -3.403861193e-09f}, {6.681224704e-02f, -2.992401216e-09f}, {5.742608756e-02f, 8.483491687e-10f},
    {6.135043502e-02f, -1.492454826e-09f}, {1.420275122e-02f, -2.039270280e-10f}, {1.112800017e-01f, -2.897034390e-09f}};

// ----------------------------------------------------------------- FP64 path
// One potential in FP64 at sky position (X, Y), D_ls/D_s = 1.
// Outputs in the sky frame: deflection (ax, ay) and, if HESS, kappa, gamma1,
// gamma2 of its Hessian.  dPIE: difference of two PIEMD terms written with
//   atan a - atan c   = atan ((a-c)/(1+ac)),
//   atanh a - atanh c = atanh((a-c)/(1-ac)),
// where a-c is formed from strictly positive pieces (no core-cut cancellation).
template <bool HESS>
__device__ __forceinline__ void eval64(const double *__restrict__ r, double X, double Y, double &ax, double &ay,
                                       double &kap, double &g1, double &g2) {
  const int kind = (int)r[D_KIND];
  double dX = X - r[D_X0], dY = Y - r[D_Y0];
  if (kind == K64_SIS || kind == K64_POINT) {
    double r2 = dX * dX + dY * dY;
    if (r2 == 0.0) {
      ax = ay = kap = g1 = g2 = 0.0;
      return;
    }
    double b = r[D_B];
    if (kind == K64_SIS) {
      double ir = rsqrt(r2);
      ax = b * dX * ir;
      ay = b * dY * ir;
      if (HESS) {
        double ir3 = ir * ir * ir;
        kap = 0.5 * b * ir;
        g1 = 0.5 * b * (dY * dY - dX * dX) * ir3;
        g2 = -b * dX * dY * ir3;
      }
    } else {
      double ir2 = 1.0 / r2;
      ax = b * dX * ir2;
      ay = b * dY * ir2;
      if (HESS) {
        double ir4 = ir2 * ir2;
        kap = 0.0;
        g1 = b * (dY * dY - dX * dX) * ir4;
        g2 = -2.0 * b * dX * dY * ir4;
      }
    }
    return;
  }
  const double c = r[D_C], s = r[D_S], q2 = r[D_Q2], u = r[D_U], u2 = r[D_U2], bq = r[D_BQ];
  const double sc = r[D_SC], st = r[D_ST], dS = r[D_DS], sS = r[D_SS];
  double x = c * dX + s * dY, y = c * dY - s * dX;
  double x2 = x * x, y2 = y * y;
  double R = q2 * x2 + y2;
  const double pc2 = R + q2 * sc * sc, pt2 = R + q2 * st * st;
  const double ic = rsqrt64(pc2), it = rsqrt64(pt2);  // 1/psi (psi >= q s > 0)
  double psc = pc2 * ic, pst = pt2 * it;
  double Sp = psc + pst;
  double Ec = psc + sc, Et = pst + st;
  double Fc = psc + q2 * sc, Ft = pst + q2 * st;
  // both denominators are positive
  double Zx = x * dS * (Sp + q2 * sS) * rcp64(Sp * (Ec * Et + u2 * x2));
  double Zy = y * q2 * dS * (Sp + sS) * rcp64(Sp * (Fc * Ft - u2 * y2));
  double axp, ayp;
  if (kind == K64_DPIE_SERIES) {
    double wx = u2 * Zx * Zx, wy = u2 * Zy * Zy;
    axp = bq * Zx * (1.0 - wx / 3.0 + wx * wx / 5.0);
    ayp = bq * Zy * (1.0 + wy / 3.0 + wy * wy / 5.0);
  } else {
    const double wx = u * Zx, wy = u * Zy, tx = wx * wx, ty = wy * wy;
    if (fmax(tx, ty) < T_SERIES64) {  // bq/u atan(u Z) = bq Z atan(w)/w
      axp = bq * Zx * atan_over_w64(tx);
      ayp = bq * Zy * atanh_over_w64(ty);
    } else {
      const double bu = bq * rcp64(u);
      axp = bu * atan64(wx);
      ayp = bu * atanh64(wy);
    }
  }
  ax = c * axp - s * ayp;
  ay = s * axp + c * ayp;
  if (HESS) {
    double r2 = x2 + y2, ymx = y2 - x2;
    double Dc = (1.0 + q2) * sc * sc + 2.0 * sc * psc + r2;
    double Dt = (1.0 + q2) * st * st + 2.0 * st * pst + r2;
    double fc = ic * rcp64(Dc), ft = it * rcp64(Dt);  // 1/(psi D)
    double g1p = 0.5 * bq * (fc * (ymx - u2 * sc * sc) - ft * (ymx - u2 * st * st));
    double g2p = -bq * (fc - ft) * x * y;
    kap = 0.5 * bq * (ic - it);
    double c2 = r[D_C2T], s2 = r[D_S2T];
    g1 = c2 * g1p - s2 * g2p;
    g2 = s2 * g1p + c2 * g2p;
  }
}


// Lensing potential of one potential in FP64 at (X, Y), D_ls/D_s = 1, up to
// the same constant as the definition: dPIE x alpha_x' + y alpha_y' minus
// b q s ln sqrt((psi + s)^2 + u^2 x^2) of each term (core minus cut); SIS
// b r; point mass theta_E^2 ln r (0 at the centre).
__device__ __forceinline__ double pot64(const double *__restrict__ r, double X, double Y) {
  const int kind = (int)r[D_KIND];
  const double dX = X - r[D_X0], dY = Y - r[D_Y0];
  const double r2 = dX * dX + dY * dY;
  if (kind == K64_SIS) return r[D_B] * sqrt(r2);
  if (kind == K64_POINT) return r2 > 0.0 ? 0.5 * r[D_B] * log(r2) : 0.0;
  // the deflection's arguments as in eval64, then the two logarithms
  const double c = r[D_C], s = r[D_S], q2 = r[D_Q2], u = r[D_U], u2 = r[D_U2], bq = r[D_BQ];
  const double sc = r[D_SC], st = r[D_ST], dS = r[D_DS], sS = r[D_SS];
  const double x = c * dX + s * dY, y = c * dY - s * dX;
  const double x2 = x * x, y2 = y * y;
  const double R = q2 * x2 + y2;
  const double pc2 = R + q2 * sc * sc, pt2 = R + q2 * st * st;
  const double psc = pc2 * rsqrt64(pc2), pst = pt2 * rsqrt64(pt2);
  const double Sp = psc + pst, Ec = psc + sc, Et = pst + st, Fc = psc + q2 * sc, Ft = pst + q2 * st;
  const double Zx = x * dS * (Sp + q2 * sS) * rcp64(Sp * (Ec * Et + u2 * x2));
  const double Zy = y * q2 * dS * (Sp + sS) * rcp64(Sp * (Fc * Ft - u2 * y2));
  double axp, ayp;  // halo-frame deflection
  if (kind == K64_DPIE_SERIES) {
    const double wx = u2 * Zx * Zx, wy = u2 * Zy * Zy;
    axp = bq * Zx * (1.0 - wx / 3.0 + wx * wx / 5.0);
    ayp = bq * Zy * (1.0 + wy / 3.0 + wy * wy / 5.0);
  } else {
    const double wx = u * Zx, wy = u * Zy, tx = wx * wx, ty = wy * wy;
    if (fmax(tx, ty) < T_SERIES64) {
      axp = bq * Zx * atan_over_w64(tx);
      ayp = bq * Zy * atanh_over_w64(ty);
    } else {
      const double bu = bq * rcp64(u);
      axp = bu * atan64(wx);
      ayp = bu * atanh64(wy);
    }
  }
  const double lc = log(Ec * Ec + u2 * x2), lt = log(Et * Et + u2 * x2);
  return x * axp + y * ayp - 0.5 * bq * (sc * lc - st * lt);
}

// ----------------------------------------------------------------- FP32 path
template <bool HESS, int KP>
struct Acc {
  float ax[KP], ay[KP], k[KP], g1[KP], g2[KP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < KP; ++i) ax[i] = ay[i] = k[i] = g1[i] = g2[i] = 0.f;
  }
};

// Kahan step: (s, c) += v, true sum ~ s - c.
__device__ __forceinline__ void kahan(float &s, float &c, float v) {
  float y = v - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <bool HESS, int KP>
__device__ __forceinline__ void fold(Acc<HESS, KP> &tot, Acc<HESS, KP> &cmp, Acc<HESS, KP> &part) {
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    kahan(tot.ax[i], cmp.ax[i], part.ax[i]);
    kahan(tot.ay[i], cmp.ay[i], part.ay[i]);
    if (HESS) {
      kahan(tot.k[i], cmp.k[i], part.k[i]);
      kahan(tot.g1[i], cmp.g1[i], part.g1[i]);
      kahan(tot.g2[i], cmp.g2[i], part.g2[i]);
    }
  }
  part.zero();
}

// atan(w)/w and atanh(w)/w as polynomials in t = w^2, valid for
// t < T_SERIES = 0.16 (|w| < 0.4): Chebyshev interpolants of the exact
// functions on [0, 0.16] (coefficients from csrc/fit_series.py), Horner with
// FMA.  Degree 4 (default): interpolation error 1.4e-8 / 2.9e-8 relative,
// 5.8e-8 / 1.1e-7 with the FP32 rounding of the evaluation; degree 5:
// 4e-10 / 1.1e-9, 3.5e-8 / 6.1e-8.  The argument Z itself carries several
// FP32 roundings, so degree 4 leaves the per-term error about where it was.
#ifndef LENS_SERIES_DEG
#define LENS_SERIES_DEG 4
#endif
constexpr float T_SERIES = 0.16f;
// coefficients, highest degree first
#if LENS_SERIES_DEG == 5
#define LENS_ATAN_W_COEF -6.186992596e-02f, 1.062997788e-01f, -1.424732623e-01f, 1.999858949e-01f, \
                         -3.333331418e-01f, 9.999999996e-01f
#define LENS_ATANH_W_COEF 1.399562492e-01f, 1.014973434e-01f, 1.436870917e-01f, 1.999682206e-01f, \
                          3.333337736e-01f, 9.999999990e-01f
#else
#define LENS_ATAN_W_COEF 8.147408669e-02f, -1.389835755e-01f, 1.997853999e-01f, -3.333291011e-01f, 9.999999865e-01f
#define LENS_ATANH_W_COEF 1.572736881e-01f, 1.359152003e-01f, 2.004095578e-01f, 3.333250231e-01f, 1.000000027e+00f
#endif
// Horner with FMA: c[0] t^n + ... + c[n]
template <typename... C>
__device__ __forceinline__ float horner(float t, float c0, C... c) {
  float p = c0;
  ((p = fmaf(p, t, c)), ...);
  return p;
}
__device__ __forceinline__ float atan_over_w(float t) { return horner(t, LENS_ATAN_W_COEF); }
__device__ __forceinline__ float atanh_over_w(float t) { return horner(t, LENS_ATANH_W_COEF); }

// One dPIE (FP32) at KP points.  (dX, dY) of each point relative to the
// potential's centre are formed by the caller from hi/lo float pairs, then
//   x = c dX + s dY,  y = c dY - s dX   (halo frame).
// Decision-grade atan for the image search: the reduction of atan64 in FP32
// (fold |w| > 1, shift [0.4, 1] about 11/16) into the degree-5 interpolant,
// branch-free so that lanes do not diverge.
__device__ __forceinline__ float atan_fast(float w) {
  const float a = fabsf(w);
  const bool inv = a > 1.f;
  float v = inv ? rcp_a(a) : a;
  const bool sh = v > 0.4f;
  v = sh ? (v - 0.6875f) * rcp_a(fmaf(v, 0.6875f, 1.f)) : v;
  float r = v * atan_over_w(v * v) + (sh ? 0.602287352f : 0.f);
  r = inv ? 1.57079637f - r : r;
  return copysignf(r, w);
}

// FAST: outside the polynomial range, atan by atan_fast and
// 2 atanh(w) = ln((1+w)/(1-w)) by the MUFU log2 (absolute error ~1e-7; the
// image search only decides which triangles seed a candidate).
//
// Per term (core s = sc, cut s = st) with psi^2 = q^2 (s^2 + x^2) + y^2:
//   alpha_x' = (b q/u) atan(u x/(psi + s)),  alpha_y' = (b q/u) atanh(u y/(psi + q^2 s)),
// and the core-cut differences as single atan / atanh of the arguments
//   Zx = x (dS Sp + dK) / (Sp (Ec Et + u^2 x^2)),
//   Zy = y (q^2 dS Sp + dK) / (Sp (Fc Ft - u^2 y^2))           (times u),
// Sp = psi_c + psi_t, E = psi + s, F = psi + q^2 s, dS = st - sc,
// dK = q^2 (st^2 - sc^2) = psi_t^2 - psi_c^2 (no cancellation in FP32).
// Hessian: D = (1 + q^2) s^2 + 2 psi s + x^2 + y^2 = E^2 + u^2 x^2, and
//   psi_xx' + psi_yy' = b q (1/psi_c - 1/psi_t),
//   psi_yy' - psi_xx' = b q ((y^2 - x^2)(fc - ft) - u^2 (sc^2 fc - st^2 ft)),
//   psi_xy' = -b q xy (fc - ft),  f = 1/(psi D),
// rotated by 2 theta.  The factor b q rides on the rotation constants.
// dX of point k: one value shared by the KP points (a map column) or one
// per point.
__device__ __forceinline__ float dx_of(float dX, int) { return dX; }
template <int KP>
__device__ __forceinline__ float dx_of(const float (&dX)[KP], int k) { return dX[k]; }

// POT: the lensing potential instead, into p.k (Acc<true, KP>; p.ax, p.ay,
// p.g1, p.g2 untouched): per term x alpha_x' + y alpha_y' - b q s ln sqrt(D)
// with D = (psi + s)^2 + u^2 x^2, the logarithms by the MUFU log2.
template <bool HESS, int KP, bool SERIES, bool FAST = false, bool POT = false, typename DX>
__device__ __forceinline__ void dpie32(const float4 *__restrict__ r4, const DX &dX, const float (&dY)[KP],
                                       Acc<HESS || POT, KP> &p) {
  const float4 A = r4[0], B = r4[1], Cq = r4[2], D = r4[3], E = r4[4];
  const float c = A.x, s = A.y, q2 = A.z, u2 = A.w;
  const float Kc = B.x, Kt = B.y, sc = B.z, st = B.w;
  const float dK = Cq.x, dS = Cq.y, q2sc = Cq.z, q2st = Cq.w;
  const float q2dS = D.y;
  const float cb = E.x, sb = E.y;
  float x[KP], y[KP], x2[KP], y2[KP], u2x2[KP], ic[KP], it[KP], psc[KP], pst[KP], Ec[KP], Et[KP];
  float Zx[KP], Zy[KP], tx[KP], ty[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const float cdX = c * dx_of(dX, k), sdX = s * dx_of(dX, k);  // once when dX is shared
    x[k] = fmaf(s, dY[k], cdX);
    y[k] = fmaf(c, dY[k], -sdX);
    x2[k] = x[k] * x[k];
    y2[k] = y[k] * y[k];
    u2x2[k] = u2 * x2[k];
    const float R = fmaf(q2, x2[k], y2[k]);
    const float pc2 = R + Kc, pt2 = R + Kt;
    ic[k] = rsqrt_a(pc2);
    it[k] = rsqrt_a(pt2);
    psc[k] = pc2 * ic[k];
    pst[k] = pt2 * it[k];
    const float Sp = psc[k] + pst[k];
    Ec[k] = psc[k] + sc;
    Et[k] = pst[k] + st;
    Zx[k] = x[k] * fmaf(dS, Sp, dK) * rcp_a(Sp * fmaf(Ec[k], Et[k], u2x2[k]));
    const float Fc = psc[k] + q2sc, Ft = pst[k] + q2st;
    Zy[k] = y[k] * fmaf(q2dS, Sp, dK) * rcp_a(Sp * fmaf(-u2, y2[k], Fc * Ft));
    tx[k] = u2 * (Zx[k] * Zx[k]);
    ty[k] = u2 * (Zy[k] * Zy[k]);
  }
  // halo-frame deflection over b q: the interpolants where every point's
  // |w|^2 < T_SERIES (always for the SERIES kind, u < 0.12: t < 0.0144),
  // one branch for all KP points
  float axp[KP], ayp[KP];
  bool poly = SERIES;
  if (!SERIES) {
    float t = fmaxf(tx[0], ty[0]);
#pragma unroll
    for (int k = 1; k < KP; ++k) t = fmaxf(t, fmaxf(tx[k], ty[k]));
    poly = t < T_SERIES;
  }
  if (poly) {
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      axp[k] = Zx[k] * atan_over_w(tx[k]);
      ayp[k] = Zy[k] * atanh_over_w(ty[k]);
    }
  } else {
    const float u = r4[6].x, iu = E.w;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      if (fmaxf(tx[k], ty[k]) < T_SERIES) {
        axp[k] = Zx[k] * atan_over_w(tx[k]);
        ayp[k] = Zy[k] * atanh_over_w(ty[k]);
      } else {
        const float wx = u * Zx[k], wy = u * Zy[k];
        if (FAST) {
          axp[k] = iu * atan_fast(wx);
          ayp[k] = iu * (0.346573590f * __log2f((1.f + wy) * rcp_a(1.f - wy)));
        } else {
          axp[k] = iu * atanf(wx);
          ayp[k] = (0.5f * iu) * log1pf((wy + wy) * rcp_a(1.f - wy));
        }
      }
    }
  }
  if constexpr (POT) {
    const float bq = 2.f * E.z;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const float Dc = fmaf(Ec[k], Ec[k], u2x2[k]), Dt = fmaf(Et[k], Et[k], u2x2[k]);
      const float lg = fmaf(sc, __log2f(Dc), -st * __log2f(Dt));  // sc log2 Dc - st log2 Dt
      p.k[k] = fmaf(bq, fmaf(x[k], axp[k], fmaf(y[k], ayp[k], -0.346573590f * lg)), p.k[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      p.ax[k] = fmaf(cb, axp[k], fmaf(-sb, ayp[k], p.ax[k]));
      p.ay[k] = fmaf(sb, axp[k], fmaf(cb, ayp[k], p.ay[k]));
      if (HESS) {
        const float4 G = r4[5];
        const float u2sc2 = D.z, u2st2 = D.w;
        const float ymx = y2[k] - x2[k];
        const float Dc = fmaf(Ec[k], Ec[k], u2x2[k]), Dt = fmaf(Et[k], Et[k], u2x2[k]);
        const float fc = rcp_a(psc[k] * Dc), ft = rcp_a(pst[k] * Dt);
        const float fd = fc - ft;
        const float g1d = fmaf(ymx, fd, -fmaf(u2sc2, fc, -u2st2 * ft));
        const float g2d = fd * (x[k] * y[k]);
        p.k[k] = fmaf(E.z, ic[k] - it[k], p.k[k]);
        p.g1[k] = fmaf(G.x, g1d, fmaf(G.y, g2d, p.g1[k]));
        p.g2[k] = fmaf(G.z, g1d, fmaf(G.w, g2d, p.g2[k]));
      }
    }
  }
}

// SIS / point mass (FP32): circular, evaluated directly on (dX, dY).
// POT: the potential b r (SIS) or b ln r (point mass, b = theta_E^2; 0 at
// the centre) into p.k.
template <bool HESS, int KP, bool POINT, bool POT = false, typename DX>
__device__ __forceinline__ void circ32(const float4 *__restrict__ r4, const DX &dX, const float (&dY)[KP],
                                       Acc<HESS || POT, KP> &p) {
  const float b = r4[7].y;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const float x = dx_of(dX, k), y = dY[k];
    const float r2 = fmaf(x, x, y * y);
    if constexpr (POT) {
      if (POINT)
        p.k[k] = fmaf(b, r2 > 0.f ? 0.346573590f * __log2f(r2) : 0.f, p.k[k]);
      else
        p.k[k] = fmaf(b, r2 > 0.f ? r2 * rsqrt_a(r2) : 0.f, p.k[k]);
      continue;
    }
    if (POINT) {
      const float ir2 = r2 > 0.f ? rcp_a(r2) : 0.f;
      const float f = b * ir2;
      p.ax[k] = fmaf(f, x, p.ax[k]);
      p.ay[k] = fmaf(f, y, p.ay[k]);
      if (HESS) {
        const float f2 = f * ir2;
        p.g1[k] = fmaf(f2, (y - x) * (y + x), p.g1[k]);
        p.g2[k] = fmaf(-2.f * f2, x * y, p.g2[k]);
      }
    } else {
      const float ir = r2 > 0.f ? rsqrt_a(r2) : 0.f;
      const float f = b * ir;
      p.ax[k] = fmaf(f, x, p.ax[k]);
      p.ay[k] = fmaf(f, y, p.ay[k]);
      if (HESS) {
        const float f3 = f * ir * ir;
        p.k[k] = fmaf(0.5f, f, p.k[k]);
        p.g1[k] = fmaf(0.5f * f3, (y - x) * (y + x), p.g1[k]);
        p.g2[k] = fmaf(-f3, x * y, p.g2[k]);
      }
    }
  }
}

// Any FP32 potential at KP points (kind is warp-uniform in the map kernel;
// per-lane in the image kernels).
template <bool HESS, int KP, bool FAST = false, typename DX>
__device__ __forceinline__ void eval32_any(const float4 *__restrict__ r4, const DX &dX, const float (&dY)[KP],
                                           Acc<HESS, KP> &p) {
  const int kind = __float_as_int(r4[7].x);
  if (kind == K32_DPIE)
    dpie32<HESS, KP, false, FAST>(r4, dX, dY, p);
  else if (kind == K32_DPIE_SERIES)
    dpie32<HESS, KP, true>(r4, dX, dY, p);
  else if (kind == K32_SIS)
    circ32<HESS, KP, false>(r4, dX, dY, p);
  else
    circ32<HESS, KP, true>(r4, dX, dY, p);
}


// ------------------------------------------------------- paired FP32 path
// The map kernels give each thread points in pairs that share every
// per-potential constant (two rows of one grid column).  Blackwell executes
// the two FP32 additions, multiplications or FMAs of a float2 as one
// instruction (FADD2 / FMUL2 / FFMA2), so a pair is evaluated side by side:
// the same FP32 work in half the issued instructions.  The MUFU
// approximations (rsqrt, rcp) have no paired form and run per point.  Each
// paired operation rounds exactly as the scalar one it replaces (a - b is
// formed as b * (-1) + a: an exact product and one rounding); a product and
// a sum that the compiler fuses into one FMA in the scalar dpie32 / circ32
// stay two roundings here, so the two forms can differ in the last bits.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrt_a(a.x), rsqrt_a(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_a(a.x), rcp_a(a.y)); }
template <typename... C>
__device__ __forceinline__ float2 horner2(float2 t, float c0, C... c) {
  float2 p = dup2(c0);
  ((p = fma2(p, t, dup2(c))), ...);
  return p;
}
// component h (0: .x, 1: .y) of a pair, h a compile-time constant after unrolling
__device__ __forceinline__ float &part2(float2 &v, int h) { return h ? v.y : v.x; }
__device__ __forceinline__ float part2(const float2 &v, int h) { return h ? v.y : v.x; }

// Sums of NP point pairs: point 2 j + h lives in component h of entry j.
// mag: half the summed magnitudes of the terms' deflections (each term's
// |alpha| taken as |alpha_x'| + |alpha_y'| in its own frame), the scale of
// the FP32 rounding error of the sum (plain FP32 sum: an estimate).
template <bool HESS, int NP>
struct Acc2 {
  float2 ax[NP], ay[NP], k[NP], g1[NP], g2[NP], mag[NP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NP; ++i) ax[i] = ay[i] = k[i] = g1[i] = g2[i] = mag[i] = make_float2(0.f, 0.f);
  }
};
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }

__device__ __forceinline__ void kahan2(float2 &s, float2 &c, float2 v) {
  const float2 y = sub2(v, c);
  const float2 t = add2(s, y);
  c = sub2(sub2(t, s), y);
  s = t;
}

template <bool HESS, int NP>
__device__ __forceinline__ void fold2(Acc2<HESS, NP> &tot, Acc2<HESS, NP> &cmp, Acc2<HESS, NP> &part) {
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    kahan2(tot.ax[i], cmp.ax[i], part.ax[i]);
    kahan2(tot.ay[i], cmp.ay[i], part.ay[i]);
    if (HESS) {
      kahan2(tot.k[i], cmp.k[i], part.k[i]);
      kahan2(tot.g1[i], cmp.g1[i], part.g1[i]);
      kahan2(tot.g2[i], cmp.g2[i], part.g2[i]);
    }
    tot.mag[i] = add2(tot.mag[i], part.mag[i]);
  }
  part.zero();
}

// The potential sums alone (p.k) folded into the compensated total.
template <bool HESS, int NP>
__device__ __forceinline__ void fold2_pot(Acc2<HESS, NP> &tot, Acc2<HESS, NP> &cmp, Acc2<HESS, NP> &part) {
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    kahan2(tot.k[i], cmp.k[i], part.k[i]);
    part.k[i] = make_float2(0.f, 0.f);
  }
}

// dX of pair k: one value shared by both points and all pairs (a map
// column), or one per point (float2 per pair)
__device__ __forceinline__ float2 dx2_of(float dX, int) { return dup2(dX); }
template <int NP>
__device__ __forceinline__ float2 dx2_of(const float2 (&dX)[NP], int k) { return dX[k]; }
// c dX of pair k, rounded as the scalar c * dX
__device__ __forceinline__ float2 cdx2(float c, float dX, int) { return dup2(c * dX); }
template <int NP>
__device__ __forceinline__ float2 cdx2(float c, const float2 (&dX)[NP], int k) { return mul2(dup2(c), dX[k]); }

#ifndef LENS_MAP_FOLD_U
#define LENS_MAP_FOLD_U 1  // paired evaluator: u folded into the general kind's constants
#endif
// One dPIE (FP32) at NP point pairs, dX shared (one grid column) or per
// point, dY per point: the arithmetic of dpie32 (same formulas, same order),
// paired.  MAG: also the magnitude sum p.mag.  FAST: outside the
// interpolants' range, dpie32's FAST forms (decision-grade, image search).
// POT: the potential (dpie32's POT form, paired) into p.k, on the plain
// (unfolded) record constants.
template <bool HESS, int NP, bool SERIES, bool MAG = true, bool FAST = false, bool POT = false, typename DX>
__device__ __forceinline__ void dpie32x2(const float4 *__restrict__ r4, const DX &dX, const float2 (&dY)[NP],
                                         Acc2<HESS, NP> &p) {
  const float4 A = r4[0], B = r4[1], Cq = r4[2], D = r4[3], E = r4[4];
  const float c = A.x, s = A.y, q2 = A.z, u2 = A.w;
  const float Kc = B.x, Kt = B.y, sc = B.z, st = B.w;
  // FOLD (the general kind, u >= U_SERIES32): Zx, Zy below carry the factor
  // u (the numerators' constants times u), so t = Z^2 needs no u^2 and the
  // rotation and magnitude constants carry 1/u instead
  constexpr bool FOLD = LENS_MAP_FOLD_U && !SERIES && !POT;
  const float4 F6 = FOLD ? r4[6] : make_float4(0.f, 0.f, 0.f, 0.f), F7 = FOLD ? r4[7] : F6;
  const float dK = FOLD ? D.x : Cq.x, dS = FOLD ? F6.y : Cq.y, q2sc = Cq.z, q2st = Cq.w;
  const float q2dS = FOLD ? F6.z : D.y;
  const float cb = FOLD ? F6.w : E.x, sb = FOLD ? F7.z : E.y, kmag = FOLD ? F7.w : E.z;
  float2 x[NP], y[NP], x2[NP], y2[NP], u2x2[NP], ic[NP], it[NP], psc[NP], pst[NP], Ec[NP], Et[NP];
  float2 Zx[NP], Zy[NP], tx[NP], ty[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float2 cdX = cdx2(c, dX, k), msdX = cdx2(-s, dX, k);  // -(s dX) exactly
    x[k] = fma2(dup2(s), dY[k], cdX);
    y[k] = fma2(dup2(c), dY[k], msdX);
    x2[k] = mul2(x[k], x[k]);
    y2[k] = mul2(y[k], y[k]);
    u2x2[k] = mul2(dup2(u2), x2[k]);
    const float2 R = fma2(dup2(q2), x2[k], y2[k]);
    const float2 pc2 = add2(R, dup2(Kc)), pt2 = add2(R, dup2(Kt));
    ic[k] = rsqrt2(pc2);
    it[k] = rsqrt2(pt2);
    psc[k] = mul2(pc2, ic[k]);
    pst[k] = mul2(pt2, it[k]);
    const float2 Sp = add2(psc[k], pst[k]);
    Ec[k] = add2(psc[k], dup2(sc));
    Et[k] = add2(pst[k], dup2(st));
    Zx[k] = mul2(mul2(x[k], fma2(dup2(dS), Sp, dup2(dK))), rcp2(mul2(Sp, fma2(Ec[k], Et[k], u2x2[k]))));
    const float2 Fc = add2(psc[k], dup2(q2sc)), Ft = add2(pst[k], dup2(q2st));
    Zy[k] = mul2(mul2(y[k], fma2(dup2(q2dS), Sp, dup2(dK))), rcp2(mul2(Sp, fma2(dup2(-u2), y2[k], mul2(Fc, Ft)))));
    if (FOLD) {
      tx[k] = mul2(Zx[k], Zx[k]);
      ty[k] = mul2(Zy[k], Zy[k]);
    } else {
      tx[k] = mul2(dup2(u2), mul2(Zx[k], Zx[k]));
      ty[k] = mul2(dup2(u2), mul2(Zy[k], Zy[k]));
    }
  }
  // the interpolants where every point's |w|^2 < T_SERIES, one branch for
  // all points of the thread (as dpie32)
  float2 axp[NP], ayp[NP];
  bool poly = SERIES;
  if (!SERIES) {
    float t = fmaxf(fmaxf(tx[0].x, tx[0].y), fmaxf(ty[0].x, ty[0].y));
#pragma unroll
    for (int k = 1; k < NP; ++k) t = fmaxf(t, fmaxf(fmaxf(tx[k].x, tx[k].y), fmaxf(ty[k].x, ty[k].y)));
    poly = t < T_SERIES;
  }
  if (poly) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      axp[k] = mul2(Zx[k], horner2(tx[k], LENS_ATAN_W_COEF));
      ayp[k] = mul2(Zy[k], horner2(ty[k], LENS_ATANH_W_COEF));
    }
  } else {
    const float u = r4[6].x, iu = E.w;
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float zx = part2(Zx[k], h), zy = part2(Zy[k], h), tX = part2(tx[k], h), tY = part2(ty[k], h);
        if (fmaxf(tX, tY) < T_SERIES) {
          part2(axp[k], h) = zx * atan_over_w(tX);
          part2(ayp[k], h) = zy * atanh_over_w(tY);
        } else {
          // folded: z is already w = u Z, and the 1/u rides on the constants
          const float wx = FOLD ? zx : u * zx, wy = FOLD ? zy : u * zy, iw = FOLD ? 1.f : iu;
          if (FAST) {
            part2(axp[k], h) = iw * atan_fast(wx);
            part2(ayp[k], h) = iw * (0.346573590f * __log2f((1.f + wy) * rcp_a(1.f - wy)));
          } else {
            part2(axp[k], h) = iw * atanf(wx);
            part2(ayp[k], h) = (0.5f * iw) * log1pf((wy + wy) * rcp_a(1.f - wy));
          }
        }
      }
  }
  if constexpr (POT) {
    // b q (x alpha_x' + y alpha_y') - b q (sc ln sqrt(Dc) - st ln sqrt(Dt)),
    // rounded as dpie32's POT form
    const float bq = 2.f * E.z;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const float2 Dc = fma2(Ec[k], Ec[k], u2x2[k]), Dt = fma2(Et[k], Et[k], u2x2[k]);
      const float2 l2c = make_float2(__log2f(Dc.x), __log2f(Dc.y)), l2t = make_float2(__log2f(Dt.x), __log2f(Dt.y));
      const float2 lg = fma2(dup2(sc), l2c, mul2(dup2(-st), l2t));
      const float2 v = fma2(x[k], axp[k], fma2(y[k], ayp[k], mul2(dup2(-0.346573590f), lg)));
      p.k[k] = fma2(dup2(bq), v, p.k[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      p.ax[k] = fma2(dup2(cb), axp[k], fma2(dup2(-sb), ayp[k], p.ax[k]));
      p.ay[k] = fma2(dup2(sb), axp[k], fma2(dup2(cb), ayp[k], p.ay[k]));
      if (MAG) p.mag[k] = fma2(dup2(kmag), add2(abs2(axp[k]), abs2(ayp[k])), p.mag[k]);  // b q / 2 (/ u folded)
      if (HESS) {
        const float4 G = r4[5];
        const float u2sc2 = D.z, u2st2 = D.w;
        const float2 ymx = sub2(y2[k], x2[k]);
        const float2 Dc = fma2(Ec[k], Ec[k], u2x2[k]), Dt = fma2(Et[k], Et[k], u2x2[k]);
        const float2 fc = rcp2(mul2(psc[k], Dc)), ft = rcp2(mul2(pst[k], Dt));
        const float2 fd = sub2(fc, ft);
        // -(u2sc2 fc - u2st2 ft), rounded as its negation in dpie32
        const float2 g1d = fma2(ymx, fd, fma2(dup2(-u2sc2), fc, mul2(dup2(u2st2), ft)));
        const float2 g2d = mul2(fd, mul2(x[k], y[k]));
        p.k[k] = fma2(dup2(E.z), sub2(ic[k], it[k]), p.k[k]);
        p.g1[k] = fma2(dup2(G.x), g1d, fma2(dup2(G.y), g2d, p.g1[k]));
        p.g2[k] = fma2(dup2(G.z), g1d, fma2(dup2(G.w), g2d, p.g2[k]));
      }
    }
  }
}

// SIS / point mass at NP point pairs: circ32, paired.
// POT: the potential b r (SIS) or b ln r (point mass) into p.k, as circ32.
template <bool HESS, int NP, bool POINT, bool MAG = true, bool POT = false, typename DX>
__device__ __forceinline__ void circ32x2(const float4 *__restrict__ r4, const DX &dX, const float2 (&dY)[NP],
                                         Acc2<HESS, NP> &p) {
  const float b = r4[7].y;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float2 x = dx2_of(dX, k);
    const float2 y = dY[k];
    const float2 r2 = fma2(x, x, mul2(y, y));
    if constexpr (POT) {
      float2 f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float v = part2(r2, h);
        part2(f, h) = v > 0.f ? (POINT ? 0.346573590f * __log2f(v) : v * rsqrt_a(v)) : 0.f;
      }
      p.k[k] = fma2(dup2(b), f, p.k[k]);
    } else {
      float2 ir;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float v = part2(r2, h);
        part2(ir, h) = v > 0.f ? (POINT ? rcp_a(v) : rsqrt_a(v)) : 0.f;
      }
      const float2 f = mul2(dup2(b), ir);
      p.ax[k] = fma2(f, x, p.ax[k]);
      p.ay[k] = fma2(f, y, p.ay[k]);
      if (MAG) p.mag[k] = fma2(dup2(0.5f), add2(abs2(mul2(f, x)), abs2(mul2(f, y))), p.mag[k]);
      if (HESS) {
        const float2 ymx = mul2(sub2(y, x), add2(y, x));
        if (POINT) {
          const float2 f2 = mul2(f, ir);
          p.g1[k] = fma2(f2, ymx, p.g1[k]);
          p.g2[k] = fma2(mul2(dup2(-2.f), f2), mul2(x, y), p.g2[k]);
        } else {
          const float2 f3 = mul2(mul2(f, ir), ir);
          p.k[k] = fma2(dup2(0.5f), f, p.k[k]);
          p.g1[k] = fma2(mul2(dup2(0.5f), f3), ymx, p.g1[k]);
          p.g2[k] = fma2(mul2(f3, dup2(-1.f)), mul2(x, y), p.g2[k]);
        }
      }
    }
  }
}

// Any FP32 potential at NP point pairs.
template <bool HESS, int NP, bool MAG = true, bool FAST = false, typename DX>
__device__ __forceinline__ void eval32x2_any(const float4 *__restrict__ r4, const DX &dX, const float2 (&dY)[NP],
                                             Acc2<HESS, NP> &p) {
  const int kind = __float_as_int(r4[7].x);
  if (kind == K32_DPIE)
    dpie32x2<HESS, NP, false, MAG, FAST>(r4, dX, dY, p);
  else if (kind == K32_DPIE_SERIES)
    dpie32x2<HESS, NP, true, MAG>(r4, dX, dY, p);
  else if (kind == K32_SIS)
    circ32x2<HESS, NP, false, MAG>(r4, dX, dY, p);
  else
    circ32x2<HESS, NP, true, MAG>(r4, dX, dY, p);
}


// ------------------------------------------------------------ double-float
// An unevaluated sum hi + lo of two floats (~48 significant bits) on the FP32
// pipe, for the image polish and the chi2 potentials: GB300's FP64 rate is
// 1/64 of its FP32 rate.
// Error-free transformations: TwoSum (Knuth), FastTwoSum and the product
// error by FMA; compound operations as in Dekker (1971).
struct df {
  float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
  const float p = a.hi * b;
  const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
  return fast_two_sum(p, e);
}
// a + b for operands of one sign (or without severe cancellation): one
// TwoSum on the high parts, error within 2^-47 (|a| + |b|) (Dekker's add).
__device__ __forceinline__ df df_add_ss(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
// a / b: MUFU reciprocal of b.hi, then two exact remainders a - b q
// correct the quotient (its first term may be off by a few 2^-24).
// Code size of the double-float evaluators: their longer operations as
// called functions (one copy per kernel) or inlined at every use.
#ifndef LENS_DF_NOINLINE_DIV
#define LENS_DF_NOINLINE_DIV 0
#endif
#ifndef LENS_DF_NOINLINE_SQRT
#define LENS_DF_NOINLINE_SQRT 0
#endif
#ifndef LENS_DF_NOINLINE_POLY
#define LENS_DF_NOINLINE_POLY 0
#endif
#if LENS_DF_NOINLINE_DIV
static __device__ __noinline__
#else
__device__ __forceinline__
#endif
df df_div(df a, df b) {
  const float ib = rcp_a(b.hi);
  const float q1 = a.hi * ib;
  df r = df_sub(a, df_mulf(b, q1));
  const float q2 = r.hi * ib;
  r = df_sub(r, df_mulf(b, q2));
  const float q3 = r.hi * ib;
  return df_add_ss(fast_two_sum(q1, q2), df{q3, 0.f});
}
// sqrt(a): MUFU reciprocal square root y of a.hi, s = a.hi y, one Newton
// correction (a - s^2) y / 2 with the residual from an FMA.
#if LENS_DF_NOINLINE_SQRT
static __device__ __noinline__
#else
__device__ __forceinline__
#endif
df df_sqrt(df a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  const float y = rsqrt_a(a.hi);
  const float s = a.hi * y;
  const float e = fmaf(-s, s, a.hi) + a.lo;
  return fast_two_sum(s, e * (0.5f * y));
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_from_double(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}

// atan(w)/w, atanh(w)/w on t = w^2 < T_SERIES64 in double-float: the FP64
// interpolants' terms t^7.. (below 5e-7 of the result) in FP32, the rest in
// double-float Horner.
#if LENS_DF_NOINLINE_POLY
static __device__ __noinline__
#else
__device__ __forceinline__
#endif
df df_poly(df t, const float (*c)[2]) {
  float tail = c[11][0];
#pragma unroll
  for (int k = 10; k >= 7; --k) tail = fmaf(tail, t.hi, c[k][0]);
  df p = df_add_ss(df{c[6][0], c[6][1]}, df_mulf(t, tail));
#pragma unroll
  for (int k = 5; k >= 0; --k) p = df_add_ss(df{c[k][0], c[k][1]}, df_mul(p, t));  // |p t| < 0.16 |p|: no cancellation
  return p;
}

// ------------------------------------------------- paired double-float
// Two double-float numbers side by side (component h of hi and lo), so that
// two potentials at one point run through the paired FP32 instructions:
// every operation below is its scalar counterpart above, component by
// component, with the same roundings (a - b as b * (-1) + a).
struct df2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b), bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ df2 df_add2(df2 a, df2 b) {
  df2 s = two_sum2(a.hi, b.hi);
  const df2 t = two_sum2(a.lo, b.lo);
  s = fast_two_sum2(s.hi, add2(s.lo, t.hi));
  return fast_two_sum2(s.hi, add2(s.lo, t.lo));
}
__device__ __forceinline__ df2 df_neg2(df2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ df2 df_sub2(df2 a, df2 b) { return df_add2(a, df_neg2(b)); }
__device__ __forceinline__ df2 df_mul2(df2 a, df2 b) {
  const float2 p = mul2(a.hi, b.hi);
  float2 e = fma2(a.hi, b.hi, neg2(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  return fast_two_sum2(p, e);
}
__device__ __forceinline__ df2 df_mulf2(df2 a, float2 b) {
  const float2 p = mul2(a.hi, b);
  const float2 e = fma2(a.lo, b, fma2(a.hi, b, neg2(p)));
  return fast_two_sum2(p, e);
}
__device__ __forceinline__ df2 df_add_ss2(df2 a, df2 b) {
  const df2 s = two_sum2(a.hi, b.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(a.lo, b.lo)));
}
__device__ __forceinline__ df2 df_div2(df2 a, df2 b) {
  const float2 ib = rcp2(b.hi);
  const float2 q1 = mul2(a.hi, ib);
  df2 r = df_sub2(a, df_mulf2(b, q1));
  const float2 q2 = mul2(r.hi, ib);
  r = df_sub2(r, df_mulf2(b, q2));
  const float2 q3 = mul2(r.hi, ib);
  return df_add_ss2(fast_two_sum2(q1, q2), df2{q3, make_float2(0.f, 0.f)});
}
__device__ __forceinline__ df2 df_sqrt2(df2 a) {
  const float2 y = rsqrt2(a.hi);
  const float2 s = mul2(a.hi, y);
  const float2 e = add2(fma2(neg2(s), s, a.hi), a.lo);
  df2 r = fast_two_sum2(s, mul2(e, mul2(dup2(0.5f), y)));
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (!(part2(a.hi, h) > 0.f)) part2(r.hi, h) = part2(r.lo, h) = 0.f;
  return r;
}
__device__ __forceinline__ df2 df_dup2(df a) { return {dup2(a.hi), dup2(a.lo)}; }
__device__ __forceinline__ df df_part2(const df2 &a, int h) { return {part2(a.hi, h), part2(a.lo, h)}; }
__device__ __forceinline__ df2 df_poly2(df2 t, const float (*c)[2]) {
  float2 tail = dup2(c[11][0]);
#pragma unroll
  for (int k = 10; k >= 7; --k) tail = fma2(tail, t.hi, dup2(c[k][0]));
  df2 p = df_add_ss2(df2{dup2(c[6][0]), dup2(c[6][1])}, df_mulf2(t, tail));
#pragma unroll
  for (int k = 5; k >= 0; --k) p = df_add_ss2(df2{dup2(c[k][0]), dup2(c[k][1])}, df_mul2(p, t));
  return p;
}

// Double-float tables of the same reductions: centre k is the pair's exact
// value c_k ~ tanh(0.8 k), and ATANH_A_DF[k] = atanh(c_k) (60 digits).
__device__ __constant__ const float ATANH_C_DF[23][2] = {
    {0.000000000e+00f, 0.000000000e+00f}, {6.640367508e-01f, 1.947439188e-08f}, {9.216685295e-01f, 2.489597328e-08f},
    {9.836748838e-01f, -2.614878802e-08f}, {9.966824055e-01f, -7.632150911e-09f}, {9.993293285e-01f, -2.879792049e-08f},
    {9.998645782e-01f, -2.654631004e-08f}, {9.999726415e-01f, 1.051378273e-08f}, {9.999944568e-01f, 2.170206415e-08f},
    {9.999988675e-01f, 1.770813363e-08f}, {9.999997616e-01f, 1.334825495e-08f}, {9.999999404e-01f, 1.416372619e-08f},
    {1.000000000e+00f, -9.174363491e-09f}, {1.000000000e+00f, -1.852272002e-09f}, {1.000000000e+00f, -3.739672738e-10f},
    {1.000000000e+00f, -7.550268744e-11f}, {1.000000000e+00f, -1.524372989e-11f}, {1.000000000e+00f, -3.077656185e-12f},
    {1.000000000e+00f, -6.213680286e-13f}, {1.000000000e+00f, -1.254520440e-13f}, {1.000000000e+00f, -2.532833155e-14f},
    {1.000000000e+00f, -5.113701803e-15f}, {1.000000000e+00f, -1.032438613e-15f}};
__device__ __constant__ const float ATANH_A_DF[23][2] = {
    {0.000000000e+00f, 0.000000000e+00f}, {8.000000119e-01f, -1.192092913e-08f}, {1.600000024e+00f, -2.384185827e-08f},
    {2.400000095e+00f, -9.536743306e-08f}, {3.200000048e+00f, -4.768376272e-08f}, {4.000000000e+00f, -1.728711168e-13f},
    {4.800000191e+00f, -1.907355482e-07f}, {5.599999905e+00f, 9.536795176e-08f}, {6.400000095e+00f, -9.532934797e-08f},
    {7.199999809e+00f, 1.907639842e-07f}, {8.000000000e+00f, -1.012165907e-10f}, {8.800000191e+00f, -1.880990936e-07f},
    {9.600000381e+00f, -3.836451583e-07f}, {1.039999962e+01f, 3.922546341e-07f}, {1.119999981e+01f, 1.936774794e-07f},
    {1.200000000e+01f, 2.282851952e-08f}, {1.280000019e+01f, -1.743534028e-07f}, {1.360000038e+01f, -3.974995195e-07f},
    {1.439999962e+01f, 3.966487157e-07f}, {1.519999981e+01f, 1.952836897e-07f}, {1.600000000e+01f, -9.008017443e-09f},
    {1.679999924e+01f, 7.680131375e-07f}, {1.760000038e+01f, -3.882470310e-07f}};
__device__ __constant__ const float ATAN_11_16_DF[2] = {6.022873521e-01f, -5.950149262e-09f};
__device__ __constant__ const float PI_2_DF[2] = {1.570796371e+00f, -4.371138829e-08f};

// atan(w) and atanh(w) in double-float for any argument (|w| < 1 for
// atanh), by the reductions of atan64 / atanh64 (pairs instead of doubles);
// atanh returns NaN beyond the table (|w| within ~1e-15 of 1).
// LENS_DF_NOINLINE_ATAN: df_atan / df_atanh as called functions (one copy
// of their code per kernel instead of one per call site)
#ifndef LENS_DF_NOINLINE_ATAN
#define LENS_DF_NOINLINE_ATAN 0
#endif
#if LENS_DF_NOINLINE_ATAN
#define LENS_DF_ATAN_INLINE static __device__ __noinline__
#else
#define LENS_DF_ATAN_INLINE __device__ __forceinline__
#endif
LENS_DF_ATAN_INLINE df df_atan(df w) {
  const bool neg = w.hi < 0.f;
  const df a = neg ? df_neg(w) : w;
  const bool inv = a.hi > 1.f;
  df v = inv ? df_div(df{1.f, 0.f}, a) : a;
  df base = {0.f, 0.f};
  if (v.hi > 0.4f) {
    v = df_div(df_sub(v, df{0.6875f, 0.f}), df_add_ss(df{1.f, 0.f}, df_mulf(v, 0.6875f)));
    base = df{ATAN_11_16_DF[0], ATAN_11_16_DF[1]};
  }
  df r = df_add(base, df_mul(v, df_poly(df_mul(v, v), C_ATAN_DF)));
  if (inv) r = df_sub(df{PI_2_DF[0], PI_2_DF[1]}, r);
  return neg ? df_neg(r) : r;
}
LENS_DF_ATAN_INLINE df df_atanh(df w) {
  const bool neg = w.hi < 0.f;
  const df a = neg ? df_neg(w) : w;
  df r;
  if (a.hi <= 0.4f) {
    r = df_mul(a, df_poly(df_mul(a, a), C_ATANH_DF));
  } else {
    const df om = df_sub(df{1.f, 0.f}, a);  // 1 - a, exact enough to pick the centre
    const float est = 0.5f * (__logf(1.f + a.hi) - __logf(om.hi));
    const int k = __float2int_rn(est * 1.25f);
    if (!(om.hi > 0.f) || k > 22) return df{__int_as_float(0x7fc00000), 0.f};
    const int kk = k < 1 ? 1 : k;
    const df c = {ATANH_C_DF[kk][0], ATANH_C_DF[kk][1]};
    const df v = df_div(df_sub(a, c), df_sub(df{1.f, 0.f}, df_mul(a, c)));
    r = df_add(df{ATANH_A_DF[kk][0], ATANH_A_DF[kk][1]}, df_mul(v, df_poly(df_mul(v, v), C_ATANH_DF)));
  }
  return neg ? df_neg(r) : r;
}

// One dPIE in double-float at (X, Y) given as pairs: deflection and, if HESS,
// kappa, gamma1, gamma2 into h[0..2] (the forms of eval64; kappa's core-minus-
// cut difference 1/psc - 1/pst as q^2 (st^2 - sc^2) / ((psc + pst) psc pst),
// free of cancellation).  ANY = false: false when |w|^2 >= 0.16 for either
// deflection term (polynomial only, the common case); ANY = true: such terms
// through df_atan / df_atanh, false only for a non-finite result.  Pair k of
// the record is r[k * stride] (stride 1: one record; stride n: field-major
// table of n records).
template <bool ANY, bool HESS = false>
__device__ __forceinline__ bool dpie_df(const float2 *__restrict__ r, int stride, df X, df Y, df &ax, df &ay,
                                        df *h = nullptr) {
  auto ld = [&](int k) {
    const float2 v = r[k * stride];
    return df{v.x, v.y};
  };
  const df c = ld(F_C), s = ld(F_S);
  const df dX = df_sub(X, ld(F_X0)), dY = df_sub(Y, ld(F_Y0));
  // rotations: the one-TwoSum add's error is bounded by 2^-47 |(dX, dY)|
  const df x = df_add_ss(df_mul(c, dX), df_mul(s, dY)), y = df_add_ss(df_mul(c, dY), df_neg(df_mul(s, dX)));
  const df q2 = ld(F_Q2), u2 = ld(F_U2);
  const df x2 = df_mul(x, x), y2 = df_mul(y, y);
  // every sum below adds non-negative terms except dS and the y denominator
  const df R = df_add_ss(df_mul(q2, x2), y2);
  const df psc = df_sqrt(df_add_ss(R, ld(F_KC)));
  const df pst = df_sqrt(df_add_ss(R, ld(F_KT)));
  const df Sp = df_add_ss(psc, pst);
  const df sc = ld(F_SC), st = ld(F_ST);
  const df Ec = df_add_ss(psc, sc), Et = df_add_ss(pst, st);
  const df dS = df_add_ss(st, df_neg(sc));  // st > sc > 0: error 2^-47 (st + sc) < 2^-46 dS
  const df numx = df_mul(df_mul(x, dS), df_add_ss(Sp, ld(F_Q2SS)));
  const df denx = df_mul(Sp, df_add_ss(df_mul(Ec, Et), df_mul(u2, x2)));
  const df Zx = df_div(numx, denx);
  const df Fc = df_add_ss(psc, ld(F_Q2SC)), Ft = df_add_ss(pst, ld(F_Q2ST));
  const df numy = df_mul(df_mul(y, ld(F_Q2DS)), df_add_ss(Sp, ld(F_SS)));
  const df deny = df_mul(Sp, df_sub(df_mul(Fc, Ft), df_mul(u2, y2)));
  const df Zy = df_div(numy, deny);
  const df tx = df_mul(u2, df_mul(Zx, Zx)), ty = df_mul(u2, df_mul(Zy, Zy));
  const df bq = ld(F_BQ);
  df axp, ayp;
  if (tx.hi < (float)T_SERIES64 && ty.hi < (float)T_SERIES64) {  // bq Z atan(w)/w, w = u Z
    axp = df_mul(df_mul(bq, Zx), df_poly(tx, C_ATAN_DF));
    ayp = df_mul(df_mul(bq, Zy), df_poly(ty, C_ATANH_DF));
  } else {
    if (!ANY) return false;  // (also for NaN)
    const df u = df_sqrt(u2), bu = df_div(bq, u);  // (bq / u) atan(u Z)
    axp = df_mul(bu, df_atan(df_mul(u, Zx)));
    ayp = df_mul(bu, df_atanh(df_mul(u, Zy)));
    if (!(fabsf(axp.hi) < INFINITY && fabsf(ayp.hi) < INFINITY)) return false;
  }
  ax = df_add_ss(df_mul(c, axp), df_neg(df_mul(s, ayp)));  // rotation back: error 2^-47 |(axp, ayp)|
  ay = df_add_ss(df_mul(s, axp), df_mul(c, ayp));
  if (HESS) {
    const df r2 = df_add_ss(x2, y2), ymx = df_sub(y2, x2);
    const df Dc = df_add_ss(df_add_ss(ld(F_DC0), df_mul(df_mulf(sc, 2.f), psc)), r2);
    const df Dt = df_add_ss(df_add_ss(ld(F_DT0), df_mul(df_mulf(st, 2.f), pst)), r2);
    const df fc = df_div(df{1.f, 0.f}, df_mul(psc, Dc)), ft = df_div(df{1.f, 0.f}, df_mul(pst, Dt));
    const df hb = ld(F_HB);
    const df g1p = df_mul(hb, df_sub(df_mul(fc, df_sub(ymx, ld(F_U2SC2))), df_mul(ft, df_sub(ymx, ld(F_U2ST2)))));
    const df g2p = df_neg(df_mul(df_mul(bq, df_sub(fc, ft)), df_mul(x, y)));
    h[0] = df_div(df_mul(hb, ld(F_KTC)), df_mul(df_mul(Sp, psc), pst));
    const df c2 = ld(F_C2), s2 = ld(F_S2);
    h[1] = df_sub(df_mul(c2, g1p), df_mul(s2, g2p));
    h[2] = df_add(df_mul(s2, g1p), df_mul(c2, g2p));
  }
  return true;
}

// Two dPIE potentials (records ra, rb, field-major with `stride`) at one
// point in double-float, side by side: dpie_df's arithmetic inside the
// interpolants' range, component by component.  ok[h]: potential h was in
// that range (its results are valid); a potential outside it (a core, or
// NaN) is left to the caller (dpie_df<true> / FP64), as dpie_df<false> does.
template <bool HESS = false>
__device__ __forceinline__ void dpie_df2(const float2 *__restrict__ ra, const float2 *__restrict__ rb, int stride,
                                         df X, df Y, df2 &ax, df2 &ay, df2 *h, bool (&ok)[2]) {
  auto ld = [&](int k) {
    const float2 va = ra[k * stride], vb = rb[k * stride];
    return df2{make_float2(va.x, vb.x), make_float2(va.y, vb.y)};
  };
  const df2 c = ld(F_C), s = ld(F_S);
  const df2 dX = df_sub2(df_dup2(X), ld(F_X0)), dY = df_sub2(df_dup2(Y), ld(F_Y0));
  const df2 x = df_add_ss2(df_mul2(c, dX), df_mul2(s, dY)), y = df_add_ss2(df_mul2(c, dY), df_neg2(df_mul2(s, dX)));
  const df2 q2 = ld(F_Q2), u2 = ld(F_U2);
  const df2 x2 = df_mul2(x, x), y2 = df_mul2(y, y);
  const df2 R = df_add_ss2(df_mul2(q2, x2), y2);
  const df2 psc = df_sqrt2(df_add_ss2(R, ld(F_KC)));
  const df2 pst = df_sqrt2(df_add_ss2(R, ld(F_KT)));
  const df2 Sp = df_add_ss2(psc, pst);
  const df2 sc = ld(F_SC), st = ld(F_ST);
  const df2 Ec = df_add_ss2(psc, sc), Et = df_add_ss2(pst, st);
  const df2 dS = df_add_ss2(st, df_neg2(sc));
  const df2 numx = df_mul2(df_mul2(x, dS), df_add_ss2(Sp, ld(F_Q2SS)));
  const df2 denx = df_mul2(Sp, df_add_ss2(df_mul2(Ec, Et), df_mul2(u2, x2)));
  const df2 Zx = df_div2(numx, denx);
  const df2 Fc = df_add_ss2(psc, ld(F_Q2SC)), Ft = df_add_ss2(pst, ld(F_Q2ST));
  const df2 numy = df_mul2(df_mul2(y, ld(F_Q2DS)), df_add_ss2(Sp, ld(F_SS)));
  const df2 deny = df_mul2(Sp, df_sub2(df_mul2(Fc, Ft), df_mul2(u2, y2)));
  const df2 Zy = df_div2(numy, deny);
  const df2 tx = df_mul2(u2, df_mul2(Zx, Zx)), ty = df_mul2(u2, df_mul2(Zy, Zy));
#pragma unroll
  for (int k = 0; k < 2; ++k)
    ok[k] = part2(tx.hi, k) < (float)T_SERIES64 && part2(ty.hi, k) < (float)T_SERIES64;  // false for NaN
  const df2 bq = ld(F_BQ);
  const df2 axp = df_mul2(df_mul2(bq, Zx), df_poly2(tx, C_ATAN_DF));
  const df2 ayp = df_mul2(df_mul2(bq, Zy), df_poly2(ty, C_ATANH_DF));
  ax = df_add_ss2(df_mul2(c, axp), df_neg2(df_mul2(s, ayp)));
  ay = df_add_ss2(df_mul2(s, axp), df_mul2(c, ayp));
  if (HESS) {
    const df2 r2 = df_add_ss2(x2, y2), ymx = df_sub2(y2, x2);
    const df2 Dc = df_add_ss2(df_add_ss2(ld(F_DC0), df_mul2(df_mulf2(sc, dup2(2.f)), psc)), r2);
    const df2 Dt = df_add_ss2(df_add_ss2(ld(F_DT0), df_mul2(df_mulf2(st, dup2(2.f)), pst)), r2);
    const df2 one = {dup2(1.f), dup2(0.f)};
    const df2 fc = df_div2(one, df_mul2(psc, Dc)), ft = df_div2(one, df_mul2(pst, Dt));
    const df2 hb = ld(F_HB);
    const df2 g1p =
        df_mul2(hb, df_sub2(df_mul2(fc, df_sub2(ymx, ld(F_U2SC2))), df_mul2(ft, df_sub2(ymx, ld(F_U2ST2)))));
    const df2 g2p = df_neg2(df_mul2(df_mul2(bq, df_sub2(fc, ft)), df_mul2(x, y)));
    h[0] = df_div2(df_mul2(hb, ld(F_KTC)), df_mul2(df_mul2(Sp, psc), pst));
    const df2 c2 = ld(F_C2), s2 = ld(F_S2);
    h[1] = df_sub2(df_mul2(c2, g1p), df_mul2(s2, g2p));
    h[2] = df_add2(df_mul2(s2, g1p), df_mul2(c2, g2p));
  }
}

// SIS (F_U2 = -1, b = F_BQ) or point mass (F_U2 = -2, b = theta_E^2 in
// F_BQ) in double-float; zero at the centre.  HESS: kappa, gamma1, gamma2
// into h[0..2].
template <bool HESS = false>
__device__ __forceinline__ void circ_df(const float2 *__restrict__ r, int stride, df X, df Y, df &ax, df &ay,
                                        df *h = nullptr) {
  const float2 x0 = r[F_X0 * stride], y0 = r[F_Y0 * stride], b2 = r[F_BQ * stride];
  const df b = {b2.x, b2.y};
  const df dX = df_sub(X, df{x0.x, x0.y}), dY = df_sub(Y, df{y0.x, y0.y});
  const df r2 = df_add_ss(df_mul(dX, dX), df_mul(dY, dY));
  if (!(r2.hi > 0.f)) {
    ax = ay = df{0.f, 0.f};
    if (HESS) h[0] = h[1] = h[2] = df{0.f, 0.f};
    return;
  }
  const bool point = r[F_U2 * stride].x < -1.5f;
  const df ir2 = df_div(df{1.f, 0.f}, r2);
  const df f = point ? df_mul(b, ir2) : df_mul(b, df_sqrt(ir2));  // b/r^2 or b/r
  ax = df_mul(f, dX);
  ay = df_mul(f, dY);
  if (HESS) {
    // SIS: kappa = b/(2r), gamma = b/(2r^3) (y^2-x^2, -2xy); point: kappa = 0,
    // gamma = b/r^4 (y^2-x^2, -2xy)
    const df g = point ? df_mul(f, ir2) : df_mul(df_mulf(f, 0.5f), ir2);
    h[0] = point ? df{0.f, 0.f} : df_mulf(f, 0.5f);
    h[1] = df_mul(g, df_sub(df_mul(dY, dY), df_mul(dX, dX)));
    h[2] = df_neg(df_mulf(df_mul(g, df_mul(dX, dY)), 2.f));
  }
}

// --------------------------------------------------------- constraint sets
// One potential at (X, Y) from its double-float record (deflection and, if
// HESS, kappa, gamma1, gamma2), added to acc[0..4] as doubles; FP64 from its
// FP64 record when the double-float evaluation fails (|w| within 1e-15 of 1,
// non-finite intermediate).
template <bool HESS>
__device__ __forceinline__ void add_potential_df(const float2 *__restrict__ rdf, int stride,
                                                 const double *__restrict__ r64, double X, double Y, double *acc) {
  const df Xd = df_from_double(X), Yd = df_from_double(Y);
  df ax, ay, h[3];
  bool ok = true;
  if (rdf[F_U2 * stride].x < 0.f)
    circ_df<HESS>(rdf, stride, Xd, Yd, ax, ay, h);
  else
    ok = dpie_df<true, HESS>(rdf, stride, Xd, Yd, ax, ay, h);
  if (ok) {
    acc[0] += df_to_double(ax);
    acc[1] += df_to_double(ay);
    if (HESS) {
      acc[2] += df_to_double(h[0]);
      acc[3] += df_to_double(h[1]);
      acc[4] += df_to_double(h[2]);
    }
  } else {
    double bx, by, bk = 0, b1 = 0, b2 = 0;
    eval64<HESS>(r64, X, Y, bx, by, bk, b1, b2);
    acc[0] += bx;
    acc[1] += by;
    acc[2] += bk;
    acc[3] += b1;
    acc[4] += b2;
  }
}

#ifndef LENS_SRC_UNROLL_V
#define LENS_SRC_UNROLL_V 0  // 1: both evaluations inlined side by side (0.363 -> 0.41 ms: the code outgrows the caches)
#endif
#ifndef LENS_DF_PAIRED
#define LENS_DF_PAIRED 0  // 1: the two varying potentials side by side (dpie_df2): measured 30 % slower
#endif
// The two varying potentials of a parameter set at (X, Y): both in
// double-float, summed in double-float and added to acc[0..4] with one
// conversion each (the FP64 pipe runs at 1/64 of the FP32 rate); FP64 for a
// potential whose double-float evaluation fails.
// The FP64 fallback of the varying potentials out of line (LENS_COLD_CALLS):
// it almost never runs, and inlined it lengthens the hot loop's code
// (source-plane chi2, 4096 sets: 0.365 -> 0.362 ms).
#ifndef LENS_COLD_CALLS
#define LENS_COLD_CALLS 1
#endif
template <bool HESS>
__device__ __noinline__ void eval64_cold(const double *__restrict__ r, double X, double Y, double *e) {
  eval64<HESS>(r, X, Y, e[0], e[1], e[2], e[3], e[4]);
}
// The same with the sum kept in double-float: acc[0..4] pairs (one-TwoSum
// accumulation, absolute error 2^-47 of the summed magnitudes), the point
// also given as pairs (Xd, Yd), so that a term costs no FP64 operation
// unless its double-float evaluation fails.
template <bool HESS>
__device__ __forceinline__ void add_potential_dfs(const float2 *__restrict__ rdf, int stride,
                                                  const double *__restrict__ r64, double X, double Y, df Xd, df Yd,
                                                  df *acc) {
  df ax, ay, h[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  bool ok = true;
  if (rdf[F_U2 * stride].x < 0.f)
    circ_df<HESS>(rdf, stride, Xd, Yd, ax, ay, h);
  else
    ok = dpie_df<true, HESS>(rdf, stride, Xd, Yd, ax, ay, h);
  if (!ok) {
    double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    eval64_cold<HESS>(r64, X, Y, e);
    ax = df_from_double(e[0]);
    ay = df_from_double(e[1]);
    h[0] = df_from_double(e[2]);
    h[1] = df_from_double(e[3]);
    h[2] = df_from_double(e[4]);
  }
  acc[0] = df_add_ss(acc[0], ax);
  acc[1] = df_add_ss(acc[1], ay);
  if (HESS)
#pragma unroll
    for (int q = 0; q < 3; ++q) acc[2 + q] = df_add_ss(acc[2 + q], h[q]);
}

template <bool HESS>
__device__ __forceinline__ void add_varying_df(const float2 *__restrict__ rdf, const double *__restrict__ r64,
                                               double X, double Y, double *acc) {
  const df Xd = df_from_double(X), Yd = df_from_double(Y);
  df sum[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  // both dPIE: the pair side by side (dpie_df2); a potential outside the
  // interpolants' range, an SIS or a point mass takes the scalar path below
  bool pok[2] = {false, false};
  df2 pax, pay, ph[3];
  if (LENS_DF_PAIRED && rdf[F_U2].x >= 0.f && rdf[RECDF + F_U2].x >= 0.f)
    dpie_df2<HESS>(rdf, rdf + RECDF, 1, Xd, Yd, pax, pay, ph, pok);
#if LENS_SRC_UNROLL_V
#pragma unroll
#else
#pragma unroll 1
#endif
  for (int v = 0; v < 2; ++v) {  // not unrolled: one copy of the (large) evaluator in the code
    const float2 *r = rdf + v * RECDF;
    df ax, ay, h[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    bool ok = true;
    if (pok[v]) {
      ax = df_part2(pax, v);
      ay = df_part2(pay, v);
      if (HESS)
        for (int q = 0; q < 3; ++q) h[q] = df_part2(ph[q], v);
    } else if (r[F_U2].x < 0.f) {
      circ_df<HESS>(r, 1, Xd, Yd, ax, ay, h);
    } else {
      ok = dpie_df<true, HESS>(r, 1, Xd, Yd, ax, ay, h);
    }
    if (ok) {
      sum[0] = df_add(sum[0], ax);
      sum[1] = df_add(sum[1], ay);
      if (HESS) {
        sum[2] = df_add(sum[2], h[0]);
        sum[3] = df_add(sum[3], h[1]);
        sum[4] = df_add(sum[4], h[2]);
      }
    } else {
      double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (LENS_COLD_CALLS)
        eval64_cold<HESS>(r64 + v * REC64, X, Y, e);
      else
        eval64<HESS>(r64 + v * REC64, X, Y, e[0], e[1], e[2], e[3], e[4]);
#pragma unroll
      for (int q = 0; q < 5; ++q) acc[q] += e[q];
    }
  }
#pragma unroll
  for (int q = 0; q < (HESS ? 5 : 2); ++q) acc[q] += df_to_double(sum[q]);
}

// Back-trace every constraint of one parameter set in FP64 (Sec. 2.1 Eq. 1):
// beta_j = theta_j - r alpha(theta_j), with alpha = static cache + the two
// varying potentials (FP64 records in s_rec; their double-float records in
// s_rdf, which, when not NULL, evaluate them on the FP32 pipe to ~1e-13),
// then each source's barycentre (Sec. 2.2, Fig. 3).  Fills s_beta [nimg][2],
// s_bary [nsrc][2] and, when s_m is not NULL, r H at every image in
// s_m [nimg][3] (hxx, hyy, hxy).  Must be called by all THREADS threads of
// the CTA; ends synchronised.
template <int THREADS, int HESS = -1>
__device__ __forceinline__ void backtrace_set(const double *__restrict__ stat, const double *__restrict__ x,
                                              const double *__restrict__ y, const double *__restrict__ ratio,
                                              const int32_t *__restrict__ src_of, const int32_t *__restrict__ img_off,
                                              int nimg, int nsrc, const double *s_rec, const float2 *s_rdf,
                                              double *s_beta, double *s_m, double *s_bary) {
  for (int j = threadIdx.x; j < nimg; j += THREADS) {
    const double X = x[j], Y = y[j];
    const double *st = stat + (size_t)j * 5;
    double acc[5] = {st[0], st[1], st[2], st[3], st[4]};
    if (s_rdf) {
      if (HESS == 1 || (HESS < 0 && s_m))
        add_varying_df<true>(s_rdf, s_rec, X, Y, acc);
      else
        add_varying_df<false>(s_rdf, s_rec, X, Y, acc);
    } else {
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        double bx, by, bk = 0, b1 = 0, b2 = 0;
        if (s_m)
          eval64<true>(s_rec + v * REC64, X, Y, bx, by, bk, b1, b2);
        else
          eval64<false>(s_rec + v * REC64, X, Y, bx, by, bk, b1, b2);
        acc[0] += bx;
        acc[1] += by;
        acc[2] += bk;
        acc[3] += b1;
        acc[4] += b2;
      }
    }
    const double r = ratio[src_of[j]];
    s_beta[2 * j] = X - r * acc[0];
    s_beta[2 * j + 1] = Y - r * acc[1];
    if (s_m) {
      s_m[3 * j] = r * (acc[2] + acc[3]);
      s_m[3 * j + 1] = r * (acc[2] - acc[3]);
      s_m[3 * j + 2] = r * acc[4];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nsrc; i += THREADS) {
    const int b = img_off[i], e = img_off[i + 1];
    double sx = 0, sy = 0;
    for (int j = b; j < e; ++j) {
      sx += s_beta[2 * j];
      sy += s_beta[2 * j + 1];
    }
    const double im = e > b ? 1.0 / (e - b) : 0.0;
    s_bary[2 * i] = sx * im;
    s_bary[2 * i + 1] = sy * im;
  }
  __syncthreads();
}

// Deterministic CTA sum of NV doubles per thread; the result is valid in
// thread 0.  s_red holds (THREADS/32) * NV doubles.  Ends synchronised.
template <int NV, int THREADS>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) s_red[warp * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < THREADS / 32; ++w) s += s_red[w * NV + k];
      v[k] = s;
    }
  __syncthreads();
}

// Varying-potential records of parameter set q (14 numbers) into s_rec[2][16];
// returns (to threads 0 and 1) whether the set is inside the model's domain.
__device__ __forceinline__ bool load_var_rec64(const double *q, int type0, int type1, int v, double *s_rec) {
  const double *w = q + 7 * v;
  const int type = v == 0 ? type0 : type1;
  make_rec64(type, w[0], w[1], w[3], w[2], w[4], w[5], w[6], s_rec + v * REC64);
  return halo_params_ok(type, w[0], w[1], w[3], w[2], w[4], w[5], w[6]);
}

}  // namespace lens
