// Device-side building blocks shared by the map and chi2 kernels:
// approximate MUFU reciprocals, mbarrier + 1-D bulk-copy (TMA) helpers with
// bounded waits, and the FP64 evaluation of one potential.
#pragma once

#include "lens_internal.cuh"

namespace lens {

// Bound on any spin on an mbarrier: ~2^24 try_wait polls (seconds), after
// which the kernel records LENS_ERR_WAIT and leaves instead of hanging.
constexpr unsigned WAIT_LIMIT = 1u << 24;
constexpr int LENS_ERR_WAIT = 1;

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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
  for (unsigned i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

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
  double psc = sqrt(R + q2 * sc * sc), pst = sqrt(R + q2 * st * st);
  double Sp = psc + pst;
  double Ec = psc + sc, Et = pst + st;
  double Zx = x * dS * (Sp + q2 * sS) / (Sp * (Ec * Et + u2 * x2));
  double Fc = psc + q2 * sc, Ft = pst + q2 * st;
  double Zy = y * q2 * dS * (Sp + sS) / (Sp * (Fc * Ft - u2 * y2));
  double axp, ayp;
  if (kind == K64_DPIE_SERIES) {
    double wx = u2 * Zx * Zx, wy = u2 * Zy * Zy;
    axp = bq * Zx * (1.0 - wx / 3.0 + wx * wx / 5.0);
    ayp = bq * Zy * (1.0 + wy / 3.0 + wy * wy / 5.0);
  } else {
    axp = bq / u * atan(u * Zx);
    ayp = bq / u * atanh(u * Zy);
  }
  ax = c * axp - s * ayp;
  ay = s * axp + c * ayp;
  if (HESS) {
    double r2 = x2 + y2, ymx = y2 - x2;
    double Dc = (1.0 + q2) * sc * sc + 2.0 * sc * psc + r2;
    double Dt = (1.0 + q2) * st * st + 2.0 * st * pst + r2;
    double fc = 1.0 / (psc * Dc), ft = 1.0 / (pst * Dt);
    double g1p = 0.5 * bq * (fc * (ymx - u2 * sc * sc) - ft * (ymx - u2 * st * st));
    double g2p = -bq * (fc - ft) * x * y;
    kap = 0.5 * bq * (1.0 / psc - 1.0 / pst);
    double c2 = r[D_C2T], s2 = r[D_S2T];
    g1 = c2 * g1p - s2 * g2p;
    g2 = s2 * g1p + c2 * g2p;
  }
}

}  // namespace lens
