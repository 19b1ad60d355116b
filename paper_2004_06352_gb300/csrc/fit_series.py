"""Coefficients of the polynomials for atan(w)/w and atanh(w)/w in t = w^2 on
[0, T] used by lens_device.cuh: FP32 (atan_over_w / atanh_over_w, degree 4
by default, 5 as a build option)
and FP64 (atan_over_w64 / atanh_over_w64, degree 11; also split into float
hi/lo pairs for the double-float evaluator), and the tables of the FP64
atan/atanh argument reduction (atan64 / atanh64).

Both interpolate the exact functions at the DEG+1 Chebyshev nodes of [0, T]:
the FP32 set with numpy (Chebyshev fit converted to monomials), the FP64 set
by solving the interpolation conditions in the monomial basis with 60-digit
mpmath arithmetic (the float64 conversion would lose digits).  Prints the
coefficients and the worst relative error on a dense grid.

  python paper_2004_06352_gb300/csrc/fit_series.py [FP32 degree]
"""
import numpy as np
from numpy.polynomial import chebyshev as Ch
from numpy.polynomial import polynomial as Pn

T, DEG = 0.16, 4


def f_atan(t):
    w = np.sqrt(t)
    return np.where(t > 0, np.arctan(w) / np.where(w > 0, w, 1), 1.0)


def f_atanh(t):
    w = np.sqrt(t)
    return np.where(t > 0, np.arctanh(w) / np.where(w > 0, w, 1), 1.0)


def fit(f):
    k = np.arange(DEG + 1)
    x = np.cos(np.pi * (k + 0.5) / (DEG + 1))
    c = Ch.chebfit(x, f(0.5 * T * (x + 1)), DEG)
    P = np.zeros(DEG + 1)
    for i, a in enumerate(Ch.cheb2poly(c)):          # x = 2t/T - 1
        P = Pn.polyadd(P, a * Pn.polypow([-1.0, 2.0 / T], i))[:DEG + 1]
    return P


def fp32_horner(P, t):
    c = P.astype(np.float32)
    acc = np.full(t.shape, c[-1], dtype=np.float32)
    for a in c[-2::-1]:
        acc = (acc.astype(np.float64) * t + a).astype(np.float32)
    return acc


def fit64(name, deg=11):
    import mpmath as mp
    mp.mp.dps = 60
    T64 = mp.mpf(T)
    f = {"atan": mp.atan, "atanh": mp.atanh}[name]
    g = lambda t: mp.mpf(1) if t == 0 else f(mp.sqrt(t)) / mp.sqrt(t)
    nodes = [T64 / 2 * (1 + mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (deg + 1))) for k in range(deg + 1)]
    A = mp.matrix([[t ** j for j in range(deg + 1)] for t in nodes])
    c = mp.lu_solve(A, mp.matrix([g(t) for t in nodes]))
    worst = max(abs(sum(c[j] * t ** j for j in range(deg + 1)) / g(t) - 1)
                for t in (T64 * i / 2000 for i in range(2001)))
    return [float(c[j]) for j in range(deg + 1)], float(worst)


def reduction_tables(step="0.8", kmax=22):
    """Centres of the FP64 atanh argument reduction: c_k = tanh(step k)
    rounded to double and the 60-digit atanh of that double; atan(11/16) and
    pi/2 as hi + lo."""
    import mpmath as mp
    mp.mp.dps = 60
    c = [float(mp.tanh(mp.mpf(step) * k)) for k in range(kmax + 1)]
    a = [float(mp.atanh(mp.mpf(v))) for v in c]
    pi2 = mp.pi / 2
    return c, a, float(mp.atan(mp.mpf(11) / 16)), float(pi2), float(pi2 - mp.mpf(float(pi2)))


if __name__ == "__main__":
    import sys
    if len(sys.argv) > 1:
        DEG = int(sys.argv[1])
    tt = np.linspace(0, T, 200001)
    t32 = tt.astype(np.float32).astype(np.float64)
    for name, f in (("atan", f_atan), ("atanh", f_atanh)):
        P = fit(f)
        e = np.max(np.abs(Pn.polyval(tt, P) / f(tt) - 1))
        e32 = np.max(np.abs(fp32_horner(P, t32) / f(t32) - 1))
        print(f"{name}: max rel err {e:.2e} (exact arithmetic), {e32:.2e} (FP32 Horner)")
        print("  " + ", ".join(f"{v:.9e}f" for v in P))
    for name in ("atan", "atanh"):
        c, worst = fit64(name)
        print(f"{name} (FP64, degree 11): max rel interpolation error {worst:.2e}")
        print("  " + ", ".join(f"{v:.17e}" for v in c))
        # the double-float table: each coefficient split into float hi + float lo
        hi = np.array(c).astype(np.float32)
        lo = (np.array(c) - hi.astype(np.float64)).astype(np.float32)
        print("  pairs: " + ", ".join(f"{{{h:.9e}f, {l:.9e}f}}" for h, l in zip(hi, lo)))
    c, a, at, ph, pl = reduction_tables()
    print("ATANH_C:", ", ".join(repr(v) for v in c))
    print("ATANH_A:", ", ".join(repr(v) for v in a))
    print("ATAN_11_16:", repr(at), " PI_2_HI, PI_2_LO:", repr(ph), repr(pl))
