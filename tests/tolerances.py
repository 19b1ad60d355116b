"""Numeric tolerances of the GPU paths against the FP64 oracle.

Derived from the arithmetic (FP32 ulp = 6e-8; compensated sums; FP64
cluster-scale potentials).  All checks are element by element.

LENS_MIXED maps (FP32 bulk):
  alpha:  |d alpha| <= 1e-6 * max(|alpha_ref|, 1e-3 * max|alpha_ref|)
          -- relative 1e-6 where the deflection is not near a zero crossing;
          within 1e-3 of the map's peak deflection it becomes an absolute
          bound of 1e-9 x peak.
  kappa, gamma1, gamma2: |d| <= 1e-5 * max(|ref|, 1)  (they enter as 1 - kappa)
  mu:     |d det| <= 3e-5 absolute, det = 1/mu = (1-k)^2 - g^2 (equivalently
          mu relative 3e-5/|det|, the form that means something where
          |det| >= 1e-2), plus the rounding of mu to the FP32 output plane
          (|d det| <= 2^-24 |det| from that alone, which passes 3e-5 where
          |det| > 500: next to the cores of concentrated FP32 potentials).
LENS_FP64 maps: relative 1e-11 (floor 1e-3 x peak) on every plane.
chi2: relative 1e-8 (FP64 on both sides), absolute floor 1e-12 for chi2 ~ 0.
Potential maps (phi is defined up to a constant; its additive part
b q s_t ln s_t is large next to its variation over the field):
  LENS_FP64: |d phi| <= 1e-11 * max|phi_ref|;
  LENS_MIXED: |d phi| <= 1e-6 * (max phi_ref - min phi_ref) + 1e-9 * max|phi_ref|
          -- each FP32 member carries ~1e-7 of its own b q s_t ln D_t term
          (~1e-5 arcsec^2 for the members of a cluster model), a few 1e-4
          over 1000 of them, against a variation of ~1e3-1e4 arcsec^2.
"""
import numpy as np

ALPHA_REL = 1e-6
ALPHA_FLOOR_FRAC = 1e-3
HESS_ABS = 1e-5
DET_ABS = 3e-5
CHI2_REL = 1e-8
POT_FP64_REL = 1e-11
POT_RANGE_REL = 1e-6
POT_ABS_REL = 1e-9


def pot_mixed_tol(ref):
    """Absolute bound on |d phi| of a LENS_MIXED potential map (see above)."""
    return POT_RANGE_REL * (ref.max() - ref.min()) + POT_ABS_REL * np.abs(ref).max()


def alpha_violations(ax, ay, rx, ry, rel=ALPHA_REL, floor_frac=ALPHA_FLOOR_FRAC, peak=None):
    """Nodes outside the deflection tolerance; `peak` is the map's largest
    |alpha| (default: the largest among the nodes compared)."""
    ra = np.hypot(rx, ry)
    err = np.hypot(ax - rx, ay - ry)
    tol = rel * np.maximum(ra, floor_frac * (ra.max() if peak is None else peak))
    return err > tol, err, tol


def hess_violations(k, g1, g2, rk, rg1, rg2, atol=HESS_ABS):
    bad = np.zeros(np.shape(k), dtype=bool)
    for a, r in ((k, rk), (g1, rg1), (g2, rg2)):
        bad |= np.abs(a - r) > atol * np.maximum(np.abs(r), 1.0)
    return bad


MU_STORE_REL = 2.0 ** -24   # rounding of mu (and so of det) to the FP32 plane


def mu_violations(mu, rmu, det_atol=DET_ABS, stored_fp32=True):
    det = 1.0 / np.asarray(mu, dtype=np.float64)
    rdet = 1.0 / np.asarray(rmu, dtype=np.float64)
    return np.abs(det - rdet) > det_atol + (MU_STORE_REL * np.abs(rdet) if stored_fp32 else 0.0)


def report(name, bad, err=None):
    n = int(np.count_nonzero(bad))
    msg = f"{name}: {n} of {bad.size} outside tolerance"
    if err is not None:
        msg += f" (max err {np.max(err):.3e})"
    return n, msg
