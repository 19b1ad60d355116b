"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module draws random numbers and lays them out; it holds none of the
lensing arithmetic (no deflection, Hessian, lens equation or chi2).  Both the
CUDA library and the CPU oracle consume exactly these arrays.

Halo table layout (float64, one row per halo), the ``lens_halo`` fields of the
C ABI in order::

    [type, x0, y0, theta, eps, rcore, rcut, b0]

``type``: 0 = dPIE, 1 = SIS, 2 = point mass.  Angles in radians measured
counter-clockwise from +x to the major axis; lengths in arcsec; ``eps`` is the
dPIE ellipticity (a-b)/(a+b) of Elíasdóttir et al. (2007), the profile family
the paper cites for its parametric sub-halos (Sec. 2.2).

Workload shapes follow the paper's benchmark model (Sec. 5: ~200 potentials,
80 sources, 227 images, a 150"x150" field at HST sampling) scaled to the sizes
named in the module-level ``CFG*`` constants.  The paper's own cluster model
and constraints are not public inputs here, so these seeded stand-ins replace
them.
"""
from __future__ import annotations

import numpy as np

DPIE, SIS, POINT = 0, 1, 2

# Parameter order of one varying halo inside a parameter set (7 per halo,
# 2 varying halos -> 14 numbers per set).
PARAM_FIELDS = ("x0", "y0", "eps", "theta", "rcore", "rcut", "b0")
_COL = {"type": 0, "x0": 1, "y0": 2, "theta": 3, "eps": 4, "rcore": 5, "rcut": 6, "b0": 7}

FIELD = (-100.0, 100.0, -100.0, 100.0)  # xmin, xmax, ymin, ymax (arcsec)


def halo_row(type_, x0, y0, theta, eps, rcore, rcut, b0):
    return np.array([type_, x0, y0, theta, eps, rcore, rcut, b0], dtype=np.float64)


def grid(n, field=FIELD, ny=None):
    """Grid descriptor: inclusive corners, row-major [j][i] with j along y."""
    xmin, xmax, ymin, ymax = field
    return dict(xmin=float(xmin), xmax=float(xmax), ymin=float(ymin), ymax=float(ymax),
                nx=int(n), ny=int(ny if ny is not None else n))


def cfg1_model(seed=1):
    """10 dPIE halos: one cluster halo at the origin plus 9 galaxies."""
    rng = np.random.default_rng(seed)
    rows = [halo_row(DPIE, 0.0, 0.0, 0.0, 0.3, 5.0, 1000.0, 30.0)]
    for _ in range(9):
        x0, y0 = rng.uniform(-60, 60, 2)
        b0 = float(np.exp(rng.uniform(np.log(0.5), np.log(3.0))))
        rc = rng.uniform(0.05, 0.2)
        rt = rng.uniform(10, 60)
        eps = rng.uniform(0, 0.6)
        th = rng.uniform(0, np.pi)
        rows.append(halo_row(DPIE, x0, y0, th, eps, rc, rt, b0))
    return np.stack(rows)


def cfg2_model(seed=2, n_members=998, rcut_star=8.0):
    """2 cluster-scale dPIE halos + luminosity-scaled members (1000 halos).

    Members: log10(L/L*) ~ N(-0.5, 0.4) clipped to [-2, 0.7];
    b0 = 1.0"(L/L*)^1/2 (b0 ~ sigma^2, sigma ~ L^1/4), rcore = 0.15"(L/L*)^1/2,
    rcut = rcut_star (L/L*)^1/2 with rcut_star = 8" by default (~45 kpc at
    z ~ 0.5); centres Gaussian (40") about the origin clipped to the field;
    eps U(0, 0.6); theta U(0, pi).  rcut_star changes no other draw.
    """
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(2):
        x0, y0 = rng.uniform(-20, 20, 2)
        rows.append(halo_row(DPIE, x0, y0, rng.uniform(0, np.pi), rng.uniform(0.1, 0.5),
                             rng.uniform(3, 10), rng.uniform(500, 1500), rng.uniform(20, 40)))
    logl = np.clip(rng.normal(-0.5, 0.4, n_members), -2.0, 0.7)
    l = 10.0 ** logl
    xy = np.clip(rng.normal(0.0, 40.0, (n_members, 2)), -100.0, 100.0)
    eps = rng.uniform(0, 0.6, n_members)
    th = rng.uniform(0, np.pi, n_members)
    for k in range(n_members):
        s = np.sqrt(l[k])
        rows.append(halo_row(DPIE, xy[k, 0], xy[k, 1], th[k], eps[k], 0.15 * s, rcut_star * s, 1.0 * s))
    return np.stack(rows)


def member_model(n, seed, field=60.0):
    """n galaxy-scale dPIE halos on the luminosity scaling of cfg2_model
    (b0 <= 2.3"), uniform centres in +/- field."""
    rng = np.random.default_rng(seed)
    l = 10.0 ** np.clip(rng.normal(-0.5, 0.4, n), -2.0, 0.7)
    rows = []
    for k in range(n):
        s = np.sqrt(l[k])
        x0, y0 = rng.uniform(-field, field, 2)
        rows.append(halo_row(DPIE, x0, y0, rng.uniform(0, np.pi), rng.uniform(0, 0.6), 0.15 * s, 8.0 * s, s))
    return np.stack(rows)


def random_model(n, seed, types=(DPIE,), field=60.0, eps_max=0.6):
    """Mixed random model for parity tests (any halo count, any type mix)."""
    rng = np.random.default_rng(seed)
    rows = []
    for k in range(n):
        t = types[k % len(types)]
        x0, y0 = rng.uniform(-field, field, 2)
        if t == DPIE:
            rc = float(np.exp(rng.uniform(np.log(0.05), np.log(5.0))))
            rows.append(halo_row(DPIE, x0, y0, rng.uniform(0, np.pi), rng.uniform(0, eps_max),
                                 rc, rc * float(np.exp(rng.uniform(np.log(3), np.log(300)))),
                                 float(np.exp(rng.uniform(np.log(0.3), np.log(20))))))
        else:
            rows.append(halo_row(t, x0, y0, 0.0, 0.0, 0.0, 0.0, rng.uniform(0.3, 5.0)))
    return np.stack(rows)


def var_params_of(model, var_halo):
    """The 14 varying parameters of halos var_halo[0], var_halo[1] as a vector."""
    out = []
    for h in var_halo:
        out.extend(model[h, _COL[f]] for f in PARAM_FIELDS)
    return np.array(out, dtype=np.float64)


def perturbed_params(model, var_halo, P, seed):
    """P parameter sets: Gaussian perturbations of the two varying halos.

    Widths: 1" on centres, 2% on b0/rcore/rcut, 0.02 on eps (kept in
    [0, 0.95]), 0.05 rad on theta.  Returns float64 [P][14].
    """
    rng = np.random.default_rng(seed)
    base = var_params_of(model, var_halo)
    out = np.tile(base, (P, 1))
    for k in range(2):
        o = 7 * k
        out[:, o + 0] += rng.normal(0, 1.0, P)
        out[:, o + 1] += rng.normal(0, 1.0, P)
        out[:, o + 2] = np.clip(out[:, o + 2] + rng.normal(0, 0.02, P), 0.0, 0.95)
        out[:, o + 3] += rng.normal(0, 0.05, P)
        out[:, o + 4] *= 1.0 + rng.normal(0, 0.02, P)
        out[:, o + 5] *= 1.0 + rng.normal(0, 0.02, P)
        out[:, o + 6] *= 1.0 + rng.normal(0, 0.02, P)
    return out


def constraints_dict(img_off, x, y, sigma, dls_ds):
    return dict(img_off=np.ascontiguousarray(img_off, dtype=np.int32),
                x=np.ascontiguousarray(x, dtype=np.float64),
                y=np.ascontiguousarray(y, dtype=np.float64),
                sigma=np.ascontiguousarray(sigma, dtype=np.float64),
                dls_ds=np.ascontiguousarray(dls_ds, dtype=np.float64))


def random_constraints(nsrc, seed, mult=(2, 7), field=60.0, sigma=0.1,
                       ratios=(0.5, 0.6, 0.7, 0.8, 0.9)):
    """Constraint table with random positions (no lens equation involved).

    Useful wherever the chi2 is needed as a function of arbitrary inputs; the
    physically consistent multiple-image sets are produced by the script in
    tests/golden that solves the lens equation with the oracle.
    """
    rng = np.random.default_rng(seed)
    m = rng.integers(mult[0], mult[1] + 1, nsrc)
    off = np.concatenate([[0], np.cumsum(m)]).astype(np.int32)
    n = int(off[-1])
    return constraints_dict(off, rng.uniform(-field, field, n), rng.uniform(-field, field, n),
                            np.full(n, sigma), rng.choice(np.asarray(ratios, dtype=np.float64), nsrc))


def source_candidates(n, seed, radius=25.0, ratios=(0.5, 0.6, 0.7, 0.8, 0.9)):
    """Candidate source positions (uniform in a disc) and per-source D_ls/D_s."""
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.uniform(0, 1, n))
    a = rng.uniform(0, 2 * np.pi, n)
    return r * np.cos(a), r * np.sin(a), rng.choice(np.asarray(ratios, dtype=np.float64), n)


def load_constraints(path):
    """A constraint table stored as JSON (img_off, x, y, dls_ds, sigma)."""
    import json
    with open(path) as f:
        d = json.load(f)
    n = len(d["x"])
    sig = d["sigma"]
    return constraints_dict(d["img_off"], d["x"], d["y"], np.full(n, sig) if np.isscalar(sig) else sig, d["dls_ds"])


def gaussian_noise(n, seed, sigma):
    return np.random.default_rng(seed).normal(0.0, sigma, (n, 2))
