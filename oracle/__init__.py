"""FP64 CPU oracle for the parametric lens model -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
it shares no code with the CUDA path: the arithmetic lives in
``lens_oracle.c`` (plain C, double precision), compiled here with gcc and
called through ctypes.  Each wrapper below names the paper passage the C
function follows; the formulas themselves are documented at the top of the C
file.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, finite differences,
analytic image positions, brute force).  Bit-level agreement with the original
Lenstool code is not pinned (no code or worked example is available); the
pins fix the mathematics instead.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lens_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblens_oracle.so")
_lock = threading.Lock()
_lib = None
_override = None  # path of an alternative build (the mutation tests load mutants)


class Halo(C.Structure):
    _fields_ = [("type", C.c_int32), ("x0", C.c_double), ("y0", C.c_double), ("theta", C.c_double),
                ("eps", C.c_double), ("rcore", C.c_double), ("rcut", C.c_double), ("b0", C.c_double)]


class Constraints(C.Structure):
    _fields_ = [("nsrc", C.c_int32), ("off", C.POINTER(C.c_int32)), ("x", C.POINTER(C.c_double)),
                ("y", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("dls_ds", C.POINTER(C.c_double))]


class Grid(C.Structure):
    _fields_ = [("xmin", C.c_double), ("xmax", C.c_double), ("ymin", C.c_double), ("ymax", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


def build(force=False):
    """Compile lens_oracle.c into oracle/_build/liblens_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(_override or build())
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
        hp, cp, gp = C.POINTER(Halo), C.POINTER(Constraints), C.POINTER(Grid)
        sig = {
            "or_num_threads": (C.c_int, []),
            "or_set_threads": (None, [C.c_int]),
            "or_halo_eval": (None, [hp, C.c_double, C.c_double, dp]),
            "or_halo_potential": (C.c_double, [hp, C.c_double, C.c_double]),
            "or_halo_kappa": (C.c_double, [hp, C.c_double, C.c_double]),
            "or_model_eval_points": (None, [hp, C.c_int32, dp, dp, C.c_int64, C.c_double, dp]),
            "or_model_potential_points": (None, [hp, C.c_int32, dp, dp, C.c_int64, C.c_double, dp]),
            "or_model_kappa_points": (None, [hp, C.c_int32, dp, dp, C.c_int64, C.c_double, dp]),
            "or_maps": (None, [hp, C.c_int32, gp, C.c_double, C.c_int32, dp]),
            "or_apply_params": (None, [hp, C.c_int32, ip, dp, hp]),
            "or_backtrace": (None, [hp, C.c_int32, cp, dp, dp]),
            "or_chi2_source": (C.c_double, [hp, C.c_int32, cp, C.c_int32]),
            "or_chi2_source_batch": (None, [hp, C.c_int32, cp, ip, dp, C.c_int32, C.c_int32, dp]),
            "or_newton": (C.c_int32, [hp, C.c_int32, C.c_double, C.c_double, C.c_double, dp, dp, C.c_int32,
                                      C.c_double, C.c_double]),
            "or_find_images": (C.c_int32, [hp, C.c_int32, gp, dp, C.c_double, C.c_double, C.c_double,
                                           C.c_int32, C.c_double, C.c_double, dp, C.c_int32, ip]),
            "or_alpha_grid": (None, [hp, C.c_int32, gp, dp]),
            "or_chi2_image": (C.c_double, [hp, C.c_int32, cp, gp, dp, C.c_int32, C.c_double, C.c_double,
                                           C.c_int32, ip]),
            "or_chi2_image_batch": (None, [hp, C.c_int32, cp, gp, ip, dp, C.c_int32, C.c_int32, C.c_double,
                                           C.c_double, C.c_int32, dp, ip]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def use_library(path):
    """Route every wrapper to the library at `path` (None: the normal build).
    Used by the tests that load deliberately broken copies of the oracle."""
    global _lib, _override
    with _lock:
        _override = path
        _lib = None


def build_variant(src_text, out_path):
    """Compile C source text (a modified copy of lens_oracle.c) to out_path."""
    src = out_path[:-3] + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", out_path, src, "-lm"],
                   check=True)
    return out_path


def source_text():
    with open(_SRC) as f:
        return f.read()


# ----------------------------------------------------------------- marshalling

def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def halos_from_table(table):
    """Halo table rows [type, x0, y0, theta, eps, rcore, rcut, b0] -> ctypes array."""
    t = np.asarray(table, dtype=np.float64).reshape(-1, 8)
    arr = (Halo * max(len(t), 1))()
    for k, r in enumerate(t):
        arr[k] = Halo(int(r[0]), *map(float, r[1:]))
    return arr, len(t)


class _ConstraintsRef:
    """Keeps the numpy buffers alive for as long as the ctypes struct is used."""

    def __init__(self, cons):
        self.off = np.ascontiguousarray(cons["img_off"], dtype=np.int32)
        self.x = np.ascontiguousarray(cons["x"], dtype=np.float64)
        self.y = np.ascontiguousarray(cons["y"], dtype=np.float64)
        self.sigma = np.ascontiguousarray(cons["sigma"], dtype=np.float64)
        self.dls = np.ascontiguousarray(cons["dls_ds"], dtype=np.float64)
        self.c = Constraints(len(self.off) - 1, _ip(self.off), _dp(self.x), _dp(self.y), _dp(self.sigma),
                             _dp(self.dls))


def _grid(g):
    return Grid(g["xmin"], g["xmax"], g["ymin"], g["ymax"], g["nx"], g["ny"])


def num_threads():
    return int(_load().or_num_threads())


def set_threads(n):
    """OpenMP threads of later calls (e.g. 1 to time a single core)."""
    _load().or_set_threads(int(n))


# ------------------------------------------------------------------ evaluation

def halo_eval(row, X, Y):
    """One potential at one point, D_ls/D_s = 1: (ax, ay, hxx, hyy, hxy).
    Per-potential derivatives of Sec. 4.1 Eq. 10 / Sec. 2.4 Eqs. 7-9."""
    lib = _load()
    h, _ = halos_from_table(row)
    out = np.zeros(5)
    lib.or_halo_eval(h, float(X), float(Y), _dp(out))
    return out


def model_eval(table, X, Y, dls_ds=1.0):
    """Summed (ax, ay, hxx, hyy, hxy) at points X, Y (Sec. 4.1 Eq. 10): [npt, 5]."""
    lib = _load()
    h, n = halos_from_table(table)
    X = np.ascontiguousarray(np.atleast_1d(X), dtype=np.float64)
    Y = np.ascontiguousarray(np.atleast_1d(Y), dtype=np.float64)
    out = np.zeros((len(X), 5))
    lib.or_model_eval_points(h, n, _dp(X), _dp(Y), len(X), float(dls_ds), _dp(out))
    return out


def potential(table, X, Y, dls_ds=1.0):
    """Lensing potential (Sec. 2.1 Eq. 2, up to a constant) at points."""
    lib = _load()
    h, n = halos_from_table(table)
    X = np.ascontiguousarray(np.atleast_1d(X), dtype=np.float64)
    Y = np.ascontiguousarray(np.atleast_1d(Y), dtype=np.float64)
    out = np.zeros(len(X))
    lib.or_model_potential_points(h, n, _dp(X), _dp(Y), len(X), float(dls_ds), _dp(out))
    return out


def kappa_profile(table, X, Y, dls_ds=1.0):
    """Surface density from the profile definitions (not from the Hessian)."""
    lib = _load()
    h, n = halos_from_table(table)
    X = np.ascontiguousarray(np.atleast_1d(X), dtype=np.float64)
    Y = np.ascontiguousarray(np.atleast_1d(Y), dtype=np.float64)
    out = np.zeros(len(X))
    lib.or_model_kappa_points(h, n, _dp(X), _dp(Y), len(X), float(dls_ds), _dp(out))
    return out


def maps(table, grid, dls_ds=1.0, nplanes=6):
    """Map planes [nplanes, ny, nx]: ax, ay (+ kappa, gamma1, gamma2, mu).
    Sec. 2.4 Eqs. 7-9 and Sec. 2.1 Eqs. 4-5 over the grid of Sec. 4.1."""
    lib = _load()
    h, n = halos_from_table(table)
    g = _grid(grid)
    out = np.zeros((nplanes, grid["ny"], grid["nx"]))
    lib.or_maps(h, n, C.byref(g), float(dls_ds), int(nplanes), _dp(out))
    return out


def apply_params(table, var_halo, p14):
    """Model with halos var_halo[0..1] replaced by the 14 parameters."""
    lib = _load()
    h, n = halos_from_table(table)
    out = (Halo * n)()
    var = np.asarray(var_halo, dtype=np.int32)
    p = np.ascontiguousarray(p14, dtype=np.float64)
    lib.or_apply_params(h, n, _ip(var), _dp(p), out)
    return np.array([[o.type, o.x0, o.y0, o.theta, o.eps, o.rcore, o.rcut, o.b0] for o in out])


def apply_params_scaled(table, var_halo, p16):
    """Model with the two varying halos from p16[0:14], and the members'
    scaling relations moved (Sec. 2.2: b0_i = b0* s_i, r_cut,i = r_cut* s_i):
    every other potential's b0 times p16[14], every other dPIE's r_cut times
    p16[15]."""
    t = apply_params(table, var_halo, p16[:14])
    others = np.array([i for i in range(len(t)) if i not in tuple(var_halo)], dtype=int)
    t[others, 7] *= p16[14]
    dp = others[t[others, 0] == 0]
    t[dp, 6] *= p16[15]
    return t


def chi2_source_scaled_batch(table, cons, var_halo, params16, variant=0):
    """Source-plane chi2 of each 16-parameter set; NaN outside the domain
    (f_b or f_t not positive, a member's r_cut not above its r_core, or the
    varying halos' own domain)."""
    params16 = np.asarray(params16, dtype=np.float64).reshape(-1, 16)
    out = np.full(len(params16), np.nan)
    for k, p in enumerate(params16):
        if not (p[14] > 0 and p[15] > 0 and params_in_domain(table, var_halo, p[:14])):
            continue
        t = apply_params_scaled(table, var_halo, p)
        if np.any((t[:, 0] == 0) & ~(t[:, 6] > t[:, 5])):
            continue
        out[k] = chi2_source(t, cons, variant)
    return out


def backtrace(table, cons):
    """beta_ij = theta_ij - alpha(theta_ij) (Sec. 2.1 Eq. 1) and per-source
    barycentres (Sec. 2.2, Fig. 3).  Returns (beta [nimg, 2], bary [nsrc, 2])."""
    lib = _load()
    h, n = halos_from_table(table)
    cr = _ConstraintsRef(cons)
    beta = np.zeros((len(cr.x), 2))
    bary = np.zeros((cr.c.nsrc, 2))
    lib.or_backtrace(h, n, C.byref(cr.c), _dp(beta), _dp(bary))
    return beta, bary


def chi2_source(table, cons, variant=0):
    """Source-plane chi2 of one model (Sec. 2.2 Eq. 6, source-plane form)."""
    lib = _load()
    h, n = halos_from_table(table)
    cr = _ConstraintsRef(cons)
    return float(lib.or_chi2_source(h, n, C.byref(cr.c), int(variant)))


def chi2_source_batch(table, cons, var_halo, params, variant=0):
    lib = _load()
    h, n = halos_from_table(table)
    cr = _ConstraintsRef(cons)
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 14)
    var = np.asarray(var_halo, dtype=np.int32)
    out = np.zeros(len(params))
    lib.or_chi2_source_batch(h, n, C.byref(cr.c), _ip(var), _dp(params), len(params), int(variant), _dp(out))
    return out


# ---------------------------------------------------------------- sampling
# Metropolis steps over the varying potentials' parameters (the Bayesian fit
# of Sec. 2.2: likelihood exp(-chi2/2) of the source-plane chi2, Eq. 6) with
# the counter-based generator Philox4x64-10 of Salmon, Moraes, Dror and Shaw
# ("Parallel random numbers: as easy as 1, 2, 3", SC 2011), written here in
# plain Python integers from that definition.

_PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
_PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
_M64 = (1 << 64) - 1


def philox4x64_10(counter, key):
    """Philox4x64 with 10 rounds: four 64-bit counter words, two key words."""
    c0, c1, c2, c3 = (int(v) & _M64 for v in counter)
    k0, k1 = (int(v) & _M64 for v in key)
    for _ in range(10):
        p0, p1 = _PHILOX_M[0] * c0, _PHILOX_M[1] * c2
        c0, c1, c2, c3 = (p1 >> 64) ^ c1 ^ k0, p1 & _M64, (p0 >> 64) ^ c3 ^ k1, p0 & _M64
        k0, k1 = (k0 + _PHILOX_W[0]) & _M64, (k1 + _PHILOX_W[1]) & _M64
    return c0, c1, c2, c3


def mcmc_uniforms(seed, step, W):
    """[W][17] uniforms in (0, 1): chain w's words are Philox with counter
    (step, w, j, 0), key (seed, 0): the 16 words of j = 0..3 (the Box-Muller
    inputs), then word 0 of j = 4 (the acceptance uniform); word x gives
    ((x >> 11) + 1/2) 2^-53."""
    out = np.empty((W, 17))
    for w in range(W):
        words = []
        for j in range(4):
            words.extend(philox4x64_10((step, w, j, 0), (seed, 0)))
        words.append(philox4x64_10((step, w, 4, 0), (seed, 0))[0])
        out[w] = [((x >> 11) + 0.5) * 2.0 ** -53 for x in words]
    return out


def params_in_domain(table, var_halo, p14):
    """The parameter set is inside the model's domain: every field finite,
    b0 > 0, and for a dPIE 0 <= eps < 1 and 0 < rcore < rcut."""
    table = np.asarray(table)
    for v in range(2):
        x0, y0, eps, theta, rcore, rcut, b0 = (float(t) for t in p14[7 * v: 7 * v + 7])
        if not all(np.isfinite([x0, y0, eps, theta, rcore, rcut, b0])) or not b0 > 0:
            return False
        if int(table[var_halo[v], 0]) == 0 and not (0.0 <= eps < 1.0 and 0.0 < rcore < rcut):
            return False
    return True


def gaussian_proposals(params, sigma, u):
    """Random-walk proposals params + sigma z, z standard normal from the
    Box-Muller transform of consecutive pairs of the uniforms u [W][npar]
    (radius sqrt(-2 ln u_2i), angle 2 pi u_2i+1; cosine to parameter 2i,
    sine to 2i+1)."""
    params = np.asarray(params, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    z = np.empty(params.shape)
    for i in range(params.shape[-1] // 2):
        rad = np.sqrt(-2.0 * np.log(u[:, 2 * i]))
        ang = 2.0 * np.pi * u[:, 2 * i + 1]
        z[:, 2 * i] = rad * np.cos(ang)
        z[:, 2 * i + 1] = rad * np.sin(ang)
    return params + np.asarray(sigma, dtype=np.float64) * z


def metropolis_accept(chi2, chi2p, u, temperature):
    """Metropolis decision for the likelihood exp(-chi2/2) of Sec. 2.2 (Eq. 6)
    tempered by 1/T: a chain moves to its proposal when the uniform u is below
    the likelihood ratio (L'/L)^(1/T) = exp(-(chi2' - chi2) / (2T)), compared
    in logarithms.  A proposal outside the domain (chi2' NaN) never moves; a
    chain whose current chi2 is NaN takes any valid proposal."""
    chi2 = np.asarray(chi2, dtype=np.float64)
    chi2p = np.asarray(chi2p, dtype=np.float64)
    return np.isfinite(chi2p) & (~np.isfinite(chi2) |
                                 (np.log(u) < -(chi2p - chi2) / (2.0 * temperature)))


def mcmc_step(table, cons, var_halo, params, chi2, sigma, temperature, seed, step, variant=0):
    """One Metropolis step of W chains over 14 parameters (chi2 as
    chi2_source_batch) or 16 (with the members' scaling factors, chi2 as
    chi2_source_scaled_batch): proposals theta + sigma z with z from
    Box-Muller pairs of the uniforms, chi2 of the proposals (NaN outside the
    domain), move when ln u < -(chi2' - chi2) / (2 T) (any valid proposal
    when chi2 is NaN).  Returns (params', chi2', accepted, proposals, chi2 of
    the proposals)."""
    params = np.asarray(params, dtype=np.float64)
    npar = params.shape[-1]
    params = params.reshape(-1, npar)
    chi2 = np.asarray(chi2, dtype=np.float64)
    W = len(params)
    u = mcmc_uniforms(seed, step, W)
    prop = gaussian_proposals(params, sigma, u[:, :npar])
    if npar == 16:
        chi2p = chi2_source_scaled_batch(table, cons, var_halo, prop, variant)
    else:
        ok = np.array([params_in_domain(table, var_halo, p) for p in prop])
        chi2p = np.full(W, np.nan)
        if ok.any():
            chi2p[ok] = chi2_source_batch(table, cons, var_halo, prop[ok], variant)
    take = metropolis_accept(chi2, chi2p, u[:, 16], temperature)
    new_p = np.where(take[:, None], prop, params)
    new_c = np.where(take, chi2p, chi2)
    return new_p, new_c, take, prop, chi2p


def newton(table, r, beta_s, theta0, maxit=40, tol=1e-6, step_max=0.0):
    """Newton solve of beta_s = theta - r alpha(theta); returns (theta, iters or -1)."""
    lib = _load()
    h, n = halos_from_table(table)
    tx, ty = C.c_double(theta0[0]), C.c_double(theta0[1])
    it = lib.or_newton(h, n, float(r), float(beta_s[0]), float(beta_s[1]), C.byref(tx), C.byref(ty),
                       int(maxit), float(tol), float(step_max))
    return np.array([tx.value, ty.value]), int(it)


def alpha_grid(table, grid):
    lib = _load()
    h, n = halos_from_table(table)
    g = _grid(grid)
    out = np.zeros((grid["ny"], grid["nx"], 2))
    lib.or_alpha_grid(h, n, C.byref(g), _dp(out))
    return out


def find_images(table, grid, r, beta_s, maxit=40, tol=1e-6, dedup=1e-3, cap=64, ag=None, with_difficulty=False):
    """Brute-force predicted images of one source (Sec. 2.3 Fig. 4; Sec. 4.2).
    With with_difficulty, also each image's difficulty (100 x refinement cut
    short + Newton iterations of its easiest candidate)."""
    lib = _load()
    h, n = halos_from_table(table)
    g = _grid(grid)
    if ag is None:
        ag = alpha_grid(table, grid)
    ag = np.ascontiguousarray(ag, dtype=np.float64)
    img = np.zeros((cap, 2))
    diff = np.zeros(cap, dtype=np.int32)
    nf = lib.or_find_images(h, n, C.byref(g), _dp(ag), float(r), float(beta_s[0]), float(beta_s[1]), int(maxit),
                            float(tol), float(dedup), _dp(img), int(cap), _ip(diff))
    k = min(nf, cap)
    if with_difficulty:
        return img[:k].copy(), int(nf), diff[:k].copy()
    return img[:k].copy(), int(nf)


def chi2_image(table, cons, grid, maxit=40, tol=1e-6, dedup=1e-3, cap=64, ag=None):
    """Image-plane chi2 of one model (Sec. 2.2 Eq. 6 with the brute-force
    search of Sec. 2.3 / Sec. 4.2).  Returns (chi2, nfound[nsrc])."""
    lib = _load()
    h, n = halos_from_table(table)
    cr = _ConstraintsRef(cons)
    g = _grid(grid)
    agp = None
    if ag is not None:
        ag = np.ascontiguousarray(ag, dtype=np.float64)
        agp = _dp(ag)
    nf = np.zeros(cr.c.nsrc, dtype=np.int32)
    v = lib.or_chi2_image(h, n, C.byref(cr.c), C.byref(g), agp, int(maxit), float(tol), float(dedup), int(cap),
                          _ip(nf))
    return float(v), nf


def chi2_image_batch(table, cons, grid, var_halo, params, maxit=40, tol=1e-6, dedup=1e-3, cap=64):
    lib = _load()
    h, n = halos_from_table(table)
    cr = _ConstraintsRef(cons)
    g = _grid(grid)
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 14)
    var = np.asarray(var_halo, dtype=np.int32)
    out = np.zeros(len(params))
    nf = np.zeros((len(params), cr.c.nsrc), dtype=np.int32)
    lib.or_chi2_image_batch(h, n, C.byref(cr.c), C.byref(g), _ip(var), _dp(params), len(params), int(maxit),
                            float(tol), float(dedup), int(cap), _dp(out), _ip(nf))
    return out, nf
