"""Pins of the FP64 oracle to facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: a closed
form derived independently (circular mass integral, SIS / point-mass lens
solutions), a conservation law (Gauss's theorem for the deflection field), an
invariant (symmetry, linearity, reflection, rotation covariance), finite
differences, or brute force.  Chosen so that a dropped term, a wrong sign or
index, or a transposed operand anywhere in the oracle fails at least one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2004_06352_gb300 import inputs as I

DPIE, SIS, POINT = I.DPIE, I.SIS, I.POINT


def circ_dpie_alpha(b0, rc, rt, r):
    """Circular dPIE deflection from the enclosed mass: alpha(r) = 2/r int_0^r kappa r' dr'
    with kappa = (b0/2)[(rc^2+r^2)^-1/2 - (rt^2+r^2)^-1/2]."""
    return b0 * ((math.sqrt(rc * rc + r * r) - rc) - (math.sqrt(rt * rt + r * r) - rt)) / r


# --------------------------------------------------------------- closed forms

@pytest.mark.parametrize("eps", [0.0, 1e-9, 1e-7])
def test_circular_limit_matches_enclosed_mass(eps):
    """eps -> 0 (incl. the series branch): radial deflection = enclosed-mass closed form."""
    b0, rc, rt = 7.0, 0.8, 40.0
    h = I.halo_row(DPIE, 1.5, -2.0, 0.3, eps, rc, rt, b0)
    rng = np.random.default_rng(0)
    for _ in range(30):
        r = float(np.exp(rng.uniform(np.log(0.01), np.log(500))))
        phi = rng.uniform(0, 2 * np.pi)
        v = oracle.halo_eval(h, 1.5 + r * math.cos(phi), -2.0 + r * math.sin(phi))
        a_exp = circ_dpie_alpha(b0, rc, rt, r)
        # radial, pointing away from the centre
        assert abs(v[0] - a_exp * math.cos(phi)) <= 1e-12 * b0 + 10 * eps * b0
        assert abs(v[1] - a_exp * math.sin(phi)) <= 1e-12 * b0 + 10 * eps * b0


def test_sis_and_point_mass_closed_forms():
    rng = np.random.default_rng(1)
    for _ in range(20):
        b = rng.uniform(0.5, 5)
        dx, dy = rng.normal(0, 10, 2)
        r = math.hypot(dx, dy)
        s = oracle.halo_eval(I.halo_row(SIS, 3.0, 4.0, 0, 0, 0, 0, b), 3.0 + dx, 4.0 + dy)
        assert np.allclose(s[:2], [b * dx / r, b * dy / r], rtol=1e-14)
        assert math.isclose(0.5 * (s[2] + s[3]), b / (2 * r), rel_tol=1e-13)  # kappa = b/(2r)
        p = oracle.halo_eval(I.halo_row(POINT, 3.0, 4.0, 0, 0, 0, 0, b), 3.0 + dx, 4.0 + dy)
        assert np.allclose(p[:2], [b * b * dx / r ** 2, b * b * dy / r ** 2], rtol=1e-14)
        assert abs(p[2] + p[3]) < 1e-14 * b * b / r ** 2  # point mass: kappa = 0 off-centre
    # exact centre: defined as zero
    assert np.all(oracle.halo_eval(I.halo_row(SIS, 1, 1, 0, 0, 0, 0, 2.0), 1, 1) == 0)
    assert np.all(oracle.halo_eval(I.halo_row(POINT, 1, 1, 0, 0, 0, 0, 2.0), 1, 1) == 0)


# ------------------------------------------------- kappa vs the profile itself

def test_half_trace_equals_profile_kappa():
    """kappa = (psi_xx + psi_yy)/2 (Sec. 2.4 Eq. 7) equals the dPIE definition
    evaluated directly -- pins b = b0(1+e), q = (1-e)/(1+e), s = r(1+e)."""
    m = I.random_model(40, seed=3, types=(DPIE, SIS, POINT))
    rng = np.random.default_rng(4)
    X, Y = rng.uniform(-80, 80, 400), rng.uniform(-80, 80, 400)
    ev = oracle.model_eval(m, X, Y, 0.7)
    k_prof = oracle.kappa_profile(m, X, Y, 0.7)
    assert np.allclose(0.5 * (ev[:, 2] + ev[:, 3]), k_prof, rtol=1e-11, atol=1e-13)


def test_gauss_law_flux_and_zero_circulation():
    """div alpha = 2 kappa and curl alpha = 0: the flux of alpha through a circle
    equals twice the enclosed mass (2-D quadrature of the profile kappa), and
    the circulation vanishes.  Pins the deflection's normalisation and
    orientation for elliptical halos independently of its formula."""
    h = I.halo_row(DPIE, 0.5, -0.3, 0.7, 0.4, 1.2, 30.0, 5.0)
    for R in (0.7, 3.0, 20.0):
        nphi = 2048
        phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
        X, Y = 0.5 + R * np.cos(phi), -0.3 + R * np.sin(phi)
        ev = oracle.model_eval(h, X, Y)
        flux = np.sum(ev[:, 0] * np.cos(phi) + ev[:, 1] * np.sin(phi)) * R * 2 * np.pi / nphi
        circ = np.sum(-ev[:, 0] * np.sin(phi) + ev[:, 1] * np.cos(phi)) * R * 2 * np.pi / nphi
        # enclosed mass: Gauss-Legendre in r, trapezoid (periodic) in phi
        xr, wr = np.polynomial.legendre.leggauss(400)
        rr = 0.5 * R * (xr + 1)
        wr = 0.5 * R * wr
        RR, PP = np.meshgrid(rr, phi, indexing="ij")
        kap = oracle.kappa_profile(h, (0.5 + RR * np.cos(PP)).ravel(), (-0.3 + RR * np.sin(PP)).ravel())
        mass = np.sum(kap.reshape(RR.shape) * RR * wr[:, None]) * 2 * np.pi / nphi
        assert math.isclose(flux, 2 * mass, rel_tol=2e-9), (R, flux, 2 * mass)
        assert abs(circ) < 1e-10 * abs(flux)


def test_far_field_monopole():
    """|theta| >> rcut: alpha -> M/(pi r) with M = pi (1-e^2) b0 (rcut - rcore).
    The enclosed mass approaches M as M(1 - O(rcut/r)), so at r = 1e8 the
    relative deviation is ~5e-8."""
    for eps in (0.0, 0.3, 0.6):
        b0, rc, rt = 2.0, 0.2, 10.0
        h = I.halo_row(DPIE, 0, 0, 0.4, eps, rc, rt, b0)
        r = 1e8
        for phi in (0.1, 1.3, 2.9):
            v = oracle.halo_eval(h, r * math.cos(phi), r * math.sin(phi))
            M = (1 - eps * eps) * b0 * (rt - rc)
            assert math.isclose(math.hypot(v[0], v[1]) * r, M, rel_tol=2e-7)


# --------------------------------------------------------- finite differences

def test_finite_differences_potential_alpha_hessian():
    """alpha = grad psi and H = grad alpha (Sec. 2.1), by central differences
    (h = 1e-4"), plus Hessian symmetry d(ax)/dy = d(ay)/dx."""
    m = I.random_model(12, seed=5, types=(DPIE, DPIE, SIS, POINT))
    rng = np.random.default_rng(6)
    h = 1e-4
    X, Y = rng.uniform(-70, 70, 60), rng.uniform(-70, 70, 60)
    f = lambda dx, dy: oracle.model_eval(m, X + dx, Y + dy)
    ev = f(0, 0)
    pot = lambda dx, dy: oracle.potential(m, X + dx, Y + dy)
    ax_fd = (pot(h, 0) - pot(-h, 0)) / (2 * h)
    ay_fd = (pot(0, h) - pot(0, -h)) / (2 * h)
    scale = np.abs(ev[:, :2]).max() + 1
    assert np.max(np.abs(ax_fd - ev[:, 0])) < 1e-7 * scale
    assert np.max(np.abs(ay_fd - ev[:, 1])) < 1e-7 * scale
    exp, eyp, exm, eym = f(h, 0), f(0, h), f(-h, 0), f(0, -h)
    hxx = (exp[:, 0] - exm[:, 0]) / (2 * h)
    hyy = (eyp[:, 1] - eym[:, 1]) / (2 * h)
    hxy_a = (eyp[:, 0] - eym[:, 0]) / (2 * h)
    hxy_b = (exp[:, 1] - exm[:, 1]) / (2 * h)
    hs = np.abs(ev[:, 2:]).max() + 1
    assert np.max(np.abs(hxx - ev[:, 2])) < 1e-6 * hs
    assert np.max(np.abs(hyy - ev[:, 3])) < 1e-6 * hs
    assert np.max(np.abs(hxy_a - ev[:, 4])) < 1e-6 * hs
    assert np.max(np.abs(hxy_b - ev[:, 4])) < 1e-6 * hs


def test_potential_differences_are_line_integrals_of_alpha():
    """psi(B) - psi(A) equals the line integral of alpha from A to B (Sec. 2.1:
    alpha = grad psi), by Gauss-Legendre quadrature along paths that pass
    within a core radius of dPIE centres and across the whole field, so that
    a constant that differed between branches or regions of the potential
    (which finite differences at isolated points would not see) fails; the
    SIS and point-mass potentials are b r and b^2 ln r exactly."""
    m = I.random_model(9, seed=7, types=(DPIE, DPIE, DPIE, SIS, POINT))
    m[0, 4] = 0.002  # one dPIE on the small-ellipticity series branch
    xg, wg = np.polynomial.legendre.leggauss(40)
    rng = np.random.default_rng(8)
    for k in range(12):
        # from a random point to a point next to a dPIE centre (or across the field)
        A = rng.uniform(-70, 70, 2)
        B = m[k % 3, 1:3] + rng.normal(0, 0.5 * m[k % 3, 5] + 1e-3, 2) if k < 9 else rng.uniform(-70, 70, 2)
        # piecewise straight path avoiding SIS / point-mass centres: 64 segments
        nodes = np.linspace(0.0, 1.0, 65)
        total = 0.0
        for a0, a1 in zip(nodes[:-1], nodes[1:]):
            t = 0.5 * (a1 - a0) * xg + 0.5 * (a1 + a0)
            P = A[None, :] + t[:, None] * (B - A)[None, :]
            ev = oracle.model_eval(m, P[:, 0], P[:, 1])
            total += 0.5 * (a1 - a0) * np.sum(wg * (ev[:, 0] * (B - A)[0] + ev[:, 1] * (B - A)[1]))
        dpsi = oracle.potential(m, B[0], B[1])[0] - oracle.potential(m, A[0], A[1])[0]
        scale = np.abs(oracle.model_eval(m, np.array([A[0], B[0]]), np.array([A[1], B[1]]))[:, :2]).max() * np.hypot(*(B - A))
        assert abs(dpsi - total) < 1e-9 * scale + 1e-12, (k, dpsi, total)
    rng = np.random.default_rng(9)
    for _ in range(10):
        b = rng.uniform(0.5, 5)
        dx, dy = rng.normal(0, 10, 2)
        r = math.hypot(dx, dy)
        ps = oracle.potential(I.halo_row(SIS, 3.0, 4.0, 0, 0, 0, 0, b)[None], 3.0 + dx, 4.0 + dy)[0]
        assert math.isclose(ps, b * r, rel_tol=1e-13)
        pp = oracle.potential(I.halo_row(POINT, 3.0, 4.0, 0, 0, 0, 0, b)[None], 3.0 + dx, 4.0 + dy)[0]
        assert math.isclose(pp, b * b * math.log(r), rel_tol=1e-12, abs_tol=1e-12)


def test_magnification_from_finite_difference_jacobian():
    """mu = 1/det(d beta/d theta) (Sec. 2.1 Eqs. 4-5), with the sign of the
    shear term as in det = (1-k)^2 - g^2 (the sum in Sec. 2.4 Eq. 9 is a typo)."""
    m = I.cfg1_model()
    g = I.grid(9, field=(-40, 40, -40, 40))
    mp = oracle.maps(m, g, 0.7, 6)
    xs = np.linspace(-40, 40, 9)
    h = 1e-5
    for j in range(0, 9, 2):
        for i in range(0, 9, 2):
            X, Y = xs[i], xs[j]
            beta = lambda x, y: np.array([x, y]) - oracle.model_eval(m, x, y, 0.7)[0, :2]
            J = np.column_stack([(beta(X + h, Y) - beta(X - h, Y)) / (2 * h),
                                 (beta(X, Y + h) - beta(X, Y - h)) / (2 * h)])
            mu_fd = 1.0 / np.linalg.det(J)
            assert math.isclose(mp[5, j, i], mu_fd, rel_tol=1e-6, abs_tol=1e-9)
            # gamma1 = (Hxx - Hyy)/2, gamma2 = Hxy with H = I - J
            H = np.eye(2) - J
            assert abs(mp[2, j, i] - 0.5 * (H[0, 0] + H[1, 1])) < 1e-7
            assert abs(mp[3, j, i] - 0.5 * (H[0, 0] - H[1, 1])) < 1e-7
            assert abs(mp[4, j, i] - H[0, 1]) < 1e-7


# ------------------------------------------------------------------ invariants

def test_linearity_and_distance_scaling():
    a = I.random_model(7, seed=8, types=(DPIE, SIS))
    b = I.random_model(5, seed=9, types=(DPIE, POINT))
    rng = np.random.default_rng(10)
    X, Y = rng.uniform(-50, 50, 100), rng.uniform(-50, 50, 100)
    ab = oracle.model_eval(np.vstack([a, b]), X, Y, 0.63)
    sep = oracle.model_eval(a, X, Y, 0.63) + oracle.model_eval(b, X, Y, 0.63)
    assert np.allclose(ab, sep, rtol=1e-13, atol=1e-13)
    assert np.allclose(oracle.model_eval(a, X, Y, 0.63), 0.63 * oracle.model_eval(a, X, Y, 1.0), rtol=1e-14,
                       atol=1e-15)


def test_point_reflection_and_rotation_covariance():
    """alpha(c+d) = -alpha(c-d), H(c+d) = H(c-d); theta -> theta + pi is the same
    halo; rotating halo and point together by phi rotates alpha by phi and H
    as R H R^T."""
    rng = np.random.default_rng(11)
    for _ in range(10):
        cx, cy = rng.uniform(-20, 20, 2)
        h = I.halo_row(DPIE, cx, cy, rng.uniform(0, np.pi), rng.uniform(0, 0.7), 0.5, 25.0, 3.0)
        d = rng.normal(0, 8, 2)
        p = oracle.halo_eval(h, cx + d[0], cy + d[1])
        mneg = oracle.halo_eval(h, cx - d[0], cy - d[1])
        assert np.allclose(p[:2], -mneg[:2], rtol=1e-12, atol=1e-14)
        assert np.allclose(p[2:], mneg[2:], rtol=1e-12, atol=1e-14)
        h2 = h.copy()
        h2[3] += np.pi
        assert np.allclose(oracle.halo_eval(h2, cx + d[0], cy + d[1]), p, rtol=1e-12, atol=1e-13)
        phi = rng.uniform(0, 2 * np.pi)
        R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
        h3 = h.copy()
        h3[3] += phi
        dr = R @ d
        q = oracle.halo_eval(h3, cx + dr[0], cy + dr[1])
        assert np.allclose(q[:2], R @ p[:2], rtol=1e-11, atol=1e-13)
        Hp = np.array([[p[2], p[4]], [p[4], p[3]]])
        Hq = R @ Hp @ R.T
        assert np.allclose([q[2], q[3], q[4]], [Hq[0, 0], Hq[1, 1], Hq[0, 1]], rtol=1e-11, atol=1e-13)


def test_major_axis_orientation():
    """Along the major axis the density falls off more slowly: kappa at distance
    r along theta exceeds kappa at r along theta + pi/2 (pins the rotation sign
    and which axis eps stretches)."""
    th = 0.6
    h = I.halo_row(DPIE, 0, 0, th, 0.4, 1.0, 50.0, 4.0)
    r = 5.0
    ev_major = oracle.model_eval(h, r * math.cos(th), r * math.sin(th))
    ev_minor = oracle.model_eval(h, -r * math.sin(th), r * math.cos(th))
    assert 0.5 * (ev_major[0, 2] + ev_major[0, 3]) > 1.5 * 0.5 * (ev_minor[0, 2] + ev_minor[0, 3])


# -------------------------------------------------------------------- images

def test_sis_and_point_mass_images():
    """Brute-force search + Newton reproduces the analytic image positions:
    SIS theta = beta +/- theta_E; point mass theta = (beta +/- sqrt(beta^2+4 tE^2))/2."""
    g = I.grid(65, field=(-10, 10, -10, 10))
    for typ in (SIS, POINT):
        tE = 2.3
        m = I.halo_row(typ, 0.0, 0.0, 0, 0, 0, 0, tE)[None]
        for beta in (0.37, 1.1):
            phi = 0.4
            bs = beta * np.array([math.cos(phi), math.sin(phi)])
            img, nf = oracle.find_images(m, g, 1.0, bs)
            if typ == SIS:
                radii = sorted([beta + tE, beta - tE])
            else:
                radii = sorted([0.5 * (beta + math.sqrt(beta ** 2 + 4 * tE ** 2)),
                                0.5 * (beta - math.sqrt(beta ** 2 + 4 * tE ** 2))])
            assert nf == 2, (typ, beta, img)
            signed = sorted(float(np.dot(x, bs) / beta) for x in img)
            assert np.allclose(signed, radii, atol=1e-9)


def test_circular_dpie_images_vs_bisection():
    """Circular dPIE: images lie on the source axis at the roots of
    beta = r - alpha(r) (signed r), found here by bisection on the closed form."""
    b0, rc, rt = 6.0, 0.6, 80.0
    m = I.halo_row(DPIE, 0, 0, 0, 0.0, rc, rt, b0)[None]
    g = I.grid(81, field=(-12, 12, -12, 12))
    beta = 0.5
    f = lambda r: r - math.copysign(circ_dpie_alpha(b0, rc, rt, abs(r)), r) - beta if r != 0 else -beta
    grid_r = np.linspace(-11.9, 11.9, 20001)
    roots = []
    fv = [f(r) for r in grid_r]
    for k in range(len(grid_r) - 1):
        if fv[k] == 0 or fv[k] * fv[k + 1] < 0:
            lo, hi = grid_r[k], grid_r[k + 1]
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if f(lo) * f(mid) <= 0:
                    hi = mid
                else:
                    lo = mid
            roots.append(0.5 * (lo + hi))
    assert len(roots) == 3
    img, nf = oracle.find_images(m, g, 1.0, (beta, 0.0))
    assert nf == 3
    assert np.allclose(sorted(img[:, 0]), sorted(roots), atol=1e-9)
    assert np.allclose(img[:, 1], 0.0, atol=1e-9)


def test_image_search_brute_force_tiny_grid():
    """On a tiny elliptical model, every found image solves the lens equation,
    and a dense brute-force scan of |beta(theta) - beta_s| finds no solution the
    triangle search missed (each scan minimum below 0.05" lies at a found image)."""
    m = np.vstack([I.halo_row(DPIE, 0.3, -0.2, 0.5, 0.35, 0.7, 60.0, 5.0),
                   I.halo_row(DPIE, 4.0, 2.5, 1.9, 0.2, 0.1, 8.0, 0.8)])
    g = I.grid(48, field=(-12, 12, -12, 12))
    bs = np.array([0.4, 0.25])
    img, nf = oracle.find_images(m, g, 0.8, bs)
    assert nf >= 3
    for x in img:
        b = x - oracle.model_eval(m, x[0], x[1], 0.8)[0, :2]
        assert np.linalg.norm(b - bs) < 1e-8
    n = 600
    xs = np.linspace(-12, 12, n)
    XX, YY = np.meshgrid(xs, xs)
    ev = oracle.model_eval(m, XX.ravel(), YY.ravel(), 0.8)
    d = np.hypot(XX.ravel() - ev[:, 0] - bs[0], YY.ravel() - ev[:, 1] - bs[1]).reshape(n, n)
    from scipy.ndimage import minimum_filter
    mins = (d == minimum_filter(d, size=5)) & (d < 0.05)
    for j, i in zip(*np.nonzero(mins)):
        p = np.array([xs[i], xs[j]])
        assert np.min(np.linalg.norm(img - p, axis=1)) < 0.2, p


# ----------------------------------------------------------------------- chi2

def _sis_images(b, beta):
    """Analytic SIS images of a source at beta (|beta| < b): beta/|beta| (|beta| +/- b)."""
    n = np.linalg.norm(beta)
    u = beta / n
    return [u * (n + b), u * (n - b)]


def test_chi2_zero_for_noise_free_constraints():
    """Constraints that are exact images of one source give chi2 = 0 in all
    source-plane variants and in the image-plane form (Sec. 2.2 Eq. 6)."""
    b = 3.0
    m = I.halo_row(SIS, 0, 0, 0, 0, 0, 0, b)[None]
    srcs = [np.array([0.5, 0.2]), np.array([-0.7, 1.1])]
    xs, ys, off = [], [], [0]
    for s in srcs:
        for p in _sis_images(b, s):
            xs.append(p[0])
            ys.append(p[1])
        off.append(len(xs))
    cons = I.constraints_dict(off, xs, ys, np.full(len(xs), 0.1), np.ones(2))
    for variant in (0, 1, 2):
        assert oracle.chi2_source(m, cons, variant) < 1e-24
    g = I.grid(81, field=(-8, 8, -8, 8))
    chi2, nf = oracle.chi2_image(m, cons, g)
    assert list(nf) == [2, 2]
    assert chi2 < 1e-12


def test_chi2_image_plane_sis_closed_form():
    """Perturbed constraints on an SIS: barycentre of the back-traced images,
    its two analytic images, nearest-image matching and Eq. 6 -- all written
    here with the SIS closed forms, compared with the oracle's general path."""
    b = 2.5
    m = I.halo_row(SIS, 0, 0, 0, 0, 0, 0, b)[None]
    rng = np.random.default_rng(12)
    s = np.array([0.6, -0.3])
    pts = [p + rng.normal(0, 0.05, 2) for p in _sis_images(b, s)]
    sig = np.array([0.1, 0.2])
    cons = I.constraints_dict([0, 2], [p[0] for p in pts], [p[1] for p in pts], sig, [0.9])
    beta = [p - 0.9 * b * p / np.linalg.norm(p) for p in pts]
    bary = 0.5 * (beta[0] + beta[1])
    pred = _sis_images(0.9 * b, bary)
    exp = sum(min(np.sum((p - q) ** 2) for q in pred) / s2 ** 2 for p, s2 in zip(pts, sig))
    g = I.grid(101, field=(-6, 6, -6, 6))
    chi2, nf = oracle.chi2_image(m, cons, g)
    assert nf[0] == 2
    assert math.isclose(chi2, exp, rel_tol=1e-9)
    # plain source-plane form
    exp_src = sum(np.sum((bary - bt) ** 2) / s2 ** 2 for bt, s2 in zip(beta, sig))
    assert math.isclose(oracle.chi2_source(m, cons, 2), exp_src, rel_tol=1e-12)


def test_chi2_source_weighted_forms_sis_closed_form():
    """The two weighted source-plane forms on an SIS, written here from its
    closed forms.  For an SIS of strength b (times the distance ratio), the
    inverse magnification matrix I - H has eigenvalue 1 along the radius and
    1 - b/|theta| across it, so det = 1 - b/|theta| and |mu| = |theta| /
    ||theta| - b|.  Variant 1 weights |bary - beta|^2 by |mu|; variant 0 maps
    the residual back to the image plane with A = (I - H)^-1, which leaves its
    radial part and divides its tangential part by 1 - b/|theta|.  The
    constraints sit on both sides of the Einstein ring, so one image has a
    negative det (the weight is |mu|, not mu)."""
    b, r = 2.5, 0.8
    m = I.halo_row(SIS, 0.4, -0.3, 0, 0, 0, 0, b)[None]
    c0 = np.array([0.4, -0.3])
    rng = np.random.default_rng(31)
    xs, ys, sig, off = [], [], [], [0]
    for s in (np.array([0.5, 0.3]), np.array([-0.2, 0.9]), np.array([0.7, -0.6])):
        for p in _sis_images(r * b, s):
            q = c0 + p + rng.normal(0, 0.08, 2)
            xs.append(q[0])
            ys.append(q[1])
            sig.append(rng.uniform(0.05, 0.2))
        off.append(len(xs))
    cons = I.constraints_dict(off, xs, ys, np.array(sig), np.full(3, r))
    be = r * b
    exp1 = exp0 = 0.0
    dets = []
    for i in range(3):
        pts = [np.array([xs[j], ys[j]]) - c0 for j in range(off[i], off[i + 1])]
        beta = [p - be * p / np.linalg.norm(p) for p in pts]
        bary = sum(beta) / len(beta)
        for k, (p, bt) in enumerate(zip(pts, beta)):
            rr = np.linalg.norm(p)
            det = 1.0 - be / rr
            dets.append(det)
            d = bary - bt
            s2 = sig[off[i] + k] ** 2
            exp1 += np.sum(d * d) * rr / abs(rr - be) / s2
            er = p / rr
            et = np.array([-er[1], er[0]])
            exp0 += ((d @ er) ** 2 + (d @ et / det) ** 2) / s2
    assert min(dets) < 0 < max(dets)
    assert math.isclose(oracle.chi2_source(m, cons, 1), exp1, rel_tol=1e-12)
    assert math.isclose(oracle.chi2_source(m, cons, 0), exp0, rel_tol=1e-12)


def test_source_plane_mapped_chi2_is_first_order_image_chi2():
    """For small noise, |A (bary - beta)| approximates the image-plane
    displacement, so the mapped source-plane chi2 (variant 0) tends to the
    image-plane chi2 (ratio -> 1 as the noise shrinks)."""
    m = np.vstack([I.halo_row(DPIE, 0.0, 0.0, 0.3, 0.25, 1.0, 200.0, 8.0),
                   I.halo_row(DPIE, 3.0, -2.0, 1.0, 0.3, 0.2, 10.0, 1.0)])
    g = I.grid(121, field=(-15, 15, -15, 15))
    bs = np.array([0.3, -0.4])
    img, nf = oracle.find_images(m, g, 1.0, bs)
    assert nf >= 3
    rng = np.random.default_rng(13)
    ratios = []
    for noise in (1e-3, 1e-4):
        pts = img + rng.normal(0, noise, img.shape)
        cons = I.constraints_dict([0, len(pts)], pts[:, 0], pts[:, 1], np.full(len(pts), noise), [1.0])
        c_img, _ = oracle.chi2_image(m, cons, g)
        c_src = oracle.chi2_source(m, cons, 0)
        ratios.append(c_src / c_img)
    assert abs(ratios[1] - 1) < 0.05
    assert abs(ratios[1] - 1) < abs(ratios[0] - 1) + 1e-3


def test_parameter_set_application():
    """A parameter set equal to the model's own varying parameters reproduces
    the model; a batch evaluates each set independently."""
    m = I.random_model(6, seed=14)
    cons = I.random_constraints(4, seed=15, field=30)
    var = (1, 4)
    base = I.var_params_of(m, var)
    assert np.array_equal(oracle.apply_params(m, var, base), m)
    P = I.perturbed_params(m, var, 5, seed=16)
    batch = oracle.chi2_source_batch(m, cons, var, P, 0)
    one = [oracle.chi2_source(oracle.apply_params(m, var, p), cons, 0) for p in P]
    assert np.allclose(batch, one, rtol=0, atol=0)
