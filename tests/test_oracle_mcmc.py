"""Pins of the oracle's Metropolis sampler (the Bayesian fit of Sec. 2.2):
its counter-based generator against numpy's own Philox4x64-10, the
uniforms' and Box-Muller normals' distributions, the stationary law of the
random walk, the acceptance frequency against the likelihood ratio, and the
acceptance rule in its limiting cases."""
import numpy as np
import pytest

import oracle
from paper_2004_06352_gb300 import inputs as I


def test_philox_matches_numpy_philox():
    """numpy.random.Philox is Philox4x64-10; its k-th block of 4 words is the
    generator applied to counter + k + 1 (it steps the counter first)."""
    for key, ctr in (([5, 7], [0, 0, 0, 0]), ([2**64 - 1, 0], [2**64 - 1, 3, 0, 9]),
                     ([0x243F6A8885A308D3, 0x13198A2E03707344], [11, 2**63, 5, 0])):
        raw = np.random.Philox(key=np.array(key, dtype=np.uint64),
                               counter=np.array(ctr, dtype=np.uint64)).random_raw(12)
        c = list(ctr)
        for k in range(3):
            # counter + 1 with carry across the four 64-bit words
            for i in range(4):
                c[i] = (c[i] + 1) % 2**64
                if c[i] != 0:
                    break
            assert list(oracle.philox4x64_10(c, key)) == [int(x) for x in raw[4 * k: 4 * k + 4]]


def test_uniforms_and_normals_distribution():
    from scipy import stats
    u = oracle.mcmc_uniforms(seed=12345, step=7, W=4000)
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u.ravel(), "uniform").pvalue > 1e-3
    # the sampler's proposal steps (params 0, sigma 1) are standard normal,
    # each coordinate and every pair uncorrelated
    z = oracle.gaussian_proposals(np.zeros((len(u), 14)), np.ones(14), u[:, :14])
    assert stats.kstest(z.ravel(), "norm").pvalue > 1e-3
    assert abs(z.var() - 1.0) < 0.02 and abs(z.mean()) < 0.02
    assert np.all(np.abs(np.corrcoef(z.T) - np.eye(14)) < 0.06)
    assert abs(np.corrcoef(u[:-1, 3], u[1:, 3])[0, 1]) < 0.05  # neighbouring chains
    assert not np.array_equal(oracle.mcmc_uniforms(12345, 8, 4), u[:4])   # steps differ
    assert np.array_equal(oracle.mcmc_uniforms(12345, 7, 4), u[:4])       # replayable


def make_small_fit():
    m = I.random_model(6, seed=71)
    m[0, 7], m[1, 7] = 8.0, 6.0
    cons = I.random_constraints(4, seed=72, field=30)
    var = (0, 1)
    params = I.perturbed_params(m, var, 6, seed=73)
    chi2 = oracle.chi2_source_batch(m, cons, var, params, 0)
    sigma = np.tile([0.3, 0.3, 0.01, 0.02, 0.02, 1.0, 0.05], 2)
    return m, cons, var, params, chi2, sigma


@pytest.fixture(scope="module")
def small_fit():
    return make_small_fit()


# pytest fixtures of this module, as plain builders (the mutation tests call
# the pins directly)
FIXTURES = {"small_fit": make_small_fit}


def test_stationary_distribution_is_the_tempered_likelihood():
    """The random walk built from the oracle's proposals and acceptance rule
    samples the posterior of the likelihood exp(-chi2/2) (Sec. 2.2) at
    temperature T: for chi2(x) = sum_k (x_k/s_k)^2 the stationary law is
    N(0, T s_k^2) in every coordinate.  Detailed balance fixes this law
    whatever the step size; 20000 independent chains after a burn-in of 400
    steps give each variance to about 1 %.  Dropping the 1/2 of the
    likelihood would halve the variances."""
    rng = np.random.default_rng(2024)
    W, T = 20000, 1.7
    s = np.array([0.5, 2.0, 1.0, 0.25])
    chi2_of = lambda x: np.sum((x / s) ** 2, axis=1)
    x = np.zeros((W, len(s)))
    c = chi2_of(x)
    rates = []
    for _ in range(400):
        prop = oracle.gaussian_proposals(x, 1.6 * s, rng.random((W, len(s))))
        cp = chi2_of(prop)
        take = oracle.metropolis_accept(c, cp, rng.random(W), T)
        rates.append(take.mean())
        x = np.where(take[:, None], prop, x)
        c = np.where(take, cp, c)
    assert 0.2 < np.mean(rates[-50:]) < 0.8
    var = x.var(axis=0) / (T * s * s)
    assert np.all(np.abs(var - 1.0) < 0.05), var
    assert np.all(np.abs(x.mean(axis=0)) < 5 * np.sqrt(T / W) * s)


def test_acceptance_frequency_matches_the_likelihood_ratio():
    """On the lens model's own chi2: bin one step's proposals by the
    difference of chi2 it reports; the fraction accepted in each bin equals
    the mean Metropolis probability min(1, exp(-d chi2 / (2T))) of its
    members, within binomial error (Sec. 2.2: likelihood exp(-chi2/2)).  The
    temperature puts the probabilities across the middle of their range."""
    m, cons, var, params, chi2, sigma = make_small_fit()
    W = 2400
    base = np.repeat(params[:1], W, axis=0)
    c0 = np.repeat(chi2[:1], W)
    # a first step fixes the scale of d chi2; T then puts exp(-d/2T) near
    # e^-1 at the median |d| (the same proposals: same seed and step)
    _, _, _, _, cp = oracle.mcmc_step(m, cons, var, base, c0, 0.4 * sigma, 1.0, seed=9, step=1)
    d = cp - c0
    T = float(np.median(np.abs(d[np.isfinite(d)]))) / 2.0
    _, _, take, prop, cp = oracle.mcmc_step(m, cons, var, base, c0, 0.4 * sigma, T, seed=9, step=1)
    d = cp - c0
    ok = np.isfinite(d)
    p = np.minimum(1.0, np.exp(-d[ok] / (2.0 * T)))
    t = take[ok].astype(float)
    edges = np.quantile(p, np.linspace(0, 1, 9))
    checked = 0
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (p >= lo) & (p <= hi)
        if sel.sum() < 50:
            continue
        mean_p = p[sel].mean()
        err = np.sqrt(max(mean_p * (1 - mean_p), 1e-3) / sel.sum())
        assert abs(t[sel].mean() - mean_p) < 4.5 * err + 1e-9, (lo, hi, t[sel].mean(), mean_p)
        checked += 1
    assert checked >= 4
    # the accepted fraction overall sits mid-range, so the test has power
    assert 0.15 < t.mean() < 0.85


def test_zero_step_always_moves_in_place(small_fit):
    m, cons, var, params, chi2, sigma = small_fit
    p2, c2, take, prop, cp = oracle.mcmc_step(m, cons, var, params, chi2, 0 * sigma, 1.0, seed=1, step=0)
    assert take.all() and np.array_equal(p2, params) and np.array_equal(c2, chi2)


def test_temperature_limits(small_fit):
    m, cons, var, params, chi2, sigma = small_fit
    _, _, take, _, cp = oracle.mcmc_step(m, cons, var, params, chi2, sigma, 1e-300, seed=2, step=3)
    assert np.array_equal(take, cp < chi2)            # T -> 0: only improvements
    _, _, take, _, cp = oracle.mcmc_step(m, cons, var, params, chi2, sigma, 1e300, seed=2, step=3)
    assert np.array_equal(take, np.isfinite(cp))      # T -> inf: every valid proposal


def test_outside_domain_refused_and_nan_start_moves(small_fit):
    m, cons, var, params, chi2, sigma = small_fit
    params = params.copy()
    chi2 = chi2.copy()
    params[0, 2] = 0.995           # eps next to 1
    big = sigma.copy()
    big[2] = 0.5                   # most eps proposals leave [0, 1)
    chi2[1] = np.nan               # chain 1 takes any valid proposal
    p2, c2, take, prop, cp = oracle.mcmc_step(m, cons, var, params, chi2, big, 1.0, seed=4, step=0)
    bad = ~np.array([oracle.params_in_domain(m, var, p) for p in prop])
    assert bad.any() and np.all(np.isnan(cp[bad])) and not take[bad].any()
    assert take[1] == np.isfinite(cp[1])


# ------------------------------------------------- members' scaling relations

def test_scaled_chi2_reduces_to_plain_at_unit_factors(small_fit):
    m, cons, var, params, chi2, sigma = small_fit
    p16 = np.hstack([params, np.ones((len(params), 2))])
    got = oracle.chi2_source_scaled_batch(m, cons, var, p16, 0)
    assert np.allclose(got, chi2, rtol=1e-13, atol=0)


def test_scaled_factors_act_on_the_static_potentials_only():
    """f_b multiplies the static potentials' deflection (the model is linear
    in b0); f_t moves a circular member's cut radius and not its core (the
    circular dPIE's closed-form deflection)."""
    m = np.stack([I.halo_row(I.DPIE, 0.0, 0.0, 0.3, 0.2, 4.0, 500.0, 20.0),
                  I.halo_row(I.DPIE, 5.0, -3.0, 1.0, 0.1, 3.0, 300.0, 15.0),
                  I.halo_row(I.DPIE, 2.0, 7.0, 0.0, 0.0, 0.2, 10.0, 1.5),
                  I.halo_row(I.SIS, -6.0, 1.0, 0, 0, 0, 0, 0.8)])
    var = (0, 1)
    base = np.hstack([m[0, [1, 2, 4, 3, 5, 6, 7]], m[1, [1, 2, 4, 3, 5, 6, 7]]])
    X, Y = np.array([30.0, -12.0, 4.0]), np.array([-8.0, 22.0, 40.0])
    stat = lambda t: oracle.model_eval(t[2:], X, Y)
    one = stat(oracle.apply_params_scaled(m, var, np.hstack([base, 1.0, 1.0])))
    two = stat(oracle.apply_params_scaled(m, var, np.hstack([base, 2.0, 1.0])))
    assert np.allclose(two, 2 * one, rtol=1e-13, atol=0)
    # varying halos untouched
    t = oracle.apply_params_scaled(m, var, np.hstack([base, 3.0, 0.5]))
    assert np.array_equal(t[:2], oracle.apply_params(m, var, base)[:2])
    # circular member alone: alpha_r = b0 [(sqrt(rc^2 + r^2) - rc) - (sqrt(rt^2 + r^2) - rt)] / r
    for ft in (0.6, 1.7):
        t = oracle.apply_params_scaled(m, var, np.hstack([base, 1.0, ft]))
        for r in (0.1, 3.0, 25.0):
            a = oracle.model_eval(t[2:3], 2.0 + r, 7.0)[0]
            rc, rt = 0.2, ft * 10.0
            exact = 1.5 * ((np.hypot(rc, r) - rc) - (np.hypot(rt, r) - rt)) / r
            assert abs(a[0] - exact) <= 1e-12 * abs(exact) and abs(a[1]) < 1e-15


def test_scaled_outside_domain_is_nan(small_fit):
    m, cons, var, params, chi2, sigma = small_fit
    p16 = np.hstack([params[:3], np.ones((3, 2))])
    p16[0, 14] = -1.0           # f_b <= 0
    p16[1, 15] = 1e-4           # members' r_cut below their r_core
    got = oracle.chi2_source_scaled_batch(m, cons, var, p16, 0)
    assert np.isnan(got[0]) and np.isnan(got[1]) and np.isfinite(got[2])
