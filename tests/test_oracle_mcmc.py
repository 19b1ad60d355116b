"""Pins of the oracle's Metropolis sampler (the Bayesian fit of Sec. 2.2):
its counter-based generator against numpy's own Philox4x64-10, the
uniforms' and Box-Muller normals' distributions, and the acceptance rule in
its limiting cases."""
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
    # the sampler's Box-Muller pairs are standard normal and uncorrelated
    rad = np.sqrt(-2.0 * np.log(u[:, 0:14:2]))
    z = np.concatenate([(rad * np.cos(2 * np.pi * u[:, 1:14:2])).ravel(),
                        (rad * np.sin(2 * np.pi * u[:, 1:14:2])).ravel()])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(u[:-1, 3], u[1:, 3])[0, 1]) < 0.05  # neighbouring chains
    assert not np.array_equal(oracle.mcmc_uniforms(12345, 8, 4), u[:4])   # steps differ
    assert np.array_equal(oracle.mcmc_uniforms(12345, 7, 4), u[:4])       # replayable


@pytest.fixture(scope="module")
def small_fit():
    m = I.random_model(6, seed=71)
    m[0, 7], m[1, 7] = 8.0, 6.0
    cons = I.random_constraints(4, seed=72, field=30)
    var = (0, 1)
    params = I.perturbed_params(m, var, 6, seed=73)
    chi2 = oracle.chi2_source_batch(m, cons, var, params, 0)
    sigma = np.tile([0.3, 0.3, 0.01, 0.02, 0.02, 1.0, 0.05], 2)
    return m, cons, var, params, chi2, sigma


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
