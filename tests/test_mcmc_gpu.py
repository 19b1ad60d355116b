"""Metropolis sampling on the device (the Bayesian fit of Sec. 2.2 over the
batched source-plane chi2) against the oracle's sampler, which draws the same
Philox4x64-10 stream: proposals, chi2 and every move decision agree step by
step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_06352_gb300 import inputs as I
from tests import tolerances as T

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_mcmc_steps_match_oracle(lens):
    from tests.golden import make_constraints
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    W = 40
    params = I.perturbed_params(m, var, W, seed=81)
    params[3, 2] = 0.995                    # eps next to 1: proposals leave the domain
    chi2 = oracle.chi2_source_batch(m, cons, var, params, 0)
    chi2[5] = np.nan                        # takes any valid proposal
    sigma = np.tile([0.2, 0.2, 0.005, 0.01, 0.05, 5.0, 0.1], 2)
    sig_gpu = sigma.copy()
    T_ = 2000.0                             # chi2 ~ 1e5: moves of a few 1e3 are taken at times
    seed = 0xC0FFEE
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        p = torch.tensor(params, device=DEV)
        c = torch.tensor(chi2, device=DEV)
        sg = torch.tensor(sig_gpu, device=DEV)
        scratch = torch.empty(16 * W, dtype=torch.float64, device=DEV)
        acc = torch.empty(W, dtype=torch.int32, device=DEV)
        po, co = params.copy(), chi2.copy()
        n_acc = 0
        for step in range(4):
            ctx.mcmc_step(cs, p, c, W, sg, T_, seed, step, scratch, acc)
            ctx.wait()
            po2, co2, take, prop, cp = oracle.mcmc_step(m, cons, var, po, co, sigma, T_, seed, step)
            got_take = acc.cpu().numpy().astype(bool)
            u = oracle.mcmc_uniforms(seed, step, W)[:, 16]
            margin = np.log(u) + (cp - co) / (2 * T_)
            sure = ~np.isfinite(margin) | (np.abs(margin) > 1e-6)   # decisions far from the threshold
            assert np.array_equal(got_take[sure], take[sure]), step
            # keep the oracle in step with the device on the (unseen so far) borderline cases
            po2 = np.where(got_take[:, None], prop, po)
            co2 = np.where(got_take, cp, co)
            gp, gc = p.cpu().numpy(), c.cpu().numpy()
            assert np.allclose(gp, po2, rtol=1e-13, atol=1e-13), step
            fin = np.isfinite(co2)
            assert np.array_equal(np.isfinite(gc), fin)
            assert np.all(np.abs(gc[fin] - co2[fin]) <= T.CHI2_REL * np.abs(co2[fin])), step
            po, co = po2, co2
            n_acc += int(got_take.sum())
        assert 0 < n_acc < 4 * W                                    # some moves taken, some refused
        assert np.isfinite(co[5])                                   # the NaN chain moved


def test_mcmc_step_replays_and_zero_step(lens):
    from tests.golden import make_constraints
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    W = 300
    params = I.perturbed_params(m, var, W, seed=82)
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        p0 = torch.tensor(params, device=DEV)
        c0 = torch.empty(W, dtype=torch.float64, device=DEV)
        ctx.chi2_source(cs, p0, W, 0, c0)
        sg = torch.tensor(np.tile([0.2, 0.2, 0.005, 0.01, 0.05, 5.0, 0.1], 2), device=DEV)
        scratch = torch.empty(16 * W, dtype=torch.float64, device=DEV)
        runs = []
        for _ in range(2):
            p, c = p0.clone(), c0.clone()
            ctx.mcmc_step(cs, p, c, W, sg, 500.0, 99, 17, scratch)
            runs.append((p, c))
        ctx.wait()
        assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
        p, c = p0.clone(), c0.clone()
        acc = torch.empty(W, dtype=torch.int32, device=DEV)
        ctx.mcmc_step(cs, p, c, W, torch.zeros_like(sg), 1.0, 99, 18, scratch, acc)
        ctx.wait()
        assert torch.equal(p, p0) and torch.equal(c, c0) and bool(acc.all())
        with pytest.raises(lens.LensError) as e:
            ctx.mcmc_step(cs, p, c, W, sg, 0.0, 1, 0, scratch)
        assert e.value.code == lens.LENS_EINVAL


def test_mcmc_steps_with_member_scaling_match_oracle(lens):
    """16-parameter chains: the cluster halos and the members' b0 and r_cut
    factors, chi2 as lens_chi2_source_scaled."""
    from tests.golden import make_constraints
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    W = 24
    rng = np.random.default_rng(84)
    params = np.hstack([I.perturbed_params(m, var, W, seed=85), rng.uniform(0.9, 1.1, (W, 2))])
    chi2 = oracle.chi2_source_scaled_batch(m, cons, var, params, 0)
    sigma = np.concatenate([np.tile([0.2, 0.2, 0.005, 0.01, 0.05, 5.0, 0.1], 2), [0.02, 0.05]])
    T_, seed = 2000.0, 77
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        p = torch.tensor(params, device=DEV)
        c = torch.tensor(chi2, device=DEV)
        sg = torch.tensor(sigma, device=DEV)
        scratch = torch.empty(18 * W, dtype=torch.float64, device=DEV)
        acc = torch.empty(W, dtype=torch.int32, device=DEV)
        po, co = params.copy(), chi2.copy()
        moved = 0
        for step in range(3):
            ctx.mcmc_step(cs, p, c, W, sg, T_, seed, step, scratch, acc)
            ctx.wait()
            _, _, take, prop, cp = oracle.mcmc_step(m, cons, var, po, co, sigma, T_, seed, step)
            got_take = acc.cpu().numpy().astype(bool)
            u = oracle.mcmc_uniforms(seed, step, W)[:, 16]
            margin = np.log(u) + (cp - co) / (2 * T_)
            sure = ~np.isfinite(margin) | (np.abs(margin) > 1e-6)
            assert np.array_equal(got_take[sure], take[sure]), step
            po = np.where(got_take[:, None], prop, po)
            co = np.where(got_take, cp, co)
            gp, gc = p.cpu().numpy(), c.cpu().numpy()
            assert np.allclose(gp, po, rtol=1e-13, atol=1e-13), step
            assert np.all(np.abs(gc - co) <= T.CHI2_REL * np.abs(co)), step
            moved += int(got_take.sum())
        assert 0 < moved < 3 * W


def test_mcmc_steps_with_scaling_cache_match_oracle(lens):
    """16-parameter chains whose chi2 comes from the scaling cache (the
    members' sums interpolated in the r_cut factor) against the oracle's
    sampler with the sums recomputed exactly; a proposal outside the cached
    factor interval is refused."""
    from tests.golden import make_constraints
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    W = 24
    rng = np.random.default_rng(86)
    params = np.hstack([I.perturbed_params(m, var, W, seed=87), rng.uniform(0.9, 1.1, (W, 2))])
    params[4, 15] = 1.499                  # next to the cache's upper end: f_t proposals leave it
    chi2 = oracle.chi2_source_scaled_batch(m, cons, var, params, 0)
    sigma = np.concatenate([np.tile([0.2, 0.2, 0.005, 0.01, 0.05, 5.0, 0.1], 2), [0.02, 0.05]])
    T_, seed = 2000.0, 91
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        ctx.cset_scaling_cache(cs, 0.6, 1.5, 32)
        p = torch.tensor(params, device=DEV)
        c = torch.tensor(chi2, device=DEV)
        sg = torch.tensor(sigma, device=DEV)
        scratch = torch.empty(18 * W, dtype=torch.float64, device=DEV)
        acc = torch.empty(W, dtype=torch.int32, device=DEV)
        po, co = params.copy(), chi2.copy()
        for step in range(2):
            ctx.mcmc_step(cs, p, c, W, sg, T_, seed, step, scratch, acc)
            ctx.wait()
            _, _, take, prop, cp = oracle.mcmc_step(m, cons, var, po, co, sigma, T_, seed, step)
            cp = np.where((prop[:, 15] >= 0.6) & (prop[:, 15] <= 1.5), cp, np.nan)  # the cache's prior
            take = np.isfinite(cp) & (~np.isfinite(co) | (np.log(oracle.mcmc_uniforms(seed, step, W)[:, 16])
                                                          < -(cp - co) / (2 * T_)))
            got_take = acc.cpu().numpy().astype(bool)
            u = oracle.mcmc_uniforms(seed, step, W)[:, 16]
            margin = np.log(u) + (cp - co) / (2 * T_)
            sure = ~np.isfinite(margin) | (np.abs(margin) > 1e-5)
            assert np.array_equal(got_take[sure], take[sure]), step
            po = np.where(got_take[:, None], prop, po)
            co = np.where(got_take, cp, co)
            assert np.allclose(p.cpu().numpy(), po, rtol=1e-13, atol=1e-13), step
            assert np.all(np.abs(c.cpu().numpy() - co) <= T.CHI2_REL * np.abs(co)), step
        ctx.cset_scaling_cache(cs, 0.0, 0.0, 0)


def test_mcmc_step_graph_replays_advance_the_device_counter(lens):
    """lens_mcmc_step_dev captured once in a CUDA graph: each replay reads
    the step counter from device memory and advances it, so replay k draws
    step s0 + k -- compared with the oracle's sampler at those steps."""
    from tests.golden import make_constraints
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    W = 32
    params = I.perturbed_params(m, var, W, seed=88)
    chi2 = oracle.chi2_source_batch(m, cons, var, params, 0)
    sigma = np.tile([0.2, 0.2, 0.005, 0.01, 0.05, 5.0, 0.1], 2)
    T_, seed, s0 = 2000.0, 4242, 11
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        p = torch.tensor(params, device=DEV)
        c = torch.tensor(chi2, device=DEV)
        sg = torch.tensor(sigma, device=DEV)
        scratch = torch.empty(16 * W, dtype=torch.float64, device=DEV)
        acc = torch.empty(W, dtype=torch.int32, device=DEV)
        ctr = torch.tensor([s0], dtype=torch.int64, device=DEV)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            ctx.mcmc_step_dev(cs, p, c, W, sg, T_, seed, ctr, scratch, acc, stream=side)
        side.synchronize()
        # capturing ran nothing: the state is still the initial one
        assert int(ctr.item()) == s0 and torch.equal(p.cpu(), torch.tensor(params))
        po, co = params.copy(), chi2.copy()
        moved = 0
        for k in range(2):
            graph.replay()
            torch.cuda.synchronize()
            _, _, take, prop, cp = oracle.mcmc_step(m, cons, var, po, co, sigma, T_, seed, s0 + k)
            got_take = acc.cpu().numpy().astype(bool)
            u = oracle.mcmc_uniforms(seed, s0 + k, W)[:, 16]
            margin = np.log(u) + (cp - co) / (2 * T_)
            sure = ~np.isfinite(margin) | (np.abs(margin) > 1e-6)
            assert np.array_equal(got_take[sure], take[sure]), k
            po = np.where(got_take[:, None], prop, po)
            co = np.where(got_take, cp, co)
            assert np.allclose(p.cpu().numpy(), po, rtol=1e-13, atol=1e-13), k
            assert np.all(np.abs(c.cpu().numpy() - co) <= T.CHI2_REL * np.abs(co)), k
            assert int(ctr.item()) == s0 + k + 1
            moved += int(got_take.sum())
        assert moved > 0
        with pytest.raises(lens.LensError) as e:
            ctx.mcmc_step_dev(cs, p, c, W, sg, T_, seed, None, scratch)
        assert e.value.code == lens.LENS_EINVAL
