"""lens_chi2_image_noalloc against lens_chi2_image, through the C ABI.

The no-allocation variant serves callers that reserve their device memory
once and may not call cudaMalloc/cudaFree while they run (a long sampler or
request loop: those calls can stall every stream on the device and can fail
mid-run).  Its working memory is one fixed device array inside the library.
Two calls in a row must both reproduce the allocating entry point, so stale
contents left in that shared array by the first call cannot leak into the
second.  This file sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2004_06352_gb300 import inputs as I
from tests import tolerances as T
from tests.golden import make_constraints

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("n", [256, 1400])
def test_noalloc_matches_allocating_entry_point_twice(lens, n):
    """256^2: the 12 sets in one batch.  1400^2: the grid's static
    deflection takes 15.7 MB of the 16 MiB array, so the batch halves from 12
    to a single set (~1.0 MB of candidate buffers and refinement lists) and
    the call runs twelve batches through the space left."""
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    g = I.grid(n)
    P = 12
    params = torch.tensor(I.perturbed_params(m, var, P, seed=61), dtype=torch.float64, device=DEV)
    nsrc = len(cons["img_off"]) - 1
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        ref = torch.empty(P, dtype=torch.float64, device=DEV)
        nf_ref = torch.empty((P, nsrc), dtype=torch.int32, device=DEV)
        ctx.chi2_image(cs, g, params, P, ref, nf_ref)
        ctx.wait()
        ref, nf_ref = ref.cpu().numpy(), nf_ref.cpu().numpy()
        assert np.all(np.isfinite(ref))
        for call in range(2):
            got = torch.full((P,), -1.0, dtype=torch.float64, device=DEV)
            nf = torch.full((P, nsrc), -7, dtype=torch.int32, device=DEV)
            ctx.chi2_image_noalloc(cs, g, params, P, got, nf)
            ctx.wait()
            got, nf = got.cpu().numpy(), nf.cpu().numpy()
            assert np.array_equal(nf, nf_ref), call
            assert np.all(np.abs(got - ref) <= T.CHI2_REL * np.abs(ref)), (call, np.abs(got - ref) / ref)


def test_noalloc_rejects_grid_beyond_fixed_scratch(lens):
    m = I.cfg2_model()
    cons = make_constraints.load()
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, (0, 1))
        params = torch.tensor(I.perturbed_params(m, (0, 1), 1, seed=62), dtype=torch.float64, device=DEV)
        out = torch.empty(1, dtype=torch.float64, device=DEV)
        with pytest.raises(lens.LensError) as e:
            ctx.chi2_image_noalloc(cs, I.grid(2048), params, 1, out)   # 32 MiB of node deflections
        assert e.value.code == lens.LENS_EINVAL
        assert "LENS_NOALLOC_SCRATCH_BYTES" in str(e.value)


def test_noalloc_single_kernel_refinement_matches_oracle(lens):
    """1420^2: the grid's static deflection takes 16.13 MB of the 16 MiB
    array, which leaves room for one set's candidate buffers (~0.22 MB) but
    not for the point-list refinement's (~1.0 MB): the call refines with the
    single-kernel Newton.  Its image counts and chi2 must agree with the
    oracle's (Sec. 2.2 Eq. 6, Sec. 2.3) where the image sets agree, for at
    least one of the two sets, and image counts may differ only rarely."""
    import oracle
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    g = I.grid(1420)
    params = I.perturbed_params(m, var, 2, seed=63)
    params[0] = I.var_params_of(m, var)
    ref, nf_ref = oracle.chi2_image_batch(m, cons, g, var, params)
    nsrc = len(cons["img_off"]) - 1
    with lens.Context(0) as ctx:
        cs = ctx.cset_create(ctx.model_upload(m), cons, var)
        got = torch.full((2,), -1.0, dtype=torch.float64, device=DEV)
        nf = torch.full((2, nsrc), -7, dtype=torch.int32, device=DEV)
        ctx.chi2_image_noalloc(cs, g, torch.tensor(params, dtype=torch.float64, device=DEV), 2, got, nf)
        ctx.wait()
        got, nf = got.cpu().numpy(), nf.cpu().numpy()
    assert np.abs(nf - nf_ref).sum() <= 0.01 * nf_ref.sum(), (nf - nf_ref)
    same = [p for p in range(2) if np.array_equal(nf[p], nf_ref[p])]
    assert same, "no parameter set had the oracle's image counts"
    for p in same:
        assert abs(got[p] - ref[p]) <= T.CHI2_REL * abs(ref[p]), (p, got[p], ref[p])
