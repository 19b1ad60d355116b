"""Image-plane chi2 parity against the FP64 oracle (Sec. 2.2 Eq. 6 with the
brute-force image search of Sec. 2.3 Fig. 4 and Sec. 4.2)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_06352_gb300 import inputs as I
from tests import tolerances as T
from tests.golden import make_constraints

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu_chi2_image(lens, m, cons, var, grid, params, ctx=None):
    P = len(params)
    own = ctx is None
    ctx = ctx or lens.Context(0)
    try:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        p = torch.tensor(params, dtype=torch.float64, device=DEV)
        out = torch.full((P,), -1.0, dtype=torch.float64, device=DEV)
        nf = torch.full((P, len(cons["img_off"]) - 1), -7, dtype=torch.int32, device=DEV)
        ctx.chi2_image(cs, grid, p, P, out, nf)
        ctx.wait()
        return out.cpu().numpy(), nf.cpu().numpy()
    finally:
        if own:
            ctx.close()


def test_chi2_image_cfg2_model_parity(lens):
    """1000-potential model, 100 sources / 372 images at 5 distance ratios,
    the two cluster halos varying; 256^2 search grid; 5 parameter sets (the
    first is the model itself)."""
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    g = I.grid(256)
    params = I.perturbed_params(m, var, 5, seed=41)
    params[0] = I.var_params_of(m, var)
    ref, nf_ref = oracle.chi2_image_batch(m, cons, g, var, params)
    got, nf = gpu_chi2_image(lens, m, cons, var, g, params)
    assert np.array_equal(nf, nf_ref), (nf - nf_ref)[np.nonzero(nf - nf_ref)]
    assert np.all(np.abs(got - ref) <= T.CHI2_REL * np.abs(ref)), np.abs(got - ref) / ref


def test_chi2_image_noise_free_is_zero(lens):
    """Constraints placed exactly on the predicted images of a source give chi2 ~ 0."""
    m = np.vstack([I.halo_row(I.DPIE, 0.3, -0.2, 0.5, 0.3, 1.5, 300.0, 12.0),
                   I.halo_row(I.DPIE, -2.0, 1.0, 1.1, 0.2, 0.8, 150.0, 6.0),
                   I.member_model(30, seed=42, field=30)])
    g = I.grid(201, field=(-40, 40, -40, 40))
    xs, ys, off, rs = [], [], [0], []
    for k, (bs, r) in enumerate([((0.4, 0.3), 0.7), ((-0.6, 0.2), 0.9), ((0.1, -0.8), 0.5)]):
        img, nfound = oracle.find_images(m, g, r, bs)
        assert nfound >= 2
        xs += list(img[:, 0])
        ys += list(img[:, 1])
        off.append(len(xs))
        rs.append(r)
    cons = I.constraints_dict(off, xs, ys, np.full(len(xs), 0.05), rs)
    params = I.var_params_of(m, (0, 1))[None]
    got, nf = gpu_chi2_image(lens, m, cons, (0, 1), g, params)
    assert got[0] < 1e-12, got
    assert list(nf[0]) == [off[i + 1] - off[i] for i in range(3)]


def test_chi2_image_invalid_set_is_nan(lens):
    m = np.vstack([I.halo_row(I.DPIE, 0.0, 0.0, 0.2, 0.3, 1.0, 200.0, 10.0),
                   I.halo_row(I.DPIE, 3.0, 1.0, 1.0, 0.2, 0.5, 100.0, 4.0),
                   I.member_model(10, seed=43, field=20)])
    cons = I.random_constraints(4, seed=44, field=10)
    g = I.grid(64, field=(-30, 30, -30, 30))
    params = I.perturbed_params(m, (0, 1), 3, seed=45)
    params[1, 2] = 1.5  # eps >= 1
    got, nf = gpu_chi2_image(lens, m, cons, (0, 1), g, params)
    assert np.isnan(got[1]) and np.all(nf[1] == 0)
    ref, nf_ref = oracle.chi2_image_batch(m, cons, g, (0, 1), params[[0, 2]])
    assert np.array_equal(nf[[0, 2]], nf_ref)
    ok = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got[[0, 2]]), ok)
    assert np.all(np.abs(got[[0, 2]][ok] - ref[ok]) <= T.CHI2_REL * np.abs(ref[ok]))
