"""Lensing potential and time-delay (Fermat) surface maps (Sec. 2.4's list of
map kinds; the potential of Sec. 2.1 Eq. 2) against the FP64 oracle, and the
potential's gradient against the deflection map by finite differences on the
GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_06352_gb300 import inputs as I
from tests import tolerances as T

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def pot_map(lens, m, g, dls, precision, beta=None):
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        out = torch.full((1 if beta is None else 2, g["ny"], g["nx"]), float("nan"), dtype=torch.float64,
                         device=DEV)
        ctx.potential_map(mid, g, dls, precision, out, beta=beta)
        ctx.wait()
        return out.cpu().numpy()


def grid_points(g):
    x = np.linspace(g["xmin"], g["xmax"], g["nx"])
    y = np.linspace(g["ymin"], g["ymax"], g["ny"])
    X, Y = np.meshgrid(x, y)
    return X, Y


def test_potential_fp64_and_mixed_all_kinds_ragged(lens):
    """Every kind (dPIE, SIS, point mass, a near-circular dPIE on the series
    path), a ragged 45 x 37 grid, D_ls/D_s = 0.7, the Fermat surface about a
    source position."""
    m = I.random_model(23, seed=41, types=(I.DPIE, I.DPIE, I.SIS, I.POINT))
    m[1, 4] = 1e-4  # eps: u < 0.12, the series kind of the FP32 path
    m[0, 7] = 12.0  # one potential above the FP64 threshold of the mixed path
    g = I.grid(45, field=(-55, 61, -48, 50), ny=37)
    X, Y = grid_points(g)
    ref = oracle.potential(m, X.ravel(), Y.ravel(), 0.7).reshape(X.shape)
    beta = (3.25, -7.5)
    tau = 0.5 * ((X - beta[0]) ** 2 + (Y - beta[1]) ** 2) - ref
    got = pot_map(lens, m, g, 0.7, lens.LENS_FP64, beta)
    scale = np.abs(ref).max()
    assert np.all(np.abs(got[0] - ref) <= T.POT_FP64_REL * scale), np.abs(got[0] - ref).max() / scale
    assert np.all(np.abs(got[1] - tau) <= T.POT_FP64_REL * scale)
    mix = pot_map(lens, m, g, 0.7, lens.LENS_MIXED, beta)
    tol = T.pot_mixed_tol(ref)
    err = np.abs(mix[0] - ref)
    assert np.all(err <= tol), (err.max(), tol)
    # the second plane is the first one's Fermat surface, formed in FP64
    X2 = g["xmin"] + np.arange(g["nx"]) * ((g["xmax"] - g["xmin"]) / (g["nx"] - 1))
    Y2 = g["ymin"] + np.arange(g["ny"]) * ((g["ymax"] - g["ymin"]) / (g["ny"] - 1))
    XX, YY = np.meshgrid(X2 - beta[0], Y2 - beta[1])
    assert np.allclose(mix[1], 0.5 * (XX ** 2 + YY ** 2) - mix[0], rtol=0, atol=1e-9 * scale)
    assert np.all(np.abs(mix[1] - tau) <= tol)


def test_potential_full_size_cfg2_sampled(lens):
    """2048^2 x 1000 potentials (2 cluster-scale in FP64, 998 members in
    FP32); 8k sampled nodes against the oracle."""
    m, g = I.cfg2_model(), I.grid(2048)
    got = pot_map(lens, m, g, 1.0, lens.LENS_MIXED)[0]
    rng = np.random.default_rng(26)
    n = 8000
    ii, jj = rng.integers(0, 2048, n), rng.integers(0, 2048, n)
    ii[:4], jj[:4] = [0, 2047, 0, 2047], [0, 0, 2047, 2047]
    dx = 200.0 / 2047
    ref = oracle.potential(m, -100.0 + ii * dx, -100.0 + jj * dx, 1.0)
    err = np.abs(got[jj, ii] - ref)
    tol = T.pot_mixed_tol(ref)
    assert np.all(err <= tol), (err.max(), tol)


def test_potential_gradient_is_the_deflection(lens):
    """Central differences of the FP64 potential map on a fine grid equal the
    FP64 deflection map there (to the differences' h^2 error): the potential
    and the deflection are computed by independent code on the GPU."""
    m = np.stack([I.halo_row(I.DPIE, 0.5, -0.3, 0.4, 0.25, 3.0, 400.0, 25.0),
                  I.halo_row(I.DPIE, 6.0, 4.0, 1.9, 0.4, 1.5, 80.0, 4.0),
                  I.halo_row(I.SIS, -7.0, 5.0, 0, 0, 0, 0, 1.5),
                  I.halo_row(I.POINT, 8.0, -9.0, 0, 0, 0, 0, 1.2)])
    h = 2e-3
    g = I.grid(201, field=(1.0, 1.0 + 200 * h, 2.0, 2.0 + 200 * h))
    phi = pot_map(lens, m, g, 1.0, lens.LENS_FP64)[0]
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        al = torch.empty((2, 201, 201), dtype=torch.float64, device=DEV)
        ctx.grad_map(mid, g, 1.0, lens.LENS_FP64, al)
        ctx.wait()
        al = al.cpu().numpy()
    fx = (phi[1:-1, 2:] - phi[1:-1, :-2]) / (2 * h)
    fy = (phi[2:, 1:-1] - phi[:-2, 1:-1]) / (2 * h)
    scale = np.abs(al).max()
    assert np.abs(fx - al[0, 1:-1, 1:-1]).max() <= 1e-6 * scale
    assert np.abs(fy - al[1, 1:-1, 1:-1]).max() <= 1e-6 * scale


def test_potential_invalid_arguments(lens):
    m = I.random_model(3, seed=42)
    g = I.grid(8)
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        out = torch.empty((2, 8, 8), dtype=torch.float64, device=DEV)
        with pytest.raises(lens.LensError) as e:
            ctx.potential_map(mid, g, 1.0, lens.LENS_MIXED, out, beta=(float("nan"), 0.0))
        assert e.value.code == lens.LENS_EINVAL
        with pytest.raises(lens.LensError) as e:
            ctx.potential_map(mid, g, 1.0, 7, out)
        assert e.value.code == lens.LENS_EINVAL
        with pytest.raises(lens.LensError) as e:
            ctx.potential_map(mid + 99, g, 1.0, lens.LENS_FP64, out)
        assert e.value.code == lens.LENS_ENOTFOUND
