"""GPU map parity against the FP64 oracle, through the C ABI.

Small grids span several 32-wide tiles with ragged tails in x and y; the
full-size 2048^2 / 1000-potential case is checked on sampled grid points in
the launch configuration the benchmark times.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_06352_gb300 import inputs as I
from tests import tolerances as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def run_map(lens, m, g, dls, precision, hess, threshold=None):
    dt = torch.float32 if precision == lens.LENS_MIXED else torch.float64
    with lens.Context(0) as ctx:
        if threshold is not None:
            ctx.set_fp64_threshold(threshold)
        mid = ctx.model_upload(m)
        out = torch.full((6 if hess else 2, g["ny"], g["nx"]), float("nan"), dtype=dt, device=DEV)
        (ctx.hessian_map if hess else ctx.grad_map)(mid, g, dls, precision, out)
        ctx.wait()
        return out.cpu().numpy().astype(np.float64)


def check_mixed(res, ref, hess, peak=None):
    bad, err, _ = T.alpha_violations(res[0], res[1], ref[0], ref[1], peak=peak)
    n, msg = T.report("alpha", bad, err)
    assert n == 0, msg
    if hess:
        badh = T.hess_violations(res[2], res[3], res[4], ref[2], ref[3], ref[4])
        assert not badh.any(), T.report("kappa/gamma", badh)[1]
        badm = T.mu_violations(res[5], ref[5])
        assert not badm.any(), T.report("mu", badm)[1]


def check_fp64(res, ref):
    for k in range(res.shape[0] - (1 if res.shape[0] == 6 else 0)):
        scale = np.maximum(np.abs(ref[k]), 1e-3 * np.abs(ref[k]).max() + 1e-300)
        assert np.all(np.abs(res[k] - ref[k]) <= 1e-11 * scale), k
    if res.shape[0] == 6:
        det, rdet = 1 / res[5], 1 / ref[5]
        assert np.all(np.abs(det - rdet) <= 1e-11 * np.maximum(1, np.abs(rdet)))


def test_fp64_grad_map_cfg1(lens):
    """The 256^2, 10-halo FP64 deflection map (plain FP64 GPU form)."""
    m, g = I.cfg1_model(), I.grid(256)
    res = run_map(lens, m, g, 0.7, lens.LENS_FP64, False)
    check_fp64(res, oracle.maps(m, g, 0.7, 2))


def test_fp64_hessian_map_mixed_types(lens):
    m = I.random_model(37, seed=21, types=(I.DPIE, I.DPIE, I.SIS, I.POINT))
    g = I.grid(71, field=(-65, 65, -50, 55), ny=43)
    res = run_map(lens, m, g, 0.55, lens.LENS_FP64, True)
    check_fp64(res, oracle.maps(m, g, 0.55, 6))


@pytest.mark.parametrize("hess", [False, True])
def test_mixed_map_ragged_tiles_all_kinds(lens, hess):
    """Several tiles, ragged in x and y; dPIE (incl. eps = 0 and the series
    branch), SIS, point mass, cluster-scale potentials on the FP64 path, and a
    light-potential count that is not a multiple of the chunk or fold size."""
    m = I.random_model(203, seed=22, types=(I.DPIE, I.DPIE, I.DPIE, I.SIS, I.POINT))
    m[0, 4], m[1, 4], m[2, 4] = 0.0, 1e-6, 0.002   # eps = 0, tiny, series branch
    m[5, 7], m[10, 7] = 28.0, 17.0                 # FP64 path
    g = I.grid(101, field=(-80, 80, -70, 75), ny=77)
    res = run_map(lens, m, g, 0.8, lens.LENS_MIXED, hess)
    check_mixed(res, oracle.maps(m, g, 0.8, 6 if hess else 2), hess)


def test_mixed_map_all_heavy_and_all_light(lens):
    """Threshold 0 puts every potential on the FP64 path; an infinite one puts
    every potential on the FP32 path (galaxy-scale halos, the class the FP32
    path is meant for)."""
    g = I.grid(40, field=(-50, 50, -50, 50))
    m = I.random_model(9, seed=23)
    check_mixed(run_map(lens, m, g, 1.0, lens.LENS_MIXED, True, threshold=0.0), oracle.maps(m, g, 1.0, 6), True)
    m = I.member_model(150, seed=25, field=50)
    check_mixed(run_map(lens, m, g, 1.0, lens.LENS_MIXED, True, threshold=1e9), oracle.maps(m, g, 1.0, 6), True)


@pytest.mark.parametrize("members", [998, 215])
def test_mixed_map_cluster_potentials_fp64_and_double_float(lens, members):
    """The two cluster-scale potentials take the FP64 path when the model has
    400 or more FP32 potentials per cluster-scale one (998 members: 499) and
    the double-float path below that (215 members: 107.5); both against the
    oracle, deflection and Hessian, on a ragged grid over the cluster."""
    m = I.cfg2_model(n_members=members)
    g = I.grid(97, field=(-100, 100, -100, 100), ny=83)
    for hess in (False, True):
        res = run_map(lens, m, g, 0.7, lens.LENS_MIXED, hess)
        check_mixed(res, oracle.maps(m, g, 0.7, 6 if hess else 2), hess)


def test_mixed_map_single_halo_and_minimal_grid(lens):
    m = I.halo_row(I.DPIE, 0.3, -0.2, 0.4, 0.35, 0.5, 30.0, 2.0)[None]
    for g in (I.grid(2, field=(-1, 1, -1, 1)), I.grid(33, field=(-10, 10, -3, 3), ny=2)):
        check_mixed(run_map(lens, m, g, 0.9, lens.LENS_MIXED, True), oracle.maps(m, g, 0.9, 6), True)


def test_point_on_sis_and_point_mass_centre(lens):
    """Grid nodes exactly on an SIS / point-mass centre get zero from it."""
    m = np.vstack([I.halo_row(I.SIS, 0.0, 0.0, 0, 0, 0, 0, 1.5),
                   I.halo_row(I.POINT, 5.0, 5.0, 0, 0, 0, 0, 1.0),
                   I.halo_row(I.DPIE, 2.0, -3.0, 0.2, 0.3, 0.4, 20.0, 2.0)])
    g = I.grid(21, field=(-10, 10, -10, 10))
    for prec in (lens.LENS_MIXED, lens.LENS_FP64):
        res = run_map(lens, m, g, 1.0, prec, True)
        assert np.all(np.isfinite(res[:5]))
    check_mixed(run_map(lens, m, g, 1.0, lens.LENS_MIXED, True), oracle.maps(m, g, 1.0, 6), True)


def test_full_size_cfg2_sampled(lens):
    """2048^2 grid, 1000 potentials (2 cluster + 998 members), the benchmark's
    launch; 12k sampled grid nodes compared with the oracle."""
    m, g = I.cfg2_model(), I.grid(2048)
    res = torch.from_numpy(run_map(lens, m, g, 1.0, lens.LENS_MIXED, True))
    rng = np.random.default_rng(24)
    n = 12000
    ii, jj = rng.integers(0, 2048, n), rng.integers(0, 2048, n)
    ii[:4], jj[:4] = [0, 2047, 0, 2047], [0, 0, 2047, 2047]  # corners
    dx = 200.0 / 2047
    X, Y = -100.0 + ii * dx, -100.0 + jj * dx
    ev = oracle.model_eval(m, X, Y, 1.0)
    ref = np.stack([ev[:, 0], ev[:, 1], 0.5 * (ev[:, 2] + ev[:, 3]), 0.5 * (ev[:, 2] - ev[:, 3]), ev[:, 4]])
    det = (1 - ref[2]) ** 2 - ref[3] ** 2 - ref[4] ** 2
    ref = np.vstack([ref, 1 / det])
    got = res[:, jj, ii].numpy()
    check_mixed(got, ref, True)
    # every node of a 48 x 48 block around the smallest deflection of the map
    # (the cluster's centre of deflection, where the absolute floor of the
    # alpha tolerance applies), against the map's peak deflection
    peak = float(np.hypot(ref[0], ref[1]).max())
    a = torch.hypot(res[0], res[1])
    j0, i0 = divmod(int(torch.argmin(a)), 2048)
    j0, i0 = min(max(j0 - 24, 0), 2048 - 48), min(max(i0 - 24, 0), 2048 - 48)
    jb, ib = np.meshgrid(np.arange(j0, j0 + 48), np.arange(i0, i0 + 48), indexing="ij")
    jb, ib = jb.ravel(), ib.ravel()
    ev = oracle.model_eval(m, -100.0 + ib * dx, -100.0 + jb * dx, 1.0)
    ref = np.stack([ev[:, 0], ev[:, 1], 0.5 * (ev[:, 2] + ev[:, 3]), 0.5 * (ev[:, 2] - ev[:, 3]), ev[:, 4]])
    ref = np.vstack([ref, 1 / ((1 - ref[2]) ** 2 - ref[3] ** 2 - ref[4] ** 2)])
    assert np.hypot(ref[0], ref[1]).min() < 0.05 * peak
    check_mixed(res[:, jb, ib].numpy(), ref, True, peak=peak)


def test_full_size_cfg2_sampled_deflection_only(lens):
    """The deflection-only kernel (its own launch shape: 4 points per thread)
    on the 2048^2 x 1000 workload; 12k sampled nodes against the oracle."""
    m, g = I.cfg2_model(), I.grid(2048)
    res = run_map(lens, m, g, 0.7, lens.LENS_MIXED, False)
    rng = np.random.default_rng(25)
    n = 12000
    ii, jj = rng.integers(0, 2048, n), rng.integers(0, 2048, n)
    ii[:4], jj[:4] = [0, 2047, 0, 2047], [0, 0, 2047, 2047]  # corners
    dx = 200.0 / 2047
    ev = oracle.model_eval(m, -100.0 + ii * dx, -100.0 + jj * dx, 0.7)
    check_mixed(res[:, jj, ii], np.stack([ev[:, 0], ev[:, 1]]), False)


def test_largest_grids_sampled(lens):
    """The largest maps: the request loop's biggest (an 8192^2 Hessian map of a
    2000-potential model) and a deflection map of 46341 x 46340 nodes, just
    under the 2^31 - 1 node limit of the 32-bit node indices (the repair
    list's entries), against the oracle at sampled nodes, the grid's corners
    and last row included; sampled on the device (the big map is 17 GB)."""
    big = dict(xmin=-100.0, xmax=100.0, ymin=-100.0, ymax=100.0, nx=46341, ny=46340)
    assert big["nx"] * big["ny"] < 2 ** 31 - 1
    cases = [(I.cfg2_model(n_members=1998), I.grid(8192), True), (I.cfg1_model(), big, False)]
    rng = np.random.default_rng(26)
    with lens.Context(0) as ctx:
        for m, g, hess in cases:
            mid = ctx.model_upload(m)
            nx, ny = g["nx"], g["ny"]
            out = torch.empty((6 if hess else 2, ny, nx), dtype=torch.float32, device=DEV)
            (ctx.hessian_map if hess else ctx.grad_map)(mid, g, 1.0, lens.LENS_MIXED, out)
            ctx.wait()
            n = 3000
            ii, jj = rng.integers(0, nx, n), rng.integers(0, ny, n)
            ii[:6], jj[:6] = [0, nx - 1, 0, nx - 1, nx // 2, nx - 2], [0, 0, ny - 1, ny - 1, ny - 1, ny - 1]
            got = out[:, torch.from_numpy(jj).to(DEV), torch.from_numpy(ii).to(DEV)].cpu().numpy()
            del out
            dx, dy = (g["xmax"] - g["xmin"]) / (nx - 1), (g["ymax"] - g["ymin"]) / (ny - 1)
            ev = oracle.model_eval(m, g["xmin"] + ii * dx, g["ymin"] + jj * dy, 1.0)
            if hess:
                ref = np.stack([ev[:, 0], ev[:, 1], 0.5 * (ev[:, 2] + ev[:, 3]), 0.5 * (ev[:, 2] - ev[:, 3]), ev[:, 4]])
                ref = np.vstack([ref, 1 / ((1 - ref[2]) ** 2 - ref[3] ** 2 - ref[4] ** 2)])
            else:
                ref = np.stack([ev[:, 0], ev[:, 1]])
            check_mixed(got.astype(np.float64), ref, hess)
            ctx.model_release(mid)


def test_invalid_inputs_rejected(lens):
    with lens.Context(0) as ctx:
        bad = [I.halo_row(I.DPIE, 0, 0, 0, 1.0, 1, 10, 1),      # eps = 1
               I.halo_row(I.DPIE, 0, 0, 0, 0.2, 10, 5, 1),      # rcut < rcore
               I.halo_row(I.DPIE, 0, 0, 0, 0.2, 0, 5, 1),       # rcore = 0
               I.halo_row(I.SIS, 0, 0, 0, 0, 0, 0, -1),         # b0 < 0
               I.halo_row(7, 0, 0, 0, 0, 0, 0, 1),              # type
               I.halo_row(I.DPIE, np.nan, 0, 0, 0.2, 1, 5, 1)]  # NaN
        for row in bad:
            with pytest.raises(lens.LensError) as e:
                ctx.model_upload(row[None])
            assert e.value.code == lens.LENS_EINVAL
        mid = ctx.model_upload(I.random_model(3, seed=1))
        out = torch.empty((2, 4, 4), device=DEV)
        for g in (dict(xmin=0, xmax=1, ymin=0, ymax=1, nx=1, ny=4), dict(xmin=1, xmax=0, ymin=0, ymax=1, nx=4, ny=4),
                  dict(xmin=0, xmax=np.inf, ymin=0, ymax=1, nx=4, ny=4),
                  # beyond 2^31 - 1 nodes and beyond the launch's rows: refused
                  # on the host before anything is launched
                  dict(xmin=0, xmax=1, ymin=0, ymax=1, nx=65536, ny=32769),
                  dict(xmin=0, xmax=1, ymin=0, ymax=1, nx=2, ny=524281)):
            with pytest.raises(lens.LensError) as e:
                ctx.grad_map(mid, g, 1.0, lens.LENS_MIXED, out)
            assert e.value.code == lens.LENS_EINVAL
        with pytest.raises(lens.LensError) as e:
            ctx.grad_map(mid + 99, I.grid(4), 1.0, lens.LENS_MIXED, out)
        assert e.value.code == lens.LENS_ENOTFOUND
        with pytest.raises(lens.LensError) as e:
            ctx.grad_map(mid, I.grid(4), -1.0, lens.LENS_MIXED, out)
        assert e.value.code == lens.LENS_EINVAL


def test_memory_budget_admission(lens):
    with lens.Context(0, mem_budget_bytes=64 * 1024) as ctx:
        ctx.model_upload(I.random_model(10, seed=2))
        with pytest.raises(lens.LensError) as e:
            ctx.model_upload(I.random_model(2000, seed=3))
        assert e.value.code == lens.LENS_ENOMEM


@pytest.mark.parametrize("hess", [True, False])
def test_map_to_host_equals_device_map(lens, hess):
    """lens_*_map_host (row bands streamed to pinned host memory) gives the
    device map's values bit for bit, on a grid whose rows are not a multiple
    of the band, in both precisions; pageable memory is rejected."""
    m = I.random_model(40, seed=81, types=(I.DPIE, I.DPIE, I.SIS, I.POINT))
    m[0, 7] = 20.0  # one potential on the FP64 path
    g = I.grid(97, field=(-60, 60, -50, 50), ny=203)
    planes = 6 if hess else 2
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        for prec, dt in ((lens.LENS_MIXED, torch.float32), (lens.LENS_FP64, torch.float64)):
            dev = torch.empty((planes, g["ny"], g["nx"]), dtype=dt, device=DEV)
            host = torch.full((planes, g["ny"], g["nx"]), float("nan"), dtype=dt, pin_memory=True)
            (ctx.hessian_map if hess else ctx.grad_map)(mid, g, 0.9, prec, dev)
            (ctx.hessian_map_host if hess else ctx.grad_map_host)(mid, g, 0.9, prec, host)
            ctx.wait()
            assert torch.equal(host, dev.cpu())
        pageable = torch.empty((planes, g["ny"], g["nx"]), dtype=torch.float32)
        with pytest.raises(lens.LensError) as e:
            (ctx.hessian_map_host if hess else ctx.grad_map_host)(mid, g, 0.9, lens.LENS_MIXED, pageable)
        assert e.value.code == lens.LENS_EINVAL


def test_model_blocks_are_reused_and_yield_to_the_budget(lens):
    """A released model's device block serves the next upload of similar
    size (no growth of the context's memory, same maps as a fresh context);
    kept blocks are freed when an upload would exceed the budget."""
    a, b = I.random_model(300, seed=12), I.random_model(290, seed=13)  # b fits in a's block
    g = I.grid(40, field=(-60, 60, -60, 60))
    with lens.Context(0) as ctx:
        ma = ctx.model_upload(a)
        nbytes = ctx.model_bytes(ma)
        assert nbytes > 300 * 400
        used = ctx.mem_used()
        ctx.model_release(ma)
        mb = ctx.model_upload(b)
        assert ctx.mem_used() == used
        out = torch.empty((6, 40, 40), device=DEV)
        ctx.hessian_map(mb, g, 1.0, lens.LENS_MIXED, out)
        ctx.wait()
    with lens.Context(0) as fresh:
        ref = torch.empty((6, 40, 40), device=DEV)
        fresh.hessian_map(fresh.model_upload(b), g, 1.0, lens.LENS_MIXED, ref)
        fresh.wait()
    assert torch.equal(out, ref)
    with lens.Context(0, mem_budget_bytes=3 * nbytes // 2) as ctx:
        ctx.model_release(ctx.model_upload(a))      # kept for reuse
        big = I.random_model(420, seed=14)          # too big to reuse, fits once the kept block goes
        mid = ctx.model_upload(big)
        assert ctx.model_bytes(mid) > nbytes
