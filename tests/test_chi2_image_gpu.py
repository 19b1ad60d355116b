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


def gpu_images(ctx, cs, grid, params, max_per_set=2048):
    P = len(params)
    imgs = torch.empty((P, max_per_set, 3), dtype=torch.float64, device=DEV)
    cnt = torch.empty(P, dtype=torch.int32, device=DEV)
    ctx.find_images(cs, grid, torch.tensor(params, dtype=torch.float64, device=DEV), P, imgs, cnt)
    ctx.wait()
    imgs, cnt = imgs.cpu().numpy(), cnt.cpu().numpy()
    return [imgs[p, :cnt[p]] for p in range(P)]


def chi2_from_images(cons, imgs):
    """Eq. 6 with each constraint matched to the nearest image of its source."""
    off = cons["img_off"]
    tot = 0.0
    for i in range(len(off) - 1):
        mine = imgs[imgs[:, 2] == i, :2]
        for j in range(off[i], off[i + 1]):
            if len(mine) == 0:
                return np.nan
            d2 = np.min(np.sum((mine - [cons["x"][j], cons["y"][j]]) ** 2, axis=1))
            tot += d2 / cons["sigma"][j] ** 2
    return tot


def check_chi2_image_parity(lens, n, P, seed):
    """The 1000-potential model, 100 sources / 372 images at 5 distance
    ratios, the two cluster halos varying, an n x n search grid over
    [-100, 100]^2; P parameter sets, the first being the model itself.

    Where a cell is far from linear (a galaxy core or a fold inside it), the
    grid search is ill-conditioned: the oracle reports such images with a
    difficulty >= 100 (refinement cut short).  So: every well-conditioned
    oracle image must be found; an image found by only one side must be an
    ill-conditioned oracle image or, on the GPU side, a true root; such
    differences stay rare; each GPU chi2 equals Eq. 6 recomputed from the
    GPU's own images, and the oracle's chi2 wherever the image sets agree,
    which must happen for at least one set."""
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    g = I.grid(n)
    params = I.perturbed_params(m, var, P, seed=seed)
    params[0] = I.var_params_of(m, var)
    ref, nf_ref = oracle.chi2_image_batch(m, cons, g, var, params)
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        got, nf = gpu_chi2_image(lens, m, cons, var, g, params, ctx=ctx)
        imgs = gpu_images(ctx, cs, g, params)
    differ, total, compared = 0, 0, 0
    for p in range(len(params)):
        mp = oracle.apply_params(m, var, params[p])
        _, bary = oracle.backtrace(mp, cons)
        ag = oracle.alpha_grid(mp, g)
        same = True
        for i in range(len(cons["img_off"]) - 1):
            r = cons["dls_ds"][i]
            ref_i, _, dif = oracle.find_images(mp, g, r, bary[i], ag=ag, with_difficulty=True)
            mine = imgs[p][imgs[p][:, 2] == i, :2]
            assert len(mine) == nf[p, i]
            total += len(ref_i)
            for x, d in zip(ref_i, dif):
                if len(mine) and np.min(np.hypot(*(mine - x).T)) < 1e-6:
                    continue
                assert d >= 100, (p, i, x, d)      # only an ill-conditioned image may be missed
                same = False
                differ += 1
            for y in mine:
                if len(ref_i) and np.min(np.hypot(*(ref_i - y).T)) < 1e-6:
                    continue
                same = False
                differ += 1
                ev = oracle.model_eval(mp, y[0], y[1], r)[0]
                assert np.hypot(*(y - ev[:2] - bary[i])) < 1e-9, (p, i, y)   # a true image
        mine_chi2 = chi2_from_images(cons, imgs[p])
        assert abs(got[p] - mine_chi2) <= T.CHI2_REL * abs(mine_chi2)
        if same:
            assert np.array_equal(nf[p], nf_ref[p])
            assert abs(got[p] - ref[p]) <= T.CHI2_REL * abs(ref[p]), (p, got[p], ref[p])
            compared += 1
    assert differ <= 0.01 * total, (differ, total)
    assert compared >= 1, "no parameter set had the oracle's image sets"
    return compared


def test_chi2_image_cfg2_model_parity(lens):
    """256^2 search grid (0.78" cells), 5 parameter sets."""
    check_chi2_image_parity(lens, 256, 5, seed=41)


def test_chi2_image_cfg2_model_parity_bench_grid(lens):
    """The benchmark's 1024^2 search grid (0.20" cells: more candidates per
    source, and the refinement starts at a finer scale), 3 parameter sets."""
    check_chi2_image_parity(lens, 1024, 3, seed=45)


def test_chi2_image_at_the_source_limit(lens):
    """1024 sources, as many as the image search's shared arrays hold, on a
    smooth lens (the two varying cluster halos scaled down, four members far
    outside the field: no galaxy core inside a search cell, few multiple
    images): per-source image counts equal to the oracle's and the chi2
    within 1e-8, for the model itself and a perturbed set."""
    m = I.cfg2_model(seed=85, n_members=4)
    m[:2, 7] *= 0.15
    m[2:, 1] += 400.0
    cons = I.random_constraints(1024, seed=86, mult=(2, 2), field=40)
    var = (0, 1)
    params = I.perturbed_params(m, var, 2, seed=87)
    params[0] = I.var_params_of(m, var)
    g = I.grid(256, field=(-60, 60, -60, 60))
    ref, nf_ref = oracle.chi2_image_batch(m, cons, g, var, params)
    got, nf = gpu_chi2_image(lens, m, cons, var, g, params)
    assert np.all(nf_ref >= 1)
    assert np.array_equal(nf, nf_ref)
    assert np.all(np.abs(got - ref) <= T.CHI2_REL * np.abs(ref)), (got, ref)


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


def test_chi2_image_batched_sets_match_single_calls(lens):
    """P = 260 spans a full 256-set batch and a ragged one; every set's chi2
    and image counts equal those of the same set evaluated alone."""
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    g = I.grid(256)
    P = 260
    params = I.perturbed_params(m, var, P, seed=71)
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        p = torch.tensor(params, device=DEV)
        allc = torch.empty(P, dtype=torch.float64, device=DEV)
        alln = torch.empty((P, len(cons["img_off"]) - 1), dtype=torch.int32, device=DEV)
        ctx.chi2_image(cs, g, p, P, allc, alln)
        ctx.wait()
        for k in (0, 1, 255, 256, 259):
            one = torch.empty(1, dtype=torch.float64, device=DEV)
            onen = torch.empty((1, alln.shape[1]), dtype=torch.int32, device=DEV)
            ctx.chi2_image(cs, g, p[k:k + 1], 1, one, onen)
            ctx.wait()
            assert torch.equal(onen[0], alln[k]), k
            a, b = float(allc[k]), float(one[0])
            assert (np.isnan(a) and np.isnan(b)) or abs(a - b) <= T.CHI2_REL * abs(b), (k, a, b)


def test_chi2_image_candidate_overflow_is_nan_and_reported(lens):
    """1024 sources (the maximum) at one position inside a five-image caustic
    produce more than the 4096 candidates a set can hold: the set's chi2 is
    NaN, every count is -1, lens_wait reports LENS_ECAPACITY once, and the
    context keeps working."""
    m = np.vstack([I.halo_row(I.DPIE, 0.0, 0.0, 0.3, 0.3, 0.5, 200.0, 20.0),
                   I.halo_row(I.DPIE, 35.0, 30.0, 0.0, 0.1, 0.2, 20.0, 1.0)])
    g = I.grid(128, field=(-50, 50, -50, 50))
    n = 1024
    cons = I.constraints_dict(np.arange(n + 1), np.full(n, 0.05), np.full(n, 0.03), np.full(n, 0.1),
                              np.full(n, 0.9))
    params = I.var_params_of(m, (0, 1))[None]
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, (0, 1))
        p = torch.tensor(params, device=DEV)
        out = torch.zeros(1, dtype=torch.float64, device=DEV)
        nf = torch.zeros((1, n), dtype=torch.int32, device=DEV)
        ctx.chi2_image(cs, g, p, 1, out, nf)
        with pytest.raises(lens.LensError) as e:
            ctx.wait()
        assert e.value.code == lens.LENS_ECAPACITY
        assert np.isnan(float(out[0])) and bool(torch.all(nf == -1))
        ctx.wait()  # the flag was cleared
        small = I.constraints_dict(np.arange(5), np.full(4, 0.05), np.full(4, 0.03), np.full(4, 0.1),
                                   np.full(4, 0.9))
        cs2 = ctx.cset_create(mid, small, (0, 1))
        nf2 = torch.zeros((1, 4), dtype=torch.int32, device=DEV)
        ctx.chi2_image(cs2, g, p, 1, out, nf2)
        ctx.wait()
        assert bool(torch.all(nf2 == 5)) and np.isfinite(float(out[0]))


def test_chi2_image_source_without_images_is_nan(lens):
    """A source far outside the lensed field has no image on the grid: its
    count is 0 and the set's chi2 is NaN (no finite Eq. 6 without a match);
    the other sources still get their images."""
    m = np.vstack([I.halo_row(I.DPIE, 0.0, 0.0, 0.3, 0.3, 0.5, 200.0, 20.0),
                   I.halo_row(I.DPIE, 35.0, 30.0, 0.0, 0.1, 0.2, 20.0, 1.0)])
    g = I.grid(96, field=(-40, 40, -30, 30), ny=72)   # nx != ny
    # source 0: one image at (0.3, 0.1) (inside the caustic); source 1: a
    # constraint at the field's edge whose back-traced source maps nowhere
    # on the grid (its images would lie outside it)
    cons = I.constraints_dict([0, 1, 2], [0.3, 1.0e3], [0.1, 1.0e3], [0.1, 0.1], [0.9, 0.9])
    params = I.var_params_of(m, (0, 1))[None]
    ref, nf_ref = oracle.chi2_image_batch(m, cons, g, (0, 1), params)
    with lens.Context(0) as ctx:
        got, nf = gpu_chi2_image(lens, m, cons, (0, 1), g, params, ctx=ctx)
    assert np.isnan(ref[0]) and np.isnan(got[0])
    assert nf_ref[0, 1] == 0 and nf[0, 1] == 0
    assert nf[0, 0] == nf_ref[0, 0] == 5


def test_chi2_image_static_sis_and_point_mass(lens):
    """Static SIS and point-mass potentials beside the varying dPIEs (their
    polish terms take the double-float circular path): constraints placed
    on the oracle's images give chi2 ~ 0 and the oracle's image counts."""
    m = np.vstack([I.halo_row(I.DPIE, 0.3, -0.2, 0.5, 0.3, 1.5, 300.0, 12.0),
                   I.halo_row(I.DPIE, -2.0, 1.0, 1.1, 0.2, 0.8, 150.0, 6.0),
                   I.halo_row(I.SIS, 6.0, -4.0, 0.0, 0.0, 0.0, 0.0, 1.2),
                   I.halo_row(I.POINT, -7.0, 5.0, 0.0, 0.0, 0.0, 0.0, 0.9),
                   I.member_model(12, seed=45, field=30)])
    g = I.grid(161, field=(-40, 40, -40, 40))
    xs, ys, off, rs = [], [], [0], []
    for bs, r in (((0.4, 0.3), 0.7), ((-0.6, 0.2), 0.9), ((1.5, -1.0), 0.8)):
        img, nfound = oracle.find_images(m, g, r, bs)
        assert nfound >= 1
        xs += list(img[:, 0])
        ys += list(img[:, 1])
        off.append(len(xs))
        rs.append(r)
    cons = I.constraints_dict(off, xs, ys, np.full(len(xs), 0.05), rs)
    params = I.var_params_of(m, (0, 1))[None]
    got, nf = gpu_chi2_image(lens, m, cons, (0, 1), g, params)
    assert got[0] < 1e-12, got
    assert list(nf[0]) == [off[i + 1] - off[i] for i in range(3)]


def test_find_images_truncates_to_capacity(lens):
    """d_count holds every set's number of images; only the first max_per_set
    are written, and they are among the images of an uncapped call."""
    m = np.vstack([I.halo_row(I.DPIE, 0.3, -0.2, 0.5, 0.3, 1.5, 300.0, 12.0),
                   I.halo_row(I.DPIE, -2.0, 1.0, 1.1, 0.2, 0.8, 150.0, 6.0),
                   I.member_model(8, seed=46, field=30)])
    g = I.grid(121, field=(-40, 40, -40, 40))
    cons = I.constraints_dict([0, 1, 2, 3], [0.4, -0.6, 1.2], [0.3, 0.2, -0.9], [0.1, 0.1, 0.1], [0.7, 0.9, 0.8])
    params = I.perturbed_params(m, (0, 1), 3, seed=47)
    with lens.Context(0) as ctx:
        cs = ctx.cset_create(ctx.model_upload(m), cons, (0, 1))
        full = gpu_images(ctx, cs, g, params, max_per_set=64)
        P = len(params)
        imgs = torch.full((P, 3, 3), -9.0, dtype=torch.float64, device=DEV)
        cnt = torch.empty(P, dtype=torch.int32, device=DEV)
        ctx.find_images(cs, g, torch.tensor(params, device=DEV), P, imgs, cnt)
        ctx.wait()
        imgs, cnt = imgs.cpu().numpy(), cnt.cpu().numpy()
    for p in range(P):
        assert cnt[p] == len(full[p]) > 3
        for row in imgs[p]:
            same_src = full[p][full[p][:, 2] == row[2]]
            assert len(same_src) and np.min(np.hypot(same_src[:, 0] - row[0], same_src[:, 1] - row[1])) < 1e-9, (p, row)


def test_calls_on_two_streams_of_one_context(lens):
    """Image-plane and no-cache source-plane chi2 of different parameter
    sets enqueued on two streams of one context at once: each call's working
    memory is its own (stream-ordered), so every result equals the one the
    same call gives alone; a model released while a map that reads it is in
    flight keeps its memory until that map is done, and an upload that reuses
    the block afterwards does not disturb it."""
    m = I.cfg2_model()
    cons = make_constraints.load()
    var = (0, 1)
    g = I.grid(256)
    pa = torch.tensor(I.perturbed_params(m, var, 40, seed=61), device=DEV)
    pb = torch.tensor(I.perturbed_params(m, var, 40, seed=62), device=DEV)
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, cons, var)
        ref = {}
        for name, p in (("a", pa), ("b", pb)):
            oi = torch.empty(40, dtype=torch.float64, device=DEV)
            on = torch.empty(40, dtype=torch.float64, device=DEV)
            ctx.chi2_image(cs, g, p, 40, oi)
            ctx.chi2_source_nocache(cs, p, 40, 0, on)
            ctx.wait()
            ref[name] = (oi.clone(), on.clone())
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        outs = {k: (torch.full((40,), -1.0, dtype=torch.float64, device=DEV),
                    torch.full((40,), -1.0, dtype=torch.float64, device=DEV)) for k in ("a", "b")}
        torch.cuda.synchronize()
        for _ in range(3):
            for name, p, st in (("a", pa, s1), ("b", pb, s2)):
                ctx.chi2_image(cs, g, p, 40, outs[name][0], stream=st)
                ctx.chi2_source_nocache(cs, p, 40, 0, outs[name][1], stream=st)
        torch.cuda.synchronize()
        # (the image search appends candidates with atomics, so the last
        # bits of an image-plane chi2 may differ from run to run)
        for k in ("a", "b"):
            for got, want in zip(outs[k], ref[k]):
                rel = (got - want).abs() / want.abs()
                assert float(rel.max()) <= T.CHI2_REL, (k, float(rel.max()))
        # release while in flight, then reuse of the released block
        m2 = I.random_model(300, seed=63)
        gm = I.grid(512, field=(-60, 60, -60, 60))
        mid2 = ctx.model_upload(m2)
        want = torch.empty((6, 512, 512), device=DEV)
        ctx.hessian_map(mid2, gm, 1.0, lens.LENS_MIXED, want)
        ctx.wait()
        got = torch.empty_like(want)
        ctx.hessian_map(mid2, gm, 1.0, lens.LENS_MIXED, got, stream=s1)
        ctx.model_release(mid2)                   # the map above is still running
        mid3 = ctx.model_upload(I.random_model(290, seed=64))   # may take the released block
        other = torch.empty_like(want)
        ctx.hessian_map(mid3, gm, 1.0, lens.LENS_MIXED, other, stream=s2)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
