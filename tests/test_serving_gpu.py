"""The native request loop: results identical alone and in a mix, admission
bounded by the device-memory pool, host-side rejection and cancellation."""
import numpy as np
import pytest
import torch

from paper_2004_06352_gb300 import inputs as I
from paper_2004_06352_gb300 import serving
from tests import tolerances as T

pytestmark = pytest.mark.gpu


def pinned(shape, dtype):
    return torch.full(shape, float("nan"), dtype=dtype, pin_memory=True)


def build_requests(ctx, lens):
    """A mixed batch over three resident models: Hessian and deflection maps
    (FP32 and FP64), source-plane and image-plane chi2 batches."""
    models = [I.cfg2_model(seed=70 + k, n_members=n) for k, n in enumerate((48, 298, 148))]
    mids = [ctx.model_upload(m) for m in models]
    csets = [ctx.cset_create(mids[k], I.random_constraints(12, seed=80 + k, field=40), (0, 1)) for k in range(3)]
    rng = np.random.default_rng(90)
    reqs = []
    for k in range(24):
        mi = k % 3
        kind = k % 4
        if kind in (0, 1):
            side = int(rng.choice([64, 96, 160, 256]))
            prec = lens.LENS_FP64 if k % 7 == 0 else lens.LENS_MIXED
            reqs.append(("map", mids[mi], side, prec, kind == 0))
        elif kind == 2:
            P = int(rng.choice([16, 64, 200]))
            reqs.append(("src", csets[mi], I.perturbed_params(models[mi], (0, 1), P, seed=100 + k)))
        else:
            reqs.append(("img", csets[mi], I.perturbed_params(models[mi], (0, 1), 4, seed=200 + k)))
    return reqs


def submit(srv, lens, r):
    if r[0] == "map":
        _, mid, side, prec, hess = r
        buf = pinned((6 if hess else 2, side, side), torch.float64 if prec == lens.LENS_FP64 else torch.float32)
        return srv.submit_map(mid, I.grid(side, field=(-80, 80, -80, 80)), 0.9, prec, hess, buf), buf
    if r[0] == "src":
        buf = pinned((len(r[2]),), torch.float64)
        return srv.submit_chi2_source(r[1], r[2], 0, buf), buf
    buf = pinned((len(r[2]),), torch.float64)
    return srv.submit_chi2_image(r[1], I.grid(96, field=(-60, 60, -60, 60)), r[2], buf), buf


def drain(srv, tickets, limit=20000):
    done = {}
    for _ in range(limit):
        for t, st, q, l in srv.progress():
            assert st == 0, st
            done[t] = (q, l)
        if set(tickets) <= set(done):
            return done
        torch.cuda.synchronize()
    raise AssertionError("requests did not complete")


def test_results_identical_alone_and_in_mix(lens):
    with lens.Context(0) as ctx:
        reqs = build_requests(ctx, lens)
        srv = lens.Server(ctx, slots=4, pool_bytes=64 << 20)
        alone = []
        for r in reqs:
            t, buf = submit(srv, lens, r)
            drain(srv, [t])
            alone.append(buf.clone())
        tickets, bufs = [], []
        for r in reqs:
            t, buf = submit(srv, lens, r)
            tickets.append(t)
            bufs.append(buf)
        drain(srv, tickets)
        st = srv.stats()
        assert st["pool_peak"] <= st["pool_bytes"]
        srv.close()
    for r, a, b in zip(reqs, alone, bufs):
        a, b = a.numpy(), b.numpy()
        if r[0] == "img":
            assert np.array_equal(np.isnan(a), np.isnan(b))
            ok = np.isfinite(a)
            assert np.all(np.abs(a[ok] - b[ok]) <= T.CHI2_REL * np.abs(a[ok]))
        else:
            # same kernels on the same inputs: bit-identical whatever else ran
            assert np.array_equal(a, b, equal_nan=True), r[0]


def test_admission_bounded_by_pool_and_slots(lens):
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(I.cfg2_model(seed=5, n_members=100))
        side = 512
        need = 6 * side * side * 4                   # one Hessian map, FP32
        srv = lens.Server(ctx, slots=8, pool_bytes=int(2.5 * need))
        tickets = []
        for _ in range(10):
            t, _ = submit(srv, lens, ("map", mid, side, lens.LENS_MIXED, True))
            tickets.append(t)
        peak_inflight = 0
        done = {}
        for _ in range(20000):
            for t, st, q, l in srv.progress():
                done[t] = l
            peak_inflight = max(peak_inflight, srv.stats()["inflight"])
            if len(done) == len(tickets):
                break
        assert len(done) == len(tickets)
        st = srv.stats()
        assert st["pool_peak"] <= st["pool_bytes"] and peak_inflight <= 2
        srv.close()


def test_rejections_and_cancel(lens):
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(I.random_model(5, seed=6))
        srv = lens.Server(ctx, slots=1, pool_bytes=4 << 20)
        with pytest.raises(lens.LensError) as e:                 # can never fit
            submit(srv, lens, ("map", mid, 1024, lens.LENS_MIXED, True))
        assert e.value.code == lens.LENS_ENOMEM
        with pytest.raises(lens.LensError) as e:                 # pageable result
            srv.submit_map(mid, I.grid(64), 1.0, lens.LENS_MIXED, True, torch.empty((6, 64, 64)))
        assert e.value.code == lens.LENS_EINVAL
        with pytest.raises(lens.LensError) as e:                 # unknown model
            srv.submit_map(mid + 77, I.grid(64), 1.0, lens.LENS_MIXED, True, pinned((6, 64, 64), torch.float32))
        assert e.value.code == lens.LENS_ENOTFOUND
        t1, _ = submit(srv, lens, ("map", mid, 256, lens.LENS_MIXED, True))
        t2, _ = submit(srv, lens, ("map", mid, 256, lens.LENS_MIXED, True))
        t3, _ = submit(srv, lens, ("map", mid, 256, lens.LENS_MIXED, True))
        srv.cancel(t3)                                           # still queued
        done = drain(srv, [t1, t2])
        assert t3 not in done
        with pytest.raises(lens.LensError) as e:
            srv.cancel(t1)                                       # already finished
        assert e.value.code == lens.LENS_ENOTFOUND
        srv.close()


def test_poisson_stream_driver(lens):
    """serving.run_stream over a short Poisson stream of mixed requests."""
    with lens.Context(0) as ctx:
        models = serving.resident_models(2, seed=3, n_range=(10, 200))
        sess = serving.Session(ctx, models)
        reqs = serving.mixed_requests(20, seed=4, n_models=2, sides=(128, 256), p_range=(16, 256))
        srv = lens.Server(ctx, slots=4, pool_bytes=256 << 20)
        lat, wall, done, bufs = serving.run_stream(srv, sess, reqs, serving.poisson_arrivals(20, 200.0, seed=5))
        assert len(lat) == 20 and all(l > 0 for l in lat)
        for t, b in bufs.items():
            assert np.all(np.isfinite(b.numpy()))
        srv.close()


def test_short_requests_go_first(lens):
    """With one slot and everything queued before the first progress call,
    requests run shortest expected work first: a 2048^2 x 300-potential map
    submitted first finishes after the small chi2 batches queued behind it."""
    with lens.Context(0) as ctx:
        m = I.cfg2_model(seed=9, n_members=298)
        mid = ctx.model_upload(m)
        cs = ctx.cset_create(mid, I.random_constraints(10, seed=10, field=40), (0, 1))
        srv = lens.Server(ctx, slots=1, pool_bytes=256 << 20)
        big = pinned((6, 2048, 2048), torch.float32)
        t_big = srv.submit_map(mid, I.grid(2048), 1.0, lens.LENS_MIXED, True, big)
        small = []
        for k in range(3):
            buf = pinned((32,), torch.float64)
            small.append((srv.submit_chi2_source(cs, I.perturbed_params(m, (0, 1), 32, seed=11 + k), 0, buf), buf))
        order = []
        for _ in range(200000):
            for t, st, q, l in srv.progress():
                assert st == 0
                order.append(t)
            if len(order) == 4:
                break
        assert order[-1] == t_big, order
        assert sorted(order[:3]) == sorted(t for t, _ in small)
        assert np.all(np.isfinite(big.numpy()[:5]))
        srv.close()


def test_image_chi2_beyond_the_kernels_limits_is_refused_everywhere(lens):
    """A constraint set with more sources than the image search's shared
    arrays hold (1025 > 1024) is refused with LENS_EINVAL before anything is
    launched: by lens_chi2_image, by the allocation-free entry point and by
    the request loop's submit (nothing queued, nothing in flight)."""
    m = I.cfg2_model(seed=77, n_members=8)
    cons = I.random_constraints(1025, seed=78, mult=(2, 2), field=40)
    params = I.perturbed_params(m, (0, 1), 2, seed=79)
    g = I.grid(64, field=(-60, 60, -60, 60))
    with lens.Context(0) as ctx:
        cs = ctx.cset_create(ctx.model_upload(m), cons, (0, 1))
        p = torch.tensor(params, dtype=torch.float64, device="cuda:0")
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda:0")
        for call in (ctx.chi2_image, ctx.chi2_image_noalloc):
            with pytest.raises(lens.LensError) as e:
                call(cs, g, p, 2, out)
            assert e.value.code == lens.LENS_EINVAL
        srv = lens.Server(ctx, slots=2, pool_bytes=256 << 20)
        buf = pinned((2,), torch.float64)
        with pytest.raises(lens.LensError) as e:
            srv.submit_chi2_image(cs, g, params, buf)
        assert e.value.code == lens.LENS_EINVAL
        st = srv.stats()
        assert st["queued"] == 0 and st["inflight"] == 0 and st["pool_used"] == 0
        srv.close()
        ctx.wait()
        assert torch.equal(out.cpu(), torch.full((2,), -1.0, dtype=torch.float64))
        assert torch.isnan(buf).all()
