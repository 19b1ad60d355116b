"""Failure detection without a GPU fault: the device-side bounded wait gives
up and reports through lens_wait, and lens_wait's own host-side limit; the
context stays usable after both."""
import numpy as np
import pytest
import torch

from paper_2004_06352_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def small_map_ok(lens, ctx):
    mid = ctx.model_upload(I.random_model(8, seed=91))
    out = torch.empty((6, 33, 33), device=DEV)
    ctx.hessian_map(mid, I.grid(33, field=(-20, 20, -20, 20)), 1.0, lens.LENS_MIXED, out)
    ctx.wait()
    return bool(torch.all(torch.isfinite(out[:5])))


def test_device_wait_gives_up_and_is_reported(lens):
    with lens.Context(0) as ctx:
        ctx.selftest_wait(64)          # an mbarrier nothing completes
        with pytest.raises(lens.LensError) as e:
            ctx.wait()
        assert e.value.code == lens.LENS_ETIMEOUT
        ctx.wait()                     # the flag was cleared
        assert small_map_ok(lens, ctx)
        with pytest.raises(lens.LensError) as e:
            ctx.selftest_wait(0)       # out of range
        assert e.value.code == lens.LENS_EINVAL


def test_host_wait_limit(lens):
    """A plain-FP64 Hessian map of 1024^2 x 1000 potentials runs for a few
    hundred ms: a zero host limit reports LENS_ETIMEOUT without stopping it,
    and a later wait returns once it is done."""
    with lens.Context(0) as ctx:
        mid = ctx.model_upload(I.cfg2_model())
        out = torch.empty((6, 1024, 1024), dtype=torch.float64, device=DEV)
        ctx.hessian_map(mid, I.grid(1024), 1.0, lens.LENS_FP64, out)
        with pytest.raises(lens.LensError) as e:
            ctx.wait(timeout_ms=0)
        assert e.value.code == lens.LENS_ETIMEOUT
        ctx.wait(timeout_ms=60000)
        assert bool(torch.all(torch.isfinite(out[:5])))
        assert small_map_ok(lens, ctx)
