"""The FP64 reciprocal and reciprocal square root used by the FP64
evaluators (MUFU approximation refined by two Newton-Raphson steps) against
CUDA's own division and rsqrt and against correctly rounded references, over
positive normal doubles from 1e-300 to 1e300."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def ulps(a, b):
    """|a - b| in units of the last place of b."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_rcp64_and_rsqrt64_within_two_ulp(lens):
    rng = np.random.default_rng(3)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 20000), rng.uniform(0.5, 2.0, 20000),
                        [1.0, 2.0, 0.5, 3.0, 1e-300, 1e300, np.nextafter(1.0, 2.0), np.nextafter(2.0, 0.0)]])
    with lens.Context(0) as ctx:
        d = torch.tensor(x, device=DEV)
        out = torch.empty((4, x.size), dtype=torch.float64, device=DEV)
        ctx.selftest_math(d, out)
        ctx.wait()
        rcp, cuda_div, rs, cuda_rs = out.cpu().numpy()
    exact_rcp = 1.0 / x                                    # correctly rounded (IEEE division)
    assert np.all(ulps(cuda_div, exact_rcp) == 0)
    assert ulps(rcp, exact_rcp).max() <= 1.0
    # 1/sqrt(x) to ~0.5 ulp: the long-double quotient rounded once
    ref_rs = (np.longdouble(1) / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    assert ulps(rs, ref_rs).max() <= 2.0
    assert ulps(rs, cuda_rs).max() <= 2.0
