"""The float64 collide's 1/rho on the GPU (lbm_probe_rcp) against its error
bound: within one unit in the last place of the exact reciprocal for x in
[2^-125, 2^126), NaN outside (zero, subnormals, infinities, NaN).  The CPU
test test_rcp_newton.py pins the same steps word by word with a modelled
seed; this one runs the device's own float32 reciprocal approximation.
Exact reference: Python's Fraction (int / int division is correctly rounded).
"""
import ctypes
import math
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def device_rcp(x):
    from paper_1703_00186_gb300 import _lib as L
    lib = L.load()
    xd = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.empty_like(xd)
    stream = torch.cuda.current_stream()
    rc = lib.lbm_probe_rcp(ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(xd.data_ptr()),
                           ctypes.c_void_p(yd.data_ptr()), xd.numel())
    assert rc == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_reciprocal_within_one_ulp():
    rng = np.random.default_rng(11)
    x = np.concatenate([np.exp2(rng.uniform(-125, 126, 4000)) * rng.choice([-1.0, 1.0], 4000),
                        rng.uniform(0.05, 20.0, 4000),               # densities of the workloads
                        [1.0, 1.25, 3.0, 0.1, 2.0 ** -125, math.nextafter(2.0 ** 126, 0.0)]])
    y = device_rcp(x)
    worst = 0.0
    for xi, yi in zip(x.tolist(), y.tolist()):
        exact = 1 / Fraction(xi)
        err = abs(Fraction(yi) - exact) / Fraction(math.ulp(float(abs(exact))))
        worst = max(worst, float(err))
        assert err <= 1, (xi, yi, float(err))
    assert worst > 0.3


def test_reciprocal_out_of_range_is_nan():
    x = np.array([0.0, -0.0, 5e-324, 2.0 ** -126, 2.0 ** -1000, 2.0 ** 126, 1e300, np.inf, -np.inf, np.nan])
    assert np.isnan(device_rcp(x)).all()


def test_reciprocal_refuses_bad_arguments_before_any_launch():
    from paper_1703_00186_gb300 import _lib as L
    lib = L.load()
    assert lib.lbm_probe_rcp(None, None, None, 0) == 0
    assert lib.lbm_probe_rcp(None, None, None, -1) == L.LBM_ERR_INVALID
    assert lib.lbm_probe_rcp(None, None, None, 5) == L.LBM_ERR_INVALID
