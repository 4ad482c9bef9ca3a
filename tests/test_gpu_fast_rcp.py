"""The double reciprocal of the FP64 arithmetic (srhd_reciprocal_f64: the
hardware approximation refined by two Newton-Raphson steps) against the IEEE
division on the same GPU: within one ulp over the whole normal range, and
exactly the IEEE result for zero, subnormal, huge and non-finite inputs."""
import ctypes

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _rcp(torch, x):
    from paper_2012_11130_gb300 import _native as N
    L = N.load()
    y = torch.empty_like(x)
    st = L.srhd_reciprocal_f64(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                               x.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == N.SRHD_OK, L.srhd_last_error()
    return y


def test_reciprocal_within_one_ulp_and_exact_specials():
    torch, _ = require_gpu()
    rng = np.random.default_rng(5)
    n = 1 << 20
    mag = 10.0 ** rng.uniform(-300, 300, n)
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    edge = []
    for e in range(-1000, 1020, 7):                  # powers of two and their neighbours
        v = 2.0 ** e
        edge += [v, np.nextafter(v, 0.0), np.nextafter(v, np.inf)]
    edge += [1.0 + k * 2.0 ** -52 for k in range(64)] + [2.0 - k * 2.0 ** -52 for k in range(64)]
    x = np.concatenate([mag * sgn, np.array(edge), -np.array(edge)])
    xd = torch.from_numpy(x).cuda()
    y = _rcp(torch, xd).cpu().numpy()
    ref = (1.0 / xd).cpu().numpy()                   # IEEE division on the device
    ulp = np.spacing(np.abs(ref))
    assert np.all(np.abs(y - ref) <= ulp), np.max(np.abs(y - ref) / ulp)
    # most results are the correctly rounded one
    assert np.mean(y == ref) > 0.9
    # special inputs take the IEEE division
    sp = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-310, 2.0 ** -1022, 2.0 ** 1021, 2.0 ** 1022,
                   1.7976931348623157e308, -2.0 ** 1023, np.inf, -np.inf, np.nan])
    sd = torch.from_numpy(sp).cuda()
    ys = _rcp(torch, sd).cpu().numpy()
    rs = (1.0 / sd).cpu().numpy()
    assert np.array_equal(ys.view(np.int64), rs.view(np.int64)), (ys, rs)


def test_reciprocal_arguments():
    torch, _ = require_gpu()
    from paper_2012_11130_gb300 import _native as N
    L = N.load()
    assert L.srhd_reciprocal_f64(None, None, 0, None) == N.SRHD_OK
    assert L.srhd_reciprocal_f64(None, None, -1, None) == N.SRHD_ERR_ARG
    assert L.srhd_reciprocal_f64(None, None, 5, None) == N.SRHD_ERR_ARG
