"""GPU test of srhd_cfl_dt_noalloc, the CFL entry point for callers that
cannot allocate device memory (an application whose device memory all comes
from its own pool, or a step loop that must not let an allocation
synchronise the device). It keeps its scratch in a static device array
instead of a context, so it is checked here against srhd_cfl_dt, which
uses a context's scratch, on two calls in a row through the C ABI.

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import ctypes

import numpy as np
import pytest

from gpu_common import require_gpu, to_dev
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

MAX_PATCHES = 131072


def _noalloc_fn():
    from paper_2012_11130_gb300 import _native as N
    L = N.load()
    f = L.srhd_cfl_dt_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                  ctypes.POINTER(N.Params), ctypes.c_void_p, ctypes.c_void_p]
    return L, f


def _batch(oracle, npatch, seed, dtype, torch):
    W = workloads.stress_batch_prims(npatch * 512, seed=seed, lg_gamma_range=(0, 1.5),
                                     T_range=(-4, 3))
    C, _ = oracle.prim2con(W)
    Cp = C.reshape(5, npatch, 512).transpose(1, 0, 2).copy()
    return to_dev(torch, Cp, dtype)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_cfl_matches_cfl_dt(oracle, prec):
    torch, srhd = require_gpu()
    from paper_2012_11130_gb300 import _native as N
    L, fn = _noalloc_fn()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    code = N.SRHD_FP64 if prec == "fp64" else N.SRHD_MIXED
    tol = 1e-12 if prec == "fp64" else 1e-5
    params = N.Params()
    L.srhd_default_params(ctypes.byref(params))
    ctx = srhd.Context(srhd.Params())
    stream = torch.cuda.current_stream()
    # two calls in a row on different batches: the second must not see the
    # first call's per-patch results left in the shared static array
    for npatch, seed, dh in ((300, 41, 0.01), (57, 42, 0.003)):
        cons = _batch(oracle, npatch, seed, dtype, torch)
        want = ctx.cfl_dt(cons, dh).item()
        dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st = fn(code, ctypes.c_void_p(cons.data_ptr()), npatch, dh, ctypes.byref(params),
                ctypes.c_void_p(dt.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == N.SRHD_OK, L.srhd_last_error()
        torch.cuda.synchronize()
        got = dt.item()
        assert np.isfinite(want) and abs(got / want - 1) <= tol, (got, want)


def test_noalloc_limits_and_empty_batch():
    torch, srhd = require_gpu()
    from paper_2012_11130_gb300 import _native as N
    L, fn = _noalloc_fn()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = fn(N.SRHD_FP64, ctypes.c_void_p(dummy.data_ptr()), MAX_PATCHES + 1, 0.1, None,
            ctypes.c_void_p(dt.data_ptr()), None)
    assert st == N.SRHD_ERR_ARG
    assert b"131072" in L.srhd_last_error()
    st = fn(N.SRHD_FP64, None, 0, 0.1, None, ctypes.c_void_p(dt.data_ptr()), None)
    assert st == N.SRHD_OK
    torch.cuda.synchronize()
    assert dt.item() == float("inf")
