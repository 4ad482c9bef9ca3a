"""GPU test of srhd_cfl_dt_noalloc, the CFL entry point for callers that
cannot allocate device memory (an application whose device memory all comes
from its own pool, or a step loop that must not let an allocation
synchronise the device). It keeps its scratch in a static device array
instead of a context. It is checked through the C ABI, on two calls in a
row, against srhd_cfl_dt (which uses a context's scratch) and against the
oracle's CFL time step (Section 3.2), in every precision, for the
light-speed mode, the polytropic EoS, the total-energy scheme and a batch
with an unphysical cell (NaN).

This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import ctypes

import numpy as np
import pytest

from gpu_common import PRECS, require_gpu, to_dev, torch_dtype
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

MAX_PATCHES = 131072
TOL = {"fp64": 1e-12, "mixed": 1e-5, "mixed_cf": 1e-5}


def _noalloc_fn():
    from paper_2012_11130_gb300 import _native as N
    L = N.load()
    f = L.srhd_cfl_dt_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                  ctypes.POINTER(N.Params), ctypes.c_void_p, ctypes.c_void_p]
    return L, f


def _prec_code(prec):
    from paper_2012_11130_gb300 import _native as N
    return {"fp64": N.SRHD_FP64, "mixed": N.SRHD_MIXED, "mixed_cf": N.SRHD_MIXED_CF}[prec]


def _batch(oracle, npatch, seed, prec, scheme=0):
    """Interior patches [np][5][8^3] of well-conditioned cells (Lorentz
    factor <= 30, T >= 1e-4), in the storage type of the precision, and the
    same values in double for the oracle ([5][n])."""
    W = workloads.stress_batch_prims(npatch * 512, seed=seed, lg_gamma_range=(0, 1.5),
                                     T_range=(-4, 3))
    C, st = oracle.prim2con(W, scheme)
    assert np.all(st == 0)
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    return C, C.reshape(5, npatch, 512).transpose(1, 0, 2).copy()


def _call(fn, torch, prec, cons_dev, npatch, dh, params):
    from paper_2012_11130_gb300 import _native as N
    L = N.load()
    dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = fn(_prec_code(prec), ctypes.c_void_p(cons_dev.data_ptr()), npatch, dh,
            ctypes.byref(params), ctypes.c_void_p(dt.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
    assert st == N.SRHD_OK, L.srhd_last_error()
    torch.cuda.synchronize()
    return dt.item()


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_cfl_matches_cfl_dt_and_oracle(oracle, prec):
    torch, srhd = require_gpu()
    L, fn = _noalloc_fn()
    dtype = torch_dtype(torch, prec)
    params = srhd.Params().to_c()
    ctx = srhd.Context(srhd.Params())
    # two calls in a row on different batches, the second smaller: it must
    # not see the first call's per-patch results left in the static array
    for npatch, seed, dh in ((300, 41, 0.01), (57, 42, 0.003)):
        C, Cp = _batch(oracle, npatch, seed, prec)
        cons = to_dev(torch, Cp, dtype)
        got = _call(fn, torch, prec, cons, npatch, dh, params)
        want_lib = ctx.cfl_dt(cons, dh, prec=prec).item()
        want = oracle.cfl_dt(C, dh)
        assert np.isfinite(want) and abs(got / want - 1) <= TOL[prec], (got, want)
        assert abs(got / want_lib - 1) <= TOL[prec], (got, want_lib)


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_cfl_modes_eos_and_scheme(oracle, prec):
    torch, srhd = require_gpu()
    L, fn = _noalloc_fn()
    dtype = torch_dtype(torch, prec)
    npatch, dh = 40, 0.02
    C, Cp = _batch(oracle, npatch, 7, prec)
    cons = to_dev(torch, Cp, dtype)
    # light-speed mode (Section 3.2: the signal speed bounded by c)
    got = _call(fn, torch, prec, cons, npatch, dh, srhd.Params(cfl_mode="light").to_c())
    assert got == 0.5 * dh
    # the original (total-energy) scheme converts E instead of Etilde
    Ct, Ctp = _batch(oracle, npatch, 8, prec, scheme=1)
    got = _call(fn, torch, prec, to_dev(torch, Ctp, dtype), npatch, dh,
                srhd.Params(scheme="total").to_c())
    want = oracle.cfl_dt(Ct, dh, scheme=1)
    assert abs(got / want - 1) <= TOL[prec], (got, want)
    # polytropic EoS with Gamma = 4/3
    with oracle.eos(oracle.EOS_POLYTROPIC, 4.0 / 3.0):
        Cq, Cqp = _batch(oracle, npatch, 9, prec)
        want = oracle.cfl_dt(Cq, dh)
    got = _call(fn, torch, prec, to_dev(torch, Cqp, dtype), npatch, dh,
                srhd.Params(eos="polytropic", gamma=4.0 / 3.0).to_c())
    assert abs(got / want - 1) <= TOL[prec], (got, want)


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_unphysical_cell_gives_nan(oracle, prec):
    torch, srhd = require_gpu()
    L, fn = _noalloc_fn()
    dtype = torch_dtype(torch, prec)
    npatch, dh = 33, 0.01
    C, Cp = _batch(oracle, npatch, 11, prec)
    C[4, 20 * 512 + 77] = -1.0       # Etilde < 0: Eq. (Unphysical result) fails
    Cp = C.reshape(5, npatch, 512).transpose(1, 0, 2).copy()
    got = _call(fn, torch, prec, to_dev(torch, Cp, dtype), npatch, dh, srhd.Params().to_c())
    assert np.isnan(got) and np.isnan(oracle.cfl_dt(C, dh))
    # the next call, on a physical batch, is not affected by the flag left
    # in the static array
    C, Cp = _batch(oracle, npatch, 12, prec)
    got = _call(fn, torch, prec, to_dev(torch, Cp, dtype), npatch, dh, srhd.Params().to_c())
    assert abs(got / oracle.cfl_dt(C, dh) - 1) <= TOL[prec]


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
