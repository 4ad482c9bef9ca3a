"""GPU parity of the batched conversions (srhd_prim2con, srhd_con2pri)
against the oracle on the con2pri stress batch (rho 1e-6..1e2, T 1e-8..1e4,
gamma 1..1e6, random direction), through the C ABI."""
import numpy as np
import pytest

from gpu_common import (BASE, EPS64, EPS_A, PRECS, kappa_of_prims, prim_rel_err, require_gpu,
                        to_dev, to_np, torch_dtype)
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu


def _inputs(oracle, n, seed, prec):
    W = workloads.stress_batch_prims(n, seed=seed)
    C, st = oracle.prim2con(W)
    assert np.all(st == 0)
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    return W, C


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [1, 997, 3 * 65536 + 37])
def test_con2pri_parity(oracle, prec, n):
    torch, srhd = require_gpu()
    dtype = torch_dtype(torch, prec)
    W, C = _inputs(oracle, n, 1000 + n, prec)
    ref = oracle.con2pri(C)
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    P = srhd.con2pri(to_dev(torch, C, dtype), cell_status=st, prec=prec)
    torch.cuda.synchronize()
    Pg, stg = to_np(P), st.cpu().numpy()
    assert set(np.unique(stg)) <= {0, 1}
    # conditioning of the state the input actually encodes (in the mixed
    # path the float rounding of Etilde can move a cold, fast cell far from
    # the drawn state), from the oracle's inversion of the same input
    with np.errstate(invalid="ignore"):
        kappa = np.where(ref["status"] == 0, kappa_of_prims(oracle, np.nan_to_num(ref["prim"], nan=1.0)),
                         np.inf)
    clear = kappa * EPS_A[prec] <= 1e-3
    # well-conditioned cells: same status, values within the tolerance
    assert np.array_equal(stg[clear], ref["status"][clear])
    ok = clear & (ref["status"] == 0)
    tol = np.maximum(BASE[prec], 10 * kappa * EPS_A[prec])
    err = prim_rel_err(Pg, ref["prim"])
    bad = ok & ~(err <= tol)
    assert not bad.any(), (np.nonzero(bad)[0][:5], err[bad][:5], tol[bad][:5])
    # unphysical cells are NaN, accepted cells are finite everywhere
    assert np.all(np.isnan(Pg[:, stg == 1]))
    assert np.all(np.isfinite(Pg[:, stg == 0]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_prim2con_parity(oracle, prec):
    torch, srhd = require_gpu()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    n = 65536 + 129
    W = workloads.stress_batch_prims(n, seed=77)
    if prec == "mixed":
        W = W.astype(np.float32).astype(np.float64)
    ref, _ = oracle.prim2con(W)
    C = to_np(srhd.prim2con(to_dev(torch, W, dtype)))
    tol = 1e-13 if prec == "fp64" else 1e-5
    rel = np.abs(C - ref) / np.maximum(np.abs(ref), np.sqrt((ref[1:4] ** 2).sum(0)))
    assert rel.max() <= tol, rel.max()


def test_conversion_edge_cases(oracle):
    torch, srhd = require_gpu()
    ctx = srhd.default_context()
    # n = 0 is a no-op
    empty = torch.empty((5, 0), dtype=torch.float64, device="cuda")
    ctx.con2pri(empty)
    ctx.prim2con(empty)
    # unphysical conserved states: D <= 0, |M| too large, Etilde <= 0
    C = np.array([[-1.0, 1.0, 1.0, 0.0],
                  [0.0, 5.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0],
                  [1.0, 1.0, -1.0, 0.0]])
    for prec in PRECS:
        st = torch.empty(4, dtype=torch.int32, device="cuda")
        P = ctx.con2pri(to_dev(torch, C, torch_dtype(torch, prec)), cell_status=st, prec=prec)
        assert st.cpu().tolist() == [1, 1, 1, 1]
        assert torch.isnan(P).all()
    ref = oracle.con2pri(C)
    assert ref["status"].tolist() == [1, 1, 1, 1]


def test_round_trip_tracks_conditioning(oracle):
    # Appendix B on the GPU (FP64): T = 1e-8, Mach 1e-4..1e6 along x=y=z;
    # the htilde error stays within a small multiple of (1+Mach^2) eps.
    torch, srhd = require_gpu()
    T = 1e-8
    cs2 = oracle.cs2_of_T(T)
    Us = np.sqrt(cs2 / (1 - cs2))
    mach = np.logspace(-4, 6, 201)
    n = mach.size
    W = np.vstack([np.ones(n), np.tile(mach * Us / np.sqrt(3), (3, 1)), np.full(n, T)])
    Wd = to_dev(torch, W, torch.float64)
    P = to_np(srhd.con2pri(srhd.prim2con(Wd)))
    ht0 = oracle.htilde_of_T(T)
    ht2 = oracle.htilde_of_T(P[4] / P[0])
    err = np.abs(1 - ht0 / ht2)
    assert np.all(err <= 64 * (1 + mach ** 2) * EPS64)


def test_mixed_conversion_at_large_density(oracle):
    # SRHD_MIXED forms A D^2 in double from the state scaled by the power of
    # two that brings D into [1, 2), then scales it back in float: densities
    # whose A D^2 (up to ~1e45 here) or 1/D^2 leave the float range must
    # convert like the oracle.
    torch, srhd = require_gpu()
    rng = np.random.default_rng(19)
    n = 4096
    rho = 10.0 ** rng.uniform(16.0, 20.0, n)          # D = rho gamma from 1e16 to ~1e21
    T = 10.0 ** rng.uniform(-3.0, 2.0, n)
    gam = 10.0 ** rng.uniform(0.0, 1.0, n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    U = np.sqrt(gam * gam - 1.0) * d
    W = np.vstack([rho, U, rho * T])
    C, st = oracle.prim2con(W)
    assert np.all(st == 0)
    C = C.astype(np.float32).astype(np.float64)
    assert (C[0] >= 1e19).mean() > 0.2
    ref = oracle.con2pri(C)
    st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    P = srhd.con2pri(to_dev(torch, C, torch.float32), cell_status=st, prec="mixed")
    torch.cuda.synchronize()
    Pg, stg = to_np(P), st.cpu().numpy()
    ok = ref["status"] == 0
    assert np.array_equal(stg, ref["status"])
    kappa = kappa_of_prims(oracle, ref["prim"][:, ok])
    tol = np.maximum(BASE["mixed"], 10 * kappa * EPS_A["mixed"])
    err = prim_rel_err(Pg[:, ok], ref["prim"][:, ok])
    assert np.all(err <= tol), err.max()
