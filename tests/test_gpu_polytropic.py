"""GPU parity of the polytropic-EoS path (srhd_params.eos =
SRHD_EOS_POLYTROPIC, Section 2.2) against the oracle run with the same EoS,
through the C ABI: conversions on the stress batch, one fused step of
smooth patches (HLLC and the HLLE-only path), the CFL bound (context and
no-allocation entry points), and a shock tube against the exact polytropic
solution."""
import numpy as np
import pytest

from gpu_common import (BASE, EPS_A, cons_rel_err, kappa_of_prims, prim_rel_err, require_gpu,
                        to_dev, to_np, torch_dtype)
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

GAMMAS = (5.0 / 3.0, 4.0 / 3.0)


def _ctx(srhd, g, **kw):
    return srhd.Context(srhd.Params(eos="polytropic", gamma=g, **kw))


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
@pytest.mark.parametrize("g", GAMMAS)
def test_conversions_parity(oracle, prec, g):
    torch, srhd = require_gpu()
    dtype = torch_dtype(torch, prec)
    n = 65536 + 77
    W = workloads.stress_batch_prims(n, seed=91)
    with oracle.eos(oracle.EOS_POLYTROPIC, g):
        C, st = oracle.prim2con(W)
        assert np.all(st == 0)
        if prec != "fp64":
            C = C.astype(np.float32).astype(np.float64)
        ref = oracle.con2pri(C)
        with np.errstate(invalid="ignore"):
            kappa = np.where(ref["status"] == 0,
                             kappa_of_prims(oracle, np.nan_to_num(ref["prim"], nan=1.0)), np.inf)
        Cref, _ = oracle.prim2con(W)
    ctx = _ctx(srhd, g)
    stg = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    P = to_np(ctx.con2pri(to_dev(torch, C, dtype), cell_status=stg, prec=prec))
    s = stg.cpu().numpy()
    clear = kappa * EPS_A[prec] <= 1e-3
    assert np.array_equal(s[clear], ref["status"][clear])
    ok = clear & (ref["status"] == 0)
    # With T = k htilde (k = (Gamma-1)/Gamma) the oracle's f of
    # Eq. (transcendental equation) sums terms (1 + 2k) htilde^2 to a value
    # (1 - 2k) htilde^2 when m >> h, so its rounding is amplified by
    # (1 + 2k)/(1 - 2k) (9 for Gamma = 5/3, 3 for 4/3) on top of kappa eps.
    k = (g - 1) / g
    amp = (1 + 2 * k) / (1 - 2 * k)
    tol = np.maximum(BASE[prec], 10 * amp * kappa * EPS_A[prec])
    err = prim_rel_err(P, ref["prim"])
    assert not (ok & ~(err <= tol)).any(), err[ok & ~(err <= tol)][:5]
    # prim -> cons
    Wd = to_dev(torch, W, dtype)
    Cg = to_np(ctx.prim2con(Wd, prec=prec))
    Wr = to_np(Wd)
    with oracle.eos(oracle.EOS_POLYTROPIC, g):
        Cr, _ = oracle.prim2con(Wr)
    rel = np.abs(Cg - Cr) / np.maximum(np.abs(Cr), np.sqrt((Cr[1:4] ** 2).sum(0)))
    assert rel.max() <= (1e-13 if prec == "fp64" else 2e-6), rel.max()


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
@pytest.mark.parametrize("riemann", ["hllc", "hlle"])
def test_patch_step_parity(oracle, prec, riemann):
    torch, srhd = require_gpu()
    npatch = 211
    Wp = workloads.smooth_patch_prims(npatch, seed=8)
    dt_dh = np.tile([0.025, 1 / 12], (npatch, 1))
    for g in GAMMAS:
        with oracle.eos(oracle.EOS_POLYTROPIC, g):
            C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
            assert np.all(st == 0)
            C = C.reshape(5, npatch, 12, 12, 12).transpose(1, 0, 2, 3, 4).copy()
            if prec != "fp64":
                C = C.astype(np.float32).astype(np.float64)
            ref = oracle.advance_patches(C, dt_dh, riemann=0 if riemann == "hllc" else 1)
            dtn_ref = oracle.cfl_dt(ref["out"].transpose(1, 0, 2, 3, 4).reshape(5, -1), 1 / 12)
        ctx = _ctx(srhd, g, riemann=riemann)
        dt = torch_dtype(torch, prec)
        stg = torch.full((npatch,), -1, dtype=torch.int32, device="cuda")
        dn = torch.empty(1, dtype=torch.float64, device="cuda")
        out = ctx.advance_patches(to_dev(torch, C, dt), to_dev(torch, dt_dh, torch.float64),
                                  dt_next=dn, patch_status=stg, prec=prec)
        assert np.all(ref["status"] == 0) and int(stg.abs().max()) == 0
        err = cons_rel_err(to_np(out).transpose(1, 0, 2, 3, 4),
                           ref["out"].transpose(1, 0, 2, 3, 4))
        assert err.max() <= (1e-12 if prec == "fp64" else 1e-5), (g, err.max())
        assert abs(dn.item() / dtn_ref - 1) <= (1e-12 if prec == "fp64" else 1e-5)
        # the context-free CFL entry point with the same parameters
        dn2 = torch.empty(1, dtype=torch.float64, device="cuda")
        srhd.cfl_dt_noalloc(out, 1 / 12, dn2, params=srhd.Params(eos="polytropic", gamma=g),
                            prec=prec)
        assert abs(dn2.item() / dtn_ref - 1) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
def test_polytropic_shock_tube_matches_oracle_l1(oracle, prec):
    # mildly relativistic shock tube (rho, v, p) = (1, 0, 1) | (0.125, 0, 0.1),
    # Gamma = 4/3, 512 cells, t = 0.4, CFL 0.5, outflow: the GPU's L1 error
    # against the exact polytropic solution equals the oracle's to 0.5 %
    torch, srhd = require_gpu()
    from test_gpu_runs import _gpu_evolve
    g, N = 4.0 / 3.0, 512
    x = (np.arange(N) + 0.5) / N
    W = np.vstack([np.where(x < 0.5, 1.0, 0.125), 0 * x, 0 * x, 0 * x,
                   np.where(x < 0.5, 1.0, 0.1)])
    with oracle.eos(oracle.EOS_POLYTROPIC, g):
        C, _ = oracle.prim2con(W)
        if prec != "fp64":
            C = C.astype(np.float32).astype(np.float64)
        ref = oracle.evolve(C.reshape(5, 1, 1, N), (1, 0, 0), 1.0 / N, 0.4, "outflow")
        Pr = oracle.con2pri(ref["cons"].reshape(5, -1))["prim"]
        rho_ex, _, _, _ = oracle.exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, 0.4, x)
    F = np.broadcast_to(C.reshape(5, 1, 1, N), (5, 8, 8, N)).copy()
    ctx = _ctx(srhd, g, ndim=1)
    U, steps, _ = _gpu_evolve(torch, srhd, ctx, workloads.patchify(F), N // 8, 1, 1,
                              ("outflow", "periodic", "periodic"), 1.0 / N, 0.4, prec)
    G = workloads.unpatchify(to_np(U), N // 8, 1, 1)[:, 0, 0, :]
    with oracle.eos(oracle.EOS_POLYTROPIC, g):
        Pg = oracle.con2pri(G)["prim"]
    l1_gpu = np.mean(np.abs(1 - Pg[0] / rho_ex))
    l1_ref = np.mean(np.abs(1 - Pr[0] / rho_ex))
    assert abs(steps - ref["steps"]) <= 1
    assert abs(l1_gpu / l1_ref - 1) < 0.005, (l1_gpu, l1_ref)


def test_invalid_gamma_is_refused():
    torch, srhd = require_gpu()
    for g in (1.0, 2.0):
        with pytest.raises(Exception, match="gamma"):
            _ctx(srhd, g)
