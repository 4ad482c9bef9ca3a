"""Multi-step GPU runs against the oracle: the 1-D shock tube to t = 0.4
(compared with the exact TM solution), and the 3-D smooth advection
(per-cell parity, conservation, convergence), plus a sampled check of one
full-size 256^3 step in the launch configuration the benchmark times."""
import numpy as np
import pytest

from gpu_common import PRECS, cons_rel_err, require_gpu, to_dev, to_np, torch_dtype
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu


def _gpu_evolve(torch, srhd, ctx, C_patches, npx, npy, npz, bc, dh, t_end, prec,
                fixed_dt=None, max_steps=100000):
    """Ghost fill + fused step with the fused CFL, until t_end."""
    U = to_dev(torch, C_patches, torch_dtype(torch, prec))
    npatch = U.shape[0]
    dd = torch.empty((npatch, 2), dtype=torch.float64, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(npatch, dtype=torch.int32, device="cuda")
    out = torch.empty_like(U)
    if fixed_dt is None:
        dt = ctx.cfl_dt(U, dh, prec=prec).item()
    t, steps, retries = 0.0, 0, 0
    while t < t_end and steps < max_steps:
        if fixed_dt is not None:
            dt = fixed_dt
        if t + dt > t_end:
            dt = t_end - t
        dd[:, 0] = dt
        dd[:, 1] = dh
        G = ctx.fill_ghosts_uniform(U, npx, npy, npz, bc=bc)
        ctx.advance_patches(G, dd, cons_out=out, dt_next=dn, patch_status=st, prec=prec)
        U, out = out, U
        s = st.cpu().numpy()
        assert np.all((s >> 8) == 0), s[s != 0][:5]
        retries += int((s & 255).sum())
        t += dt
        steps += 1
        dt = dn.item()
    return U, steps, retries


@pytest.mark.parametrize("prec", PRECS)
def test_shock_tube_vs_exact_and_oracle(oracle, prec):
    # 1024 cells, (1, 0, 1e3) | (1, 0, 1e-2), t = 0.4, CFL 0.5 with the 1-D
    # signal-speed bound, outflow; the patch grid is 128 x 1 x 1 with
    # periodic (uniform) y and z.
    torch, srhd = require_gpu()
    N = 1024
    W, x = workloads.shock_tube_prims(N)
    C, _ = oracle.prim2con(W)
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    F = np.broadcast_to(C.reshape(5, 1, 1, N), (5, 8, 8, N)).copy()
    ctx = srhd.Context(srhd.Params(ndim=1))
    U, steps, retries = _gpu_evolve(torch, srhd, ctx, workloads.patchify(F), N // 8, 1, 1,
                                    ("outflow", "periodic", "periodic"), 1.0 / N, 0.4, prec)
    G = workloads.unpatchify(to_np(U), N // 8, 1, 1)
    # y/z-uniform: every row equals the first
    assert np.array_equal(G, np.broadcast_to(G[:, :1, :1, :], G.shape))
    Pg = oracle.con2pri(G[:, 0, 0, :])["prim"]
    ref = oracle.evolve(C.reshape(5, 1, 1, N), (1, 0, 0), 1.0 / N, 0.4, "outflow")
    Pr = oracle.con2pri(ref["cons"].reshape(5, -1))["prim"]
    rho, _, _, _ = oracle.exact_riemann((1, 0, 1e3), (1, 0, 1e-2), 0.5, 0.4, x)
    l1_gpu = np.mean(np.abs(1 - Pg[0] / rho))
    l1_ref = np.mean(np.abs(1 - Pr[0] / rho))
    assert abs(steps - ref["steps"]) <= 1
    # L1 error against the exact solution matches the oracle's to 2 digits
    assert abs(l1_gpu / l1_ref - 1) < 0.005, (l1_gpu, l1_ref)
    if prec == "fp64":
        assert np.max(np.abs(Pg[0] / Pr[0] - 1)) < 1e-6


@pytest.mark.parametrize("prec", PRECS)
def test_advection_steps_parity_and_conservation(oracle, prec):
    torch, srhd = require_gpu()
    N = 32
    Wf = workloads.advection_prims(N)
    C, _ = oracle.prim2con(Wf.reshape(5, -1))
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    C = C.reshape(5, N, N, N)
    dh = 1.0 / N
    dt = 0.45 * dh
    nsteps = 8
    ctx = srhd.Context(srhd.Params())
    U, steps, _ = _gpu_evolve(torch, srhd, ctx, workloads.patchify(C), 4, 4, 4, ("periodic",) * 3,
                              dh, nsteps * dt * (1 - 1e-12), prec, fixed_dt=dt)
    assert steps == nsteps
    G = workloads.unpatchify(to_np(U), 4, 4, 4)
    R = C.copy()
    for _ in range(nsteps):
        r = oracle.advance_block(oracle.fill_ghosts(R, (1, 1, 1), "periodic"), (N, N, N),
                                 (1, 1, 1), dt, dh)
        assert r["status"] == 0
        R = r["out"]
    err = cons_rel_err(G, R)
    # FP64: rounding only. Float storage: rounding the conserved state to
    # float perturbs the conversion by (1 + Mach^2) eps_float
    # (Eq. ImprovedRelativeError; Mach = |U| / U_s, U_s^2 = cs^2 / (1 - cs^2)),
    # once per step. Here gamma = 10 at T ~ 1 gives Mach^2 ~ 200.
    P0 = oracle.con2pri(C.reshape(5, -1))["prim"]
    cs2 = oracle.cs2_of_T(P0[4] / P0[0])
    mach2 = (P0[1] ** 2 + P0[2] ** 2 + P0[3] ** 2) * (1 - cs2) / cs2
    tol32 = nsteps * (1 + mach2.max()) * 2.0 ** -24
    assert err.max() <= (1e-11 if prec == "fp64" else tol32), (err.max(), tol32)
    tot0 = C.reshape(5, -1).sum(1)
    totg = G.reshape(5, -1).sum(1)
    scale = np.abs(G.reshape(5, -1)).sum(1)
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert np.all(np.abs(totg - tot0) <= tol * scale)


def test_advection_convergence_mixed_vs_fp64(oracle):
    # One period of the diagonal wave at 16^3 and 32^3: L1(rho) of Eq.
    # (relative L1 error) falls at about second order in both precisions and
    # the mixed L1 equals the FP64 L1 to two digits.
    torch, srhd = require_gpu()
    l1 = {}
    for prec in PRECS:
        for N in (16, 32):
            Wf = workloads.advection_prims(N)
            C, _ = oracle.prim2con(Wf.reshape(5, -1))
            v = float(np.sqrt(99.0 / 3.0) / np.sqrt(1.0 + 99.0))
            T_period = 1.0 / (3 * v)
            ctx = srhd.Context(srhd.Params())
            U, steps, _ = _gpu_evolve(torch, srhd, ctx, workloads.patchify(C.reshape(5, N, N, N)),
                                      N // 8, N // 8, N // 8, ("periodic",) * 3, 1.0 / N, T_period,
                                      prec)
            G = workloads.unpatchify(to_np(U), N // 8, N // 8, N // 8)
            rho = oracle.con2pri(G.reshape(5, -1))["prim"][0]
            exact = workloads.advection_prims(N, t=T_period)[0].reshape(-1)
            l1[prec, N] = np.mean(np.abs(1 - rho / exact))
    for prec in PRECS:
        assert np.log2(l1[prec, 16] / l1[prec, 32]) > 1.6, l1
    assert abs(l1["mixed", 32] / l1["fp64", 32] - 1) < 0.01, l1
    assert abs(l1["mixed_cf", 32] / l1["fp64", 32] - 1) < 0.01, l1


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_step_sampled(oracle, prec):
    # One step of the 256^3 smooth-advection batch (32768 patches) in the
    # configuration the benchmark times (fused CFL, status, one launch);
    # 24 sampled patches are recomputed by the oracle from the same inputs.
    torch, srhd = require_gpu()
    N = 256
    Wf = workloads.advection_prims(N)
    C, _ = oracle.prim2con(Wf.reshape(5, -1))
    C = C.reshape(5, N, N, N)
    if prec != "fp64":
        C = C.astype(np.float32)
    G = workloads.ghosted_patches(C)
    dtype = torch_dtype(torch, prec)
    npatch = G.shape[0]
    dh = 1.0 / N
    dd = torch.tensor([[0.4 * dh, dh]], dtype=torch.float64, device="cuda").repeat(npatch, 1)
    st = torch.empty(npatch, dtype=torch.int32, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    out = srhd.advance_patches(to_dev(torch, G, dtype), dd, dt_next=dn, patch_status=st, prec=prec)
    torch.cuda.synchronize()
    assert int(st.abs().max()) == 0
    rng = np.random.default_rng(11)
    pick = np.concatenate([[0, npatch - 1], rng.choice(npatch, 22, replace=False)])
    ref = oracle.advance_patches(G[pick].astype(np.float64), np.tile([0.4 * dh, dh], (pick.size, 1)))
    o = to_np(out[torch.as_tensor(pick, device="cuda")])
    err = cons_rel_err(o.transpose(1, 0, 2, 3, 4), ref["out"].transpose(1, 0, 2, 3, 4))
    assert err.max() <= (1e-12 if prec == "fp64" else 1e-5), err.max()
    assert np.isfinite(dn.item()) and dn.item() > 0


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_uniform_steps_sampled(oracle, prec):
    # The two 256^3 time-loop steps the benchmark also times, in their
    # launch configuration: srhd_advance_uniform (tiles gathered from the
    # neighbouring patches, staged slabs) and srhd_advance_uniform_prim (the
    # tiles' primitives from a cache seeded by srhd_con2pri_patches). Two
    # consecutive steps each, so the second cached step reads the cache the
    # first one wrote; 24 sampled patches of both steps are recomputed by
    # the oracle from the ghosted tiles of the same inputs.
    torch, srhd = require_gpu()
    N = 256
    Wf = workloads.advection_prims(N)
    C, _ = oracle.prim2con(Wf.reshape(5, -1))
    C = C.reshape(5, N, N, N)
    if prec != "fp64":
        C = C.astype(np.float32)
    G = workloads.ghosted_patches(C)
    npatch, npx = G.shape[0], N // 8
    dtype = torch_dtype(torch, prec)
    dh = 1.0 / N
    dd = torch.tensor([[0.4 * dh, dh]], dtype=torch.float64, device="cuda").repeat(npatch, 1)
    U0 = to_dev(torch, np.ascontiguousarray(G[:, :, 2:10, 2:10, 2:10]), dtype)
    rng = np.random.default_rng(12)
    pick = np.concatenate([[0, npx - 1, npatch - 1], rng.choice(npatch, 21, replace=False)])

    def tiles(field):
        # the periodic 12^3 tiles of the picked patches of field [5][N][N][N]
        out = []
        for q in pick:
            ix, iy, iz = q % npx, (q // npx) % npx, q // (npx * npx)
            zi, yi, xi = ((np.arange(-2, 10) + 8 * c) % N for c in (iz, iy, ix))
            out.append(field[:, zi][:, :, yi][:, :, :, xi])
        return np.stack(out)

    assert np.array_equal(tiles(C), G[pick])
    del G
    tol = 1e-12 if prec == "fp64" else 1e-5
    ctx = srhd.Context()
    results = {}
    for cached in (False, True):
        st = torch.empty(npatch, dtype=torch.int32, device="cuda")
        dn = torch.empty(1, dtype=torch.float64, device="cuda")
        U = U0
        P = ctx.con2pri_patches(U, prec=prec) if cached else None
        states = [to_np(U[torch.as_tensor(pick, device="cuda")])]
        for _ in range(2):
            if cached:
                V, P = ctx.advance_uniform_prim(U, P, npx, npx, npx, dd, dt_next=dn,
                                                patch_status=st, prec=prec)
            else:
                V = ctx.advance_uniform(U, npx, npx, npx, dd, dt_next=dn, patch_status=st,
                                        prec=prec)
            torch.cuda.synchronize()
            assert int(st.abs().max()) == 0
            assert np.isfinite(dn.item()) and dn.item() > 0
            if cached:
                # the cache written for the new state is its conversion
                Pn = to_np(P[torch.as_tensor(pick, device="cuda")]).astype(np.float64)
                Vn = to_np(V[torch.as_tensor(pick, device="cuda")]).astype(np.float64)
                ref = oracle.con2pri(Vn.transpose(1, 0, 2, 3, 4).reshape(5, -1))["prim"]
                got = Pn.transpose(1, 0, 2, 3, 4).reshape(6, -1)[:5]
                assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) <= 10 * tol
            # the sampled patches of the new state against the oracle's step
            # of their ghosted tiles (from the state this step read)
            Gs = tiles(workloads.unpatchify(to_np(U), npx, npx, npx))
            ref = oracle.advance_patches(Gs.astype(np.float64), np.tile([0.4 * dh, dh], (pick.size, 1)))
            o = to_np(V[torch.as_tensor(pick, device="cuda")])
            err = cons_rel_err(o.transpose(1, 0, 2, 3, 4), ref["out"].transpose(1, 0, 2, 3, 4))
            assert err.max() <= tol, (cached, err.max())
            states.append(o)
            U = V
        results[cached] = states
    # cached and uncached loops agree with each other as well
    for a, b in zip(results[False], results[True]):
        err = cons_rel_err(a.transpose(1, 0, 2, 3, 4), b.transpose(1, 0, 2, 3, 4))
        assert err.max() <= 2 * tol
