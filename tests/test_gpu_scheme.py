"""The paper's comparison of energy formulations on the GPU: the original
scheme (total energy E with flux M, SRHD_SCHEME_TOTAL) against the oracle's
original scheme, and the cold sound wave of Section 4.1, where the reduced
energy converges and the total energy stalls (FP64) or cannot even
represent the gas (float storage)."""
import numpy as np
import pytest

from gpu_common import cons_rel_err, prim_rel_err, require_gpu, to_dev, to_np, torch_dtype
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
def test_total_energy_scheme_parity(oracle, prec):
    torch, srhd = require_gpu()
    npatch = 97
    Wp = workloads.smooth_patch_prims(npatch, seed=31)
    C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1), oracle.ORIGINAL)
    assert np.all(st == 0)
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    ctx = srhd.Context(srhd.Params(scheme="total"))
    dtype = torch_dtype(torch, prec)
    # conversions
    P = to_np(ctx.con2pri(to_dev(torch, C, dtype), prec=prec))
    ref = oracle.con2pri(C, oracle.ORIGINAL)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.all(ref["status"] == 0)
    assert prim_rel_err(P, ref["prim"]).max() <= tol
    Wd = to_dev(torch, Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1), dtype)
    Cg = to_np(ctx.prim2con(Wd, prec=prec))
    Cr, _ = oracle.prim2con(to_np(Wd), oracle.ORIGINAL)
    assert cons_rel_err(Cg, Cr).max() <= (1e-13 if prec == "fp64" else 1e-6)
    # one fused step of ghosted patches
    G = C.reshape(5, npatch, 12, 12, 12).transpose(1, 0, 2, 3, 4).copy()
    dt_dh = np.tile([0.02, 1 / 12], (npatch, 1))
    refp = oracle.advance_patches(G, dt_dh, scheme=oracle.ORIGINAL)
    st = torch.full((npatch,), -1, dtype=torch.int32, device="cuda")
    out = to_np(ctx.advance_patches(to_dev(torch, G, dtype), to_dev(torch, dt_dh, torch.float64),
                                    patch_status=st, prec=prec))
    assert np.all(refp["status"] == 0) and int(st.abs().max()) == 0
    err = cons_rel_err(out.transpose(1, 0, 2, 3, 4), refp["out"].transpose(1, 0, 2, 3, 4))
    assert err.max() <= tol, err.max()


def _sound_wave_gpu(torch, srhd, oracle, N, scheme, prec, T0=1e-10, amp=1e-6):
    cs = np.sqrt(oracle.cs2_of_T(T0))
    x = (np.arange(N) + 0.5) / N
    s = np.sin(2 * np.pi * x)
    rho = 1 + amp * s
    W = np.vstack([rho, cs * amp * s, 0 * x, 0 * x, T0 * (1 + 5 / 3 * amp * s)])
    C, _ = oracle.prim2con(W, oracle.NEW if scheme == "reduced" else oracle.ORIGINAL)
    F = np.broadcast_to(C.reshape(5, 1, 1, N), (5, 8, 8, N)).copy()
    ctx = srhd.Context(srhd.Params(ndim=1, scheme=scheme))
    U = to_dev(torch, workloads.patchify(F), torch_dtype(torch, prec))
    npx = N // 8
    dh = 1.0 / N
    t_end = 1.0 / cs
    dd = torch.empty((npx, 2), dtype=torch.float64, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(npx, dtype=torch.int32, device="cuda")
    out = torch.empty_like(U)
    dt = ctx.cfl_dt(U, dh, prec=prec).item()
    if not np.isfinite(dt):
        return None  # the stored state is already unphysical
    t = 0.0
    while t < t_end:
        dt = min(dt, t_end - t)
        dd[:, 0] = dt
        dd[:, 1] = dh
        G = ctx.fill_ghosts_uniform(U, npx, 1, 1, bc=("periodic",) * 3)
        ctx.advance_patches(G, dd, cons_out=out, dt_next=dn, patch_status=st, prec=prec)
        U, out = out, U
        assert int(st.abs().max()) == 0
        t += dt
        dt = dn.item()
    G = workloads.unpatchify(to_np(U), npx, 1, 1)[:, 0, 0, :]
    P = oracle.con2pri(G, oracle.NEW if scheme == "reduced" else oracle.ORIGINAL)["prim"]
    return float(np.mean(np.abs(1 - P[0] / rho)))


def test_cold_sound_wave_reduced_vs_total_energy(oracle):
    # Section 4.1 on the GPU (T = 1e-10, delta rho / rho = 1e-6, one period):
    # FP64 reduced energy converges at second order, FP64 total energy
    # stalls near 2e-6; with float storage the reduced energy stays at the
    # float resolution of the 1e-6 wave (below the FP64 total-energy
    # plateau) while E = D (1 + 1.5e-10) rounds to D and the total-energy
    # state is unphysical from the start.
    torch, srhd = require_gpu()
    red = [_sound_wave_gpu(torch, srhd, oracle, N, "reduced", "fp64") for N in (32, 64)]
    tot = [_sound_wave_gpu(torch, srhd, oracle, N, "total", "fp64") for N in (32, 64)]
    assert np.log2(red[0] / red[1]) > 1.7, red
    assert all(1e-6 < e < 1e-5 for e in tot), tot
    red32 = _sound_wave_gpu(torch, srhd, oracle, 64, "reduced", "mixed_cf")
    assert red32 is not None and red32 < 1e-6 and red32 < tot[1] / 3, (red32, tot)
    assert _sound_wave_gpu(torch, srhd, oracle, 64, "total", "mixed_cf") is None


def _riemann_gpu(torch, srhd, C, n, scheme, prec, t_end):
    """A 1-D Riemann problem on [0, 1] on the GPU as a row of n/8 patches
    (periodic y, z; outflow x), the fused 1-D CFL bound setting each step."""
    ctx = srhd.Context(srhd.Params(ndim=1, scheme=scheme))
    npx = n // 8
    F = np.broadcast_to(C.reshape(5, 1, 1, n), (5, 8, 8, n)).copy()
    U = to_dev(torch, workloads.patchify(F), torch_dtype(torch, prec))
    V = torch.empty_like(U)
    dd = torch.empty((npx, 2), dtype=torch.float64, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(npx, dtype=torch.int32, device="cuda")
    dh = 1.0 / n
    dt = ctx.cfl_dt(U, dh, prec=prec).item()
    t, steps, worst = 0.0, 0, 0
    while t < t_end:
        dt = min(dt, t_end - t)
        dd[:, 0] = dt
        dd[:, 1] = dh
        ctx.advance_uniform(U, npx, 1, 1, dd, bc=("outflow", "periodic", "periodic"), cons_out=V,
                            dt_next=dn, patch_status=st, prec=prec)
        worst = max(worst, int((st >> 8).max()))
        U, V = V, U
        t += dt
        steps += 1
        dt = dn.item()
    G = workloads.unpatchify(to_np(U), npx, 1, 1)
    assert np.array_equal(G, np.broadcast_to(G[:, :1, :1, :], G.shape))
    return G[:, 0, 0, :].astype(np.float64), steps, worst


def _riemann_oracle(oracle, C, n, t_end, scheme=None):
    """The oracle's run of the same problem with the GPU's retry granularity:
    one 8-cell block per patch (a patch of the GPU's row is uniform in y and
    z, so its y and z flux differences vanish and it fails or passes with
    its 8-cell row), each block retried on its own (oracle.evolve retries
    the whole domain at once)."""
    scheme = oracle.NEW if scheme is None else scheme
    dh = 1.0 / n
    cons, t, steps = C.copy(), 0.0, 0
    while t < t_end:
        dt = min(oracle.cfl_dt(cons, dh, cfl=0.5, ndim=1, scheme=scheme), t_end - t)
        G = oracle.fill_ghosts(cons.reshape(5, 1, 1, n), (1, 0, 0), "outflow")
        out = np.empty_like(cons)
        for b in range(n // 8):
            r = oracle.advance_block(G[:, :, :, 8 * b:8 * b + 12], (8, 1, 1), (1, 0, 0), dt, dh,
                                     scheme=scheme)
            assert r["status"] in (oracle.BLK_OK, oracle.BLK_NOCONV)
            out[:, 8 * b:8 * b + 8] = r["out"].reshape(5, 8)
        cons, t, steps = out, t + dt, steps + 1
    return cons, steps


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
def test_mixed_limits_riemann_problem(oracle, prec):
    # The initial states of Section 4.2.2 (Table "tb:IC_RiemannProblems",
    # second row: a cold left state, T = 1e-6, against an ultra-relativistic
    # right-moving stream), shortened to [0, 1] with 1024 cells (the
    # paper's cell size) and t = 0.4 so that the oracle runs it too. With the
    # reduced energy the GPU's errors against the exact solution match the
    # oracle's and the cold state keeps its pressure; with the
    # total energy in float storage the cold state's pressure is off by about
    # a per cent from the first step (E = D h gamma - p stores the thermal
    # energy, 1.5e-6 of E, at float resolution: the error of the paper's
    # Eq. (error in the NR limit) that makes its original-scheme run of this
    # problem 23 % wrong near the rarefaction). The density jumps by 4e10
    # across the contact, so a domain-wide relative L1 would measure only
    # the few smeared contact cells; the comparison is made on the shocked
    # right plateau (rho, p against the exact solution), the shock position
    # and the cold state.
    torch, srhd = require_gpu()
    n, x0, t_end = 1024, 0.05, 0.4
    x = (np.arange(n) + 0.5) / n
    left = x < x0
    W = np.zeros((5, n))
    W[0] = np.where(left, 1e2, 1e-12)
    W[1] = np.where(left, 1e-3, -1e2)
    W[4] = np.where(left, 1e-4, 1e-10)
    rho_ex, _, p_ex, info = oracle.exact_riemann((1e2, 1e-3, 1e-4), (1e-12, -1e2, 1e-10), x0,
                                                 t_end, x)
    us = info["Ushock_R"]
    x_shock = x0 + t_end * us / np.sqrt(1 + us * us)
    cold = x < 0.04  # the undisturbed left state at t = 0.4
    plateau = (x > 0.07) & (x < x_shock - 0.02)

    def plateau_err(P):
        return (np.mean(np.abs(P[0][plateau] / rho_ex[plateau] - 1)),
                np.mean(np.abs(P[4][plateau] / p_ex[plateau] - 1)))

    def shock_cell(P):  # first cell past half the jump to the right state
        return int(np.argmax((x > 0.1) & (P[0] < 0.5 * (info["rho_CR"] + 1e-12))))
    C, _ = oracle.prim2con(W, oracle.NEW)
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    G, steps, worst = _riemann_gpu(torch, srhd, C, n, "reduced", prec, t_end)
    assert worst == 0
    Pg = oracle.con2pri(G, oracle.NEW)["prim"]
    ref, ref_steps = _riemann_oracle(oracle, C, n, t_end)
    Pr = oracle.con2pri(ref, oracle.NEW)["prim"]
    assert abs(steps - ref_steps) <= 1
    # the plateau errors (about 2e-3, set by the shock's start-up) match the
    # oracle's to 10 %, the shock lies in the same cell (+-1)
    eg, er = plateau_err(Pg), plateau_err(Pr)
    assert all(abs(a - b) < 0.1 * b for a, b in zip(eg, er)), (eg, er)
    assert abs(shock_cell(Pg) - shock_cell(Pr)) <= 1
    assert np.max(np.abs(Pg[4][cold] / 1e-4 - 1)) < (1e-12 if prec == "fp64" else 1e-5)
    if prec == "fp64":
        smooth = cold | plateau
        assert np.max(np.abs(Pg[0][smooth] / Pr[0][smooth] - 1)) < 1e-6
        return
    Ct, _ = oracle.prim2con(W, oracle.ORIGINAL)
    Ct = Ct.astype(np.float32).astype(np.float64)
    Gt, _, worst_t = _riemann_gpu(torch, srhd, Ct, n, "total", prec, t_end)
    Pt = oracle.con2pri(Gt, oracle.ORIGINAL)["prim"]
    assert np.max(np.abs(Pt[4][cold] / 1e-4 - 1)) > 5e-3, worst_t


def test_ultra_relativistic_head_on_collision(oracle):
    # Section 4.2.1 on the GPU in FP64: two streams with U = +-1e6 and
    # T = 1e5 (Table "tb:IC_RiemannProblems", first row) collide at x = 0.5;
    # 512 cells, t = 1. Each scheme matches an oracle run with the GPU's
    # per-patch retries; the two schemes agree with each other, as the paper
    # finds (the reduced energy loses nothing in the ultra-relativistic
    # limit); the shocked gas between the two shocks (Appendix C solution:
    # rho = 40, p = 5.33e12, T ~ 1.3e11) and the shock positions match the
    # exact solution.
    torch, srhd = require_gpu()
    n, t_end = 512, 1.0
    x = (np.arange(n) + 0.5) / n
    W = np.zeros((5, n))
    W[0] = 1e-5
    W[1] = np.where(x < 0.5, 1e6, -1e6)
    W[4] = 1.0
    rho_ex, _, p_ex, info = oracle.exact_riemann((1e-5, 1e6, 1.0), (1e-5, -1e6, 1.0), 0.5, t_end, x)
    assert info["shock_L"] == 1 and info["shock_R"] == 1
    us = info["Ushock_R"]
    xs = t_end * us / np.sqrt(1 + us * us)  # distance of each shock from x = 0.5
    prims = {}
    for scheme, code in (("reduced", oracle.NEW), ("total", oracle.ORIGINAL)):
        C, st = oracle.prim2con(W, code)
        assert np.all(st == 0)
        G, steps, worst = _riemann_gpu(torch, srhd, C, n, scheme, "fp64", t_end)
        assert worst == 0
        ref, ref_steps = _riemann_oracle(oracle, C, n, t_end, code)
        assert steps == ref_steps
        Pg = oracle.con2pri(G, code)["prim"]
        Pr = oracle.con2pri(ref, code)["prim"]
        for v in (0, 4):
            assert np.max(np.abs(Pg[v] / Pr[v] - 1)) < 1e-6, (scheme, v)
        prims[scheme] = Pg
    a, b = prims["reduced"], prims["total"]
    assert max(np.max(np.abs(a[v] / b[v] - 1)) for v in (0, 4)) < 1e-6
    inner = np.abs(x - 0.5) < 0.8 * xs
    # (the post-shock gas carries the spurious waves the paper describes:
    # about 1 % in p at most, a few tenths of a per cent on average)
    assert np.mean(np.abs(a[0][inner] / rho_ex[inner] - 1)) < 0.02
    assert np.mean(np.abs(a[4][inner] / p_ex[inner] - 1)) < 5e-3
    assert np.max(np.abs(a[4][inner] / p_ex[inner] - 1)) < 0.05
    # the shocks: where rho falls half way from the shocked gas to the
    # inflow, within two cells of the exact positions
    half = 0.5 * (rho_ex.max() + 1e-5)
    right = x[np.argmax((x > 0.5) & (a[0] < half))]
    left = x[n - 1 - np.argmax(((x < 0.5) & (a[0] < half))[::-1])]
    assert abs(right - (0.5 + xs)) < 2.0 / n and abs(left - (0.5 - xs)) < 2.0 / n
