"""GPU parity of the fused patch kernel (srhd_advance_patches,
srhd_flux_patches), srhd_cfl_dt and srhd_fill_ghosts_uniform against the
oracle, through the C ABI: smooth patches, rough patches that exercise the
limiter retry, edge cases."""
import numpy as np
import pytest

from gpu_common import (BASE_FP64, EPS64, PRECS, cons_rel_err, flux_rel_err, kappa_of_prims,
                        require_gpu, to_dev, to_np, torch_dtype)
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

# Smooth patches: tolerances after one step (FP64 1e-12; mixed 1e-5, the
# target for smooth flows).
TOL = {"fp64": BASE_FP64, "mixed": 1e-5, "mixed_cf": 1e-5}


def _cons_patches(oracle, Wp, prec):
    npatch = Wp.shape[0]
    C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    assert np.all(st == 0)
    C = C.reshape(5, npatch, 12, 12, 12).transpose(1, 0, 2, 3, 4).copy()
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    return C


def _dtype(torch, prec):
    return torch_dtype(torch, prec)


@pytest.fixture(scope="module")
def smooth_case(oracle):
    npatch = 333  # several patches per CTA plus a ragged tail
    Wp = workloads.smooth_patch_prims(npatch, seed=21)
    dt_dh = np.empty((npatch, 2))
    dt_dh[:, 1] = 1.0 / 12.0 * (1 + 0.1 * np.arange(npatch) / npatch)
    dt_dh[:, 0] = 0.3 * dt_dh[:, 1]
    out = {}
    for prec in ("fp64", "mixed"):
        C = _cons_patches(oracle, Wp, prec)
        ref = oracle.advance_patches(C, dt_dh, want_flux=True)
        out[prec] = (C, ref)
    out["mixed_cf"] = out["mixed"]  # same float inputs
    return dt_dh, out


def _ref_patch_faces(flux):
    """Oracle face fluxes [np][3][5][576] -> patch-face fluxes [np][6][5][64]."""
    npatch = flux.shape[0]
    F = flux.reshape(npatch, 3, 5, 576)
    out = np.empty((npatch, 6, 5, 64))
    fx = F[:, 0].reshape(npatch, 5, 8, 8, 9)   # [k][j][fx]
    fy = F[:, 1].reshape(npatch, 5, 8, 9, 8)   # [k][fy][i]
    fz = F[:, 2].reshape(npatch, 5, 9, 8, 8)   # [fz][j][i]
    out[:, 0] = fx[..., 0].reshape(npatch, 5, 64)
    out[:, 1] = fx[..., 8].reshape(npatch, 5, 64)
    out[:, 2] = fy[:, :, :, 0, :].reshape(npatch, 5, 64)
    out[:, 3] = fy[:, :, :, 8, :].reshape(npatch, 5, 64)
    out[:, 4] = fz[:, :, 0].reshape(npatch, 5, 64)
    out[:, 5] = fz[:, :, 8].reshape(npatch, 5, 64)
    return out


@pytest.mark.parametrize("prec", PRECS)
def test_advance_smooth_parity(oracle, smooth_case, prec):
    torch, srhd = require_gpu()
    dt_dh, cases = smooth_case
    C, ref = cases[prec]
    npatch = C.shape[0]
    dtype = _dtype(torch, prec)
    ctx = srhd.Context(srhd.Params())
    st = torch.full((npatch,), -1, dtype=torch.int32, device="cuda")
    pf = torch.empty((npatch, 6, 5, 64), dtype=dtype, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    out = ctx.advance_patches(to_dev(torch, C, dtype), to_dev(torch, dt_dh, torch.float64),
                              patch_face_flux=pf, dt_next=dn, patch_status=st, prec=prec)
    torch.cuda.synchronize()
    assert np.all(ref["status"] == 0) and np.all(ref["retries"] == 0)
    assert np.all(st.cpu().numpy() == 0)
    err = cons_rel_err(to_np(out).transpose(1, 0, 2, 3, 4), ref["out"].transpose(1, 0, 2, 3, 4))
    assert err.max() <= TOL[prec], err.max()
    # patch-face fluxes (for flux correction) equal the face fluxes there
    pf_ref = _ref_patch_faces(ref["flux"])
    ferr = flux_rel_err(to_np(pf).transpose(2, 0, 1, 3), pf_ref.transpose(2, 0, 1, 3))
    assert ferr.max() <= 10 * TOL[prec], ferr.max()
    # fused CFL of the updated state
    dts = [oracle.cfl_dt(ref["out"][q], dt_dh[q, 1]) for q in range(npatch)]
    assert abs(dn.item() / min(dts) - 1) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_flux_patches_parity(oracle, smooth_case, prec):
    torch, srhd = require_gpu()
    dt_dh, cases = smooth_case
    C, ref = cases[prec]
    npatch = C.shape[0]
    dtype = _dtype(torch, prec)
    st = torch.full((npatch,), -1, dtype=torch.int32, device="cuda")
    F = srhd.flux_patches(to_dev(torch, C, dtype), to_dev(torch, dt_dh, torch.float64),
                          patch_status=st, prec=prec)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    Fg = to_np(F).transpose(2, 0, 1, 3)          # [5][np][3][576]
    Fr = ref["flux"].reshape(npatch, 3, 5, 576).transpose(2, 0, 1, 3)
    err = flux_rel_err(Fg, Fr)
    assert err.max() <= 10 * TOL[prec], err.max()


def test_worklist_subset(oracle, smooth_case):
    torch, srhd = require_gpu()
    dt_dh, cases = smooth_case
    C, ref = cases["fp64"]
    npatch = C.shape[0]
    g = to_dev(torch, C, torch.float64)
    dd = to_dev(torch, dt_dh, torch.float64)
    full = srhd.advance_patches(g, dd)
    rng = np.random.default_rng(3)
    wl = rng.permutation(npatch)[:101].astype(np.int32)
    sent = torch.full((npatch, 5, 8, 8, 8), 7.0, dtype=torch.float64, device="cuda")
    st = torch.full((npatch,), -1, dtype=torch.int32, device="cuda")
    srhd.advance_patches(g, dd, cons_out=sent, worklist=to_dev(torch, wl, torch.int32),
                         patch_status=st)
    torch.cuda.synchronize()
    s, f = to_np(sent), to_np(full)
    mask = np.zeros(npatch, bool)
    mask[wl] = True
    assert np.array_equal(s[mask], f[mask])          # same kernel, same inputs
    assert np.all(s[~mask] == 7.0)                   # other patches untouched
    stn = st.cpu().numpy()
    assert np.all(stn[mask] == 0) and np.all(stn[~mask] == -1)


def kernel_theta(k, prec, theta0=1.5, factor=0.75, floor=1e-2):
    """Limiter coefficient of the kernel's attempt k (Section 3.3 (1)): the
    coefficient times 0.75 per retry, replaced by 0 once below 1e-2 of the
    initial one, in the kernel's arithmetic type (double for FP64, float for
    the float paths, where the product is rounded at every retry)."""
    if prec == "fp64":
        t, f, lim = theta0, factor, floor * theta0
    else:
        t, f, lim = np.float32(theta0), np.float32(factor), np.float32(floor * theta0)
    for _ in range(k):
        t = t * f
        if t < lim:
            t = t * 0
    return float(t)


@pytest.mark.parametrize("prec", PRECS)
def test_rough_patches_retry_parity(oracle, prec):
    # Section 3.3 (1): a patch whose update is unphysical is recomputed with
    # the limiter coefficient times 0.75 per retry, down to 0. Rough patches
    # (uncorrelated cells) retry 10 to 13 times. Each patch reports its retry
    # count k, so the coefficient of its last attempt is known (kernel_theta);
    # the oracle's single attempt at that coefficient must pass and agree
    # cell by cell, and in FP64 the retry count and status must equal the
    # oracle's own. Tolerance per patch: max(base, 10 kappa eps), kappa =
    # 1 + Mach^2 the largest conditioning of the patch's cells (Eq.
    # ImprovedRelativeError) and eps the precision of the stored states
    # (double, or float for the float paths, whose predicted face states are
    # rounded to float before their conversion).
    torch, srhd = require_gpu()
    npatch = 48
    Wp = workloads.rough_patch_prims(npatch, seed=5, spread=1.0)
    C = _cons_patches(oracle, Wp, prec)
    dt_dh = np.empty((npatch, 2))
    dt_dh[:, 1] = 1 / 64
    dt_dh[:, 0] = [oracle.cfl_dt(C[q].reshape(5, -1), 1 / 64) for q in range(npatch)]
    ref = oracle.advance_patches(C, dt_dh)
    assert ref["retries"].min() >= 10
    dtype = _dtype(torch, prec)
    st = torch.full((npatch,), -1, dtype=torch.int32, device="cuda")
    out = srhd.advance_patches(to_dev(torch, C, dtype), to_dev(torch, dt_dh, torch.float64),
                               patch_status=st, prec=prec)
    torch.cuda.synchronize()
    stn = st.cpu().numpy()
    code, retries = stn >> 8, stn & 255
    o = to_np(out)
    assert np.all((code & ~4) == 0), code
    if prec == "fp64":
        assert np.array_equal(retries, ref["retries"]), (retries, ref["retries"])
        assert np.array_equal(code & ~4, ref["status"] & ~4)
    eps = EPS64 if prec == "fp64" else 2.0 ** -24
    worst = 0.0
    for q in range(npatch):
        kappa = kappa_of_prims(oracle, Wp[q]).max()
        tol = max(TOL[prec], 10 * kappa * eps)
        one = oracle.advance_block(C[q], (8, 8, 8), (1, 1, 1), dt_dh[q, 0], dt_dh[q, 1],
                                   theta=kernel_theta(retries[q], prec))
        assert one["retries"] == 0 and one["status"] == 0, (q, retries[q], one)
        err = cons_rel_err(o[q].reshape(5, -1), one["out"].reshape(5, -1))
        worst = max(worst, err.max() / tol)
        assert err.max() <= tol, (q, retries[q], err.max(), tol)
        if retries[q] > 0:
            # the kernel's previous coefficient fails in the oracle too
            tp = kernel_theta(retries[q] - 1, prec)
            prev = oracle.advance_block(C[q], (8, 8, 8), (1, 1, 1), dt_dh[q, 0], dt_dh[q, 1],
                                        theta=tp, retry_factor=0.0)
            assert prev["retries"] == 1, (q, retries[q])
    print(f"retry parity {prec}: retries {retries.min()}..{retries.max()}, "
          f"largest error / tolerance {worst:.3g}")
    A = oracle.con2pri(o.transpose(1, 0, 2, 3, 4).reshape(5, -1))["A"]
    assert np.all(A > 2e-16)


def test_bad_input_and_unused_corner(oracle):
    torch, srhd = require_gpu()
    Wp = workloads.smooth_patch_prims(3, seed=2)
    C = _cons_patches(oracle, Wp, "fp64")
    C[1, 0, 6, 0, 6] = -1.0      # a face ghost cell the step reads: bad input
    C[2, 0, 0, 0, 0] = -1.0      # a corner ghost cell the step never reads
    dt_dh = np.tile([1e-3, 0.1], (3, 1))
    st = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    out = srhd.advance_patches(to_dev(torch, C, torch.float64),
                               to_dev(torch, dt_dh, torch.float64), patch_status=st, dt_next=dn)
    torch.cuda.synchronize()
    stn = st.cpu().numpy()
    assert stn[0] == 0 and stn[2] == 0
    assert stn[1] >> 8 == 2                       # SRHD_PATCH_BAD_INPUT
    o = to_np(out)
    assert np.all(np.isnan(o[1])) and np.all(np.isfinite(o[[0, 2]]))
    assert np.isnan(dn.item())
    ref = oracle.advance_patches(C, dt_dh)
    assert ref["status"].tolist() == [0, 2, 0]
    assert np.abs(o[2] - ref["out"][2]).max() <= 1e-12 * np.abs(ref["out"][2]).max()


def test_uniform_state_is_fixed_point():
    torch, srhd = require_gpu()
    for prec in PRECS:
        dtype = torch_dtype(torch, prec)
        W = torch.tensor([[2e-3], [30.0], [-4.0], [0.5], [7e-5]], dtype=dtype, device="cuda")
        U = srhd.prim2con(W)
        G = U.reshape(1, 5, 1, 1, 1).expand(4, 5, 12, 12, 12).contiguous()
        dd = torch.tensor([[1e-3, 1e-2]] * 4, dtype=torch.float64, device="cuda")
        out = srhd.advance_patches(G, dd, prec=prec)
        assert torch.equal(out, G[:, :, 2:10, 2:10, 2:10])


def test_empty_batch():
    torch, srhd = require_gpu()
    g = torch.empty((0, 5, 12, 12, 12), dtype=torch.float64, device="cuda")
    dd = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = srhd.advance_patches(g, dd, dt_next=dn)
    torch.cuda.synchronize()
    assert out.shape[0] == 0 and dn.item() == float("inf")
    dt = srhd.cfl_dt(torch.empty((0, 5, 8, 8, 8), dtype=torch.float64, device="cuda"), 0.1)
    assert dt.item() == float("inf")


@pytest.mark.parametrize("prec", PRECS)
def test_cfl_dt_parity(oracle, prec):
    torch, srhd = require_gpu()
    npatch = 77
    dtype = _dtype(torch, prec)
    # well-conditioned cells (gamma <= 30, T >= 1e-4): values agree
    W = workloads.stress_batch_prims(npatch * 512, seed=9, lg_gamma_range=(0, 1.5),
                                     T_range=(-4, 3))
    C, _ = oracle.prim2con(W)
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    Cp = C.reshape(5, npatch, 512).transpose(1, 0, 2).copy()
    dt = srhd.cfl_dt(to_dev(torch, Cp, dtype), 0.01, prec=prec).item()
    ref = oracle.cfl_dt(C, 0.01)
    assert np.isfinite(ref) and abs(dt / ref - 1) <= (1e-12 if prec == "fp64" else 1e-5)
    # light-speed mode
    ctx = srhd.Context(srhd.Params(cfl_mode="light"))
    assert ctx.cfl_dt(to_dev(torch, Cp, dtype), 0.01, prec=prec).item() == 0.5 * 0.01
    # a batch with an unphysical cell gives NaN on both sides
    C2 = C.copy()
    C2[4, 1234] = -1.0
    Cp2 = C2.reshape(5, npatch, 512).transpose(1, 0, 2).copy()
    assert np.isnan(srhd.cfl_dt(to_dev(torch, Cp2, dtype), 0.01, prec=prec).item())
    assert np.isnan(oracle.cfl_dt(C2, 0.01))


def test_fill_ghosts_uniform(oracle):
    torch, srhd = require_gpu()
    rng = np.random.default_rng(4)
    for bc in (("periodic",) * 3, ("outflow", "periodic", "outflow")):
        F = rng.normal(size=(5, 16, 24, 32))
        P = workloads.patchify(F)
        G = srhd.fill_ghosts_uniform(to_dev(torch, P, torch.float64), 4, 3, 2, bc=bc)
        assert np.array_equal(to_np(G), workloads.ghosted_patches(F, bc))


def test_argument_errors():
    torch, srhd = require_gpu()
    from paper_2012_11130_gb300 import _native as N
    g = torch.zeros((2, 5, 12, 12, 12), dtype=torch.float64, device="cuda")
    dd = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(N.SrhdError, match="npatch"):
        srhd.advance_patches(g, dd, npatch=-1)
    with pytest.raises(N.SrhdError, match="cfl"):
        srhd.Context(srhd.Params(cfl=2.0))
    with pytest.raises(TypeError):
        srhd.advance_patches(g.to(torch.float16), dd)


@pytest.mark.parametrize("prec", ["mixed_cf", "fp64"])
def test_host_buffer_path_matches_device_path(oracle, smooth_case, prec):
    # The public call with pinned host tensors (chunked copies overlapping
    # the fused steps on three streams) returns the device path's result.
    torch, srhd = require_gpu()
    dt_dh, cases = smooth_case
    C, ref = cases[prec]
    dtype = _dtype(torch, prec)
    ctx = srhd.Context(srhd.Params())
    g = to_dev(torch, C, dtype)
    dd = to_dev(torch, dt_dh, torch.float64)
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    want = to_np(ctx.advance_patches(g, dd, dt_next=dn, prec=prec))
    gh = g.cpu().pin_memory()
    ddh = dd.cpu().pin_memory()
    outh = torch.empty((C.shape[0], 5, 8, 8, 8), dtype=dtype).pin_memory()
    dnh = torch.empty(1, dtype=torch.float64).pin_memory()
    sth = torch.full((C.shape[0],), -1, dtype=torch.int32).pin_memory()
    for _ in range(2):  # the second call reuses the device buffers
        ctx.advance_patches(gh, ddh, cons_out=outh, dt_next=dnh, patch_status=sth, prec=prec)
        assert np.array_equal(outh.double().numpy(), want)
        assert dnh.item() == dn.item()
        assert np.all(sth.numpy() == 0)
