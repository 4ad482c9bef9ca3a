"""GPU tests of the primitive cache of uniform-grid steps
(srhd_con2pri_patches, srhd_advance_uniform_prim).

The update phase converts each new state anyway (CFL bound of Section 3.2,
check of Eq. Unphysical result); the cached step keeps those primitives and
the next step gathers its tiles' primitives from them. Checked here:
* srhd_con2pri_patches gives the primitives of srhd_con2pri bitwise and a
  solver variable consistent with them (T = p/rho from the conic parameter);
* several cached steps, ping-ponging state and primitives, follow the
  uncached steps (srhd_advance_uniform) to the rounding of the Newton roots,
  with equal statuses and CFL bounds, on periodic and mixed boundaries and on
  a field that makes patches retry; the cached primitives are the conversion
  of the new state; a grid split into two patch ranges gives the same step;
* a NaN in the cache marks the patches that read it SRHD_PATCH_BAD_INPUT,
  with NaN outputs; aliasing outputs are refused."""
import numpy as np
import pytest

from gpu_common import cons_rel_err, require_gpu
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

NPX, NPY, NPZ = 3, 2, 4
NP = NPX * NPY * NPZ
# per-step agreement of cached and uncached steps (both correct to rounding)
TOL = {"fp64": 1e-12, "mixed": 1e-5, "mixed_cf": 1e-5}


def _smooth_grid(oracle, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = 8 * NPZ, 8 * NPY, 8 * NPX
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                          indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 5)
    W = np.stack([1 + 0.3 * np.sin(2 * np.pi * (x + 2 * y) + ph[0]),
                  0.6 * np.sin(2 * np.pi * (x + z) + ph[2]),
                  0.6 * np.cos(2 * np.pi * (x - y) + ph[3]),
                  0.6 * np.sin(2 * np.pi * z + ph[4]),
                  1 + 0.3 * np.sin(2 * np.pi * (y - z) + ph[1])]).reshape(5, -1)
    C, st = oracle.prim2con(W)
    assert np.all(st == 0)
    return workloads.patchify(C.reshape(5, nz, ny, nx))


def _rough_grid(oracle):
    Wp = workloads.rough_patch_prims(NP, seed=2, spread=0.5, lg_gamma_max=0.7, edge=8)
    C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    assert np.all(st == 0)
    return C.reshape(5, -1, 8, 8, 8).transpose(1, 0, 2, 3, 4)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_cf"])
def test_con2pri_patches(oracle, prec):
    torch, srhd = require_gpu()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    n = 40
    W = workloads.stress_batch_prims(n * 512, seed=31, lg_gamma_range=(0, 3), T_range=(-6, 3))
    C, _ = oracle.prim2con(W)
    Cp = torch.from_numpy(np.ascontiguousarray(C.reshape(5, n, 512).transpose(1, 0, 2))).to(dtype)
    Cp = Cp.cuda()
    Cp[3, 1, 17] = 2 * (Cp[3, 4, 17] + Cp[3, 0, 17])  # one unphysical cell: |M| > Etilde + D
    ctx = srhd.Context(srhd.Params())
    P6 = ctx.con2pri_patches(Cp.view(n, 5, 8, 8, 8), prec=prec)
    flat = Cp.transpose(0, 1).reshape(5, -1).contiguous()
    P5 = ctx.con2pri(flat, prec=prec)
    torch.cuda.synchronize()
    got = P6.view(n, 6, 512).transpose(0, 1).reshape(6, -1)
    assert torch.equal(torch.nan_to_num(got[:5], nan=-7.0), torch.nan_to_num(P5, nan=-7.0))
    g = got.double().cpu().numpy()
    bad = 3 * 512 + 17
    assert np.all(np.isnan(g[:, bad]))
    # cells unphysical after rounding to float (extreme Lorentz factors and
    # temperatures) are NaN as well, in both conversions
    ok = ~np.isnan(g[0])
    assert np.all(np.isnan(g[:, ~ok])) and ok.mean() > 0.9
    tau = g[5, ok]
    t = 1.0 + tau
    T = tau * (2.0 + tau) / (3.0 * t)                 # TM conic parametrisation
    T_ref = g[4, ok] / g[0, ok]
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.all(np.abs(T / T_ref - 1) <= tol), np.abs(T / T_ref - 1).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_cf"])
@pytest.mark.parametrize("case", ["smooth-periodic", "smooth-mixed-bc", "rough-periodic"])
def test_cached_steps_follow_uncached(oracle, prec, case):
    torch, srhd = require_gpu()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    bc = ("outflow", "periodic", "outflow") if case == "smooth-mixed-bc" else ("periodic",) * 3
    P = _rough_grid(oracle) if case.startswith("rough") else _smooth_grid(oracle, 4)
    U0 = torch.from_numpy(np.ascontiguousarray(P)).to(dtype).cuda()
    ctx = srhd.Context(srhd.Params())
    rough = case.startswith("rough")
    dt = 0.004 if rough else 0.3 / 32
    dd = torch.tensor([[dt, 1 / 32]] * NP, dtype=torch.float64, device="cuda")
    # A retry is a block-wide vote on the unphysical check; on the rough
    # field a float rounding difference can flip a marginal vote, after which
    # the runs differ by more than rounding, so in float it is one step.
    nsteps = 1 if rough and prec != "fp64" else 4
    # uncached reference
    Ua = U0.clone()
    ref = []
    for _ in range(nsteps):
        st = torch.full((NP,), -1, dtype=torch.int32, device="cuda")
        dn = torch.empty(1, dtype=torch.float64, device="cuda")
        Ua = ctx.advance_uniform(Ua, NPX, NPY, NPZ, dd, bc=bc, dt_next=dn, patch_status=st,
                                 prec=prec)
        ref.append((Ua.clone(), st.clone(), dn.clone()))
    # cached: ping-pong of state and primitives
    Ub = U0.clone()
    Pb = ctx.con2pri_patches(Ub, prec=prec)
    retried = 0
    for k in range(nsteps):
        st = torch.full((NP,), -1, dtype=torch.int32, device="cuda")
        dn = torch.empty(1, dtype=torch.float64, device="cuda")
        Ub, Pb = ctx.advance_uniform_prim(Ub, Pb, NPX, NPY, NPZ, dd, bc=bc, dt_next=dn,
                                          patch_status=st, prec=prec)
        torch.cuda.synchronize()
        Ur, sr, dr = ref[k]
        assert torch.equal(st, sr), k
        retried += int((st & 255).max())
        err = cons_rel_err(Ub.double().cpu().numpy().transpose(1, 0, 2, 3, 4),
                           Ur.double().cpu().numpy().transpose(1, 0, 2, 3, 4))
        assert err.max() <= TOL[prec] * (k + 1), (k, err.max())
        assert abs(dn.item() / dr.item() - 1) <= TOL[prec] * (k + 1)
        # the cache holds the conversion of the new state
        Pc = ctx.con2pri_patches(Ub, prec=prec)
        torch.cuda.synchronize()
        a, b = Pb.double().cpu().numpy(), Pc.double().cpu().numpy()
        rel = np.abs(a[:, :5] - b[:, :5]) / (np.abs(b[:, :5]) + np.abs(b[:, :1]))
        assert rel.max() <= (1e-13 if prec == "fp64" else 2e-6), rel.max()
    if rough:
        assert retried > 0


def test_cached_ranges_and_errors(oracle):
    torch, srhd = require_gpu()
    from paper_2012_11130_gb300 import _native as N
    P = _smooth_grid(oracle, 9)
    U = torch.from_numpy(np.ascontiguousarray(P)).float().cuda()
    ctx = srhd.Context(srhd.Params())
    dd = torch.tensor([[0.3 / 32, 1 / 32]] * NP, dtype=torch.float64, device="cuda")
    Pc = ctx.con2pri_patches(U)
    whole_u, whole_p = ctx.advance_uniform_prim(U, Pc, NPX, NPY, NPZ, dd)
    # the same step as two patch ranges writing into slices of one output
    out_u = torch.empty_like(whole_u)
    out_p = torch.empty_like(whole_p)
    k = 10
    ctx.advance_uniform_prim(U, Pc, NPX, NPY, NPZ, dd[:k], p0=0, n=k, cons_out=out_u[:k],
                             prim_out=out_p[:k])
    ctx.advance_uniform_prim(U, Pc, NPX, NPY, NPZ, dd[k:], p0=k, n=NP - k, cons_out=out_u[k:],
                             prim_out=out_p[k:])
    torch.cuda.synchronize()
    assert torch.equal(out_u, whole_u) and torch.equal(out_p, whole_p)
    # a NaN in the cache: every patch whose tile reads that cell is bad input
    bad = Pc.clone()
    bad[5, 0, 0, 0, 0] = float("nan")             # patch 5 = (2, 1, 0), corner cell (0, 0, 0)
    st = torch.full((NP,), -1, dtype=torch.int32, device="cuda")
    ou, op = ctx.advance_uniform_prim(U, bad, NPX, NPY, NPZ, dd, patch_status=st)
    torch.cuda.synchronize()
    code = (st.cpu().numpy() >> 8)
    flagged = set(np.nonzero(code & N.PATCH_BAD_INPUT)[0].tolist())
    # readers of cell (0,0,0) of patch (2,1,0): the patch itself and its face
    # neighbours at lower x, y, z (edges of the first ghost layer are read too)
    assert {5, 4, 2, 5 + 18} <= flagged
    for q in flagged:
        assert torch.isnan(ou[q]).all() and torch.isnan(op[q]).all()
    assert not torch.isnan(ou[0]).any()
    # outputs that alias the inputs are refused
    with pytest.raises(N.SrhdError, match="alias"):
        ctx.advance_uniform_prim(U, Pc, NPX, NPY, NPZ, dd, cons_out=U[:NP], prim_out=op)
    with pytest.raises(N.SrhdError, match="alias"):
        ctx.advance_uniform_prim(U, Pc, NPX, NPY, NPZ, dd, prim_out=Pc)
