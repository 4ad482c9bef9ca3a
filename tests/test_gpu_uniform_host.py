"""GPU parity of the uniform-grid steps. srhd_advance_uniform (the patch
kernel gathering its tiles from the grid) is bit-identical to the ghost
fill followed by srhd_advance_patches, for whole grids and patch ranges.
The host-resident step (srhd_advance_uniform_host): the chunked pipeline (copies in, ghost fill,
fused step, copies out on four streams) equals the oracle's MUSCL-Hancock
step of the whole periodic or mixed-boundary grid, is bit-identical for
every chunk count, in place, with pageable memory and to the device-resident
path (fill + srhd_advance_patches), and reports unphysical cells and bad
arguments; at the full 256^3 size of the benchmark it is bit-identical to the
device-resident gathering step."""
import numpy as np
import pytest
import torch as _torch

from gpu_common import cons_rel_err, require_gpu
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

NPX, NPY, NPZ = 3, 2, 4


def _field(oracle, seed):
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
    return C.reshape(5, nz, ny, nx)


def _pad(C, bc):
    mode = {"periodic": "wrap", "outflow": "edge"}
    for ax, b in zip((3, 2, 1), bc):
        pads = [(0, 0)] * 4
        pads[ax] = (2, 2)
        C = np.pad(C, pads, mode=mode[b])
    return C


def _same_bits(a, b):
    """Bitwise equality (NaN included)."""
    it = {8: _torch.int64, 4: _torch.int32}[a.element_size()]
    return a.dtype == b.dtype and _torch.equal(a.view(it), b.view(it))


def _host(a, dtype, pinned=True):
    t = _torch.from_numpy(np.ascontiguousarray(a)).to(dtype)
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_cf"])
@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow")])
def test_gather_equals_fill_and_advance(oracle, prec, bc):
    torch, srhd = require_gpu()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    # a rough field, so that some patches retry with a smaller limiter
    Wp = workloads.rough_patch_prims(NPX * NPY * NPZ, seed=2, spread=0.5, lg_gamma_max=0.7,
                                     edge=8)
    C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    assert np.all(st == 0)
    P = C.reshape(5, -1, 8, 8, 8).transpose(1, 0, 2, 3, 4)
    U = torch.from_numpy(np.ascontiguousarray(P)).to(dtype).cuda()
    npatch = NPX * NPY * NPZ
    ctx = srhd.Context()
    dd = torch.tensor([[0.004 + 1e-4 * i, 1 / 32] for i in range(npatch)], dtype=torch.float64,
                      device="cuda")
    G = ctx.fill_ghosts_uniform(U, NPX, NPY, NPZ, bc=bc)

    def run(step, rows):
        n = len(rows)
        pf = torch.zeros((n, 6, 5, 64), dtype=dtype, device="cuda")
        dn = torch.empty(1, dtype=torch.float64, device="cuda")
        stt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        out = step(pf, dn, stt)
        return out.cpu(), pf.cpu(), dn.item(), stt.cpu()

    for p0, n in ((0, npatch), (5, 9), (npatch - 7, 7)):
        rows = list(range(p0, p0 + n))
        wl = torch.tensor(rows, dtype=torch.int32, device="cuda")
        want = run(lambda pf, dn, stt: ctx.advance_patches(
            G[p0:p0 + n].contiguous(), dd[p0:p0 + n].contiguous(), patch_face_flux=pf,
            dt_next=dn, patch_status=stt, prec=prec), rows)
        got = run(lambda pf, dn, stt: ctx.advance_uniform(
            U, NPX, NPY, NPZ, dd[p0:p0 + n].contiguous(), bc=bc, p0=p0, n=n, patch_face_flux=pf,
            dt_next=dn, patch_status=stt, prec=prec), rows)
        assert _same_bits(got[0], want[0]) and _same_bits(got[1], want[1])
        assert _same_bits(torch.tensor(got[2]), torch.tensor(want[2]))
        assert torch.equal(got[3], want[3])
        del wl
    # the rough field exercises the limiter retry
    assert int((want[3] & 255).max()) > 0


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow")])
def test_matches_oracle_and_every_chunking(oracle, prec, bc):
    torch, srhd = require_gpu()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    C = _field(oracle, seed=3)
    if prec != "fp64":
        C = C.astype(np.float32).astype(np.float64)
    dh, dt = 1.0 / 32, 0.4 / 32
    ref = oracle.advance_block(_pad(C, bc), (8 * NPX, 8 * NPY, 8 * NPZ), (1, 1, 1), dt, dh)
    assert ref["status"] == 0 and ref["retries"] == 0
    want_dt = oracle.cfl_dt(ref["out"], dh)
    ctx = srhd.Context()
    U = _host(workloads.patchify(C), dtype)
    npatch = NPX * NPY * NPZ
    outs = []
    for chunks in (1, 2, 3, 4, 9, 32):
        st = torch.full((npatch,), -1, dtype=torch.int32)
        out, dn = ctx.advance_uniform_host(U, NPX, NPY, NPZ, dt, dh, bc=bc, patch_status=st,
                                           chunks=chunks, prec=prec)
        assert int(st.abs().max()) == 0
        outs.append((out.clone(), dn))
    for out, dn in outs[1:]:
        assert torch.equal(out, outs[0][0]) and dn == outs[0][1]
    got = workloads.unpatchify(outs[0][0].double().numpy(), NPX, NPY, NPZ)
    tol = 1e-12 if prec == "fp64" else 1e-5
    err = cons_rel_err(got.reshape(5, -1), ref["out"].reshape(5, -1))
    assert err.max() <= tol, err.max()
    assert abs(outs[0][1] / want_dt - 1) <= tol
    # the device-resident path gives the same bits
    Ud = U.cuda()
    G = ctx.fill_ghosts_uniform(Ud, NPX, NPY, NPZ, bc=bc)
    dd = torch.tensor([[dt, dh]] * npatch, dtype=torch.float64, device="cuda")
    dnd = torch.empty(1, dtype=torch.float64, device="cuda")
    outd = ctx.advance_patches(G, dd, dt_next=dnd, prec=prec)
    assert torch.equal(outd.cpu(), outs[0][0]) and dnd.item() == outs[0][1]
    # in place, and from pageable memory
    V = U.clone()
    out, dn = ctx.advance_uniform_host(V, NPX, NPY, NPZ, dt, dh, bc=bc, cons_out=V, chunks=3,
                                       prec=prec)
    assert out is V and torch.equal(V, outs[0][0]) and dn == outs[0][1]
    Up = _host(workloads.patchify(C), dtype, pinned=False)
    out, dn = ctx.advance_uniform_host(Up, NPX, NPY, NPZ, dt, dh, bc=bc, chunks=2, prec=prec)
    assert torch.equal(out, outs[0][0]) and dn == outs[0][1]


def test_unphysical_cell_and_bad_arguments(oracle):
    torch, srhd = require_gpu()
    C = _field(oracle, seed=5)
    P = workloads.patchify(C)
    P[7, 0, 3, 3, 3] = -1.0  # negative D in patch 7
    U = _host(P, torch.float64)
    ctx = srhd.Context()
    st = torch.zeros(NPX * NPY * NPZ, dtype=torch.int32)
    out, dn = ctx.advance_uniform_host(U, NPX, NPY, NPZ, 1e-3, 1.0 / 32, patch_status=st)
    assert np.isnan(dn)
    s = st.numpy()
    assert s[7] >> 8 == 2 and (np.delete(s, 7) == 0).all()
    assert torch.isnan(out[7]).all() and not torch.isnan(out[:7]).any()
    # a grid larger than the first allocates a larger stage
    big = _host(np.concatenate([P, P]), torch.float64)
    out, dn = ctx.advance_uniform_host(big, NPX, NPY, 2 * NPZ, 1e-3, 1.0 / 32)
    assert np.isnan(dn)
    for kw in (dict(chunks=0), dict(chunks=65), dict(dt=-1.0), dict(dh=0.0)):
        args = dict(dt=1e-3, dh=1.0 / 32, chunks=4)
        args.update(kw)
        with pytest.raises(Exception):
            ctx.advance_uniform_host(U, NPX, NPY, NPZ, args["dt"], args["dh"],
                                     chunks=args["chunks"])
    with pytest.raises(ValueError):
        ctx.advance_uniform_host(U.cuda(), NPX, NPY, NPZ, 1e-3, 1.0 / 32)


def test_uniform_edge_cases(oracle):
    torch, srhd = require_gpu()
    ctx = srhd.Context()
    # a grid one slab deep (npz = 1): one chunk whatever is asked, z periodic
    npx, npy, npz = 4, 3, 1
    rng = np.random.default_rng(11)
    W = np.stack([1 + 0.2 * rng.random((8, 24, 32)), 0.1 * rng.standard_normal((8, 24, 32)),
                  0.1 * rng.standard_normal((8, 24, 32)), 0.1 * rng.standard_normal((8, 24, 32)),
                  1 + 0.2 * rng.random((8, 24, 32))]).reshape(5, -1)
    C, st = oracle.prim2con(W)
    assert np.all(st == 0)
    C = C.reshape(5, 8, 24, 32)
    U = _host(workloads.patchify(C), torch.float64)
    out, dn = ctx.advance_uniform_host(U, npx, npy, npz, 1e-3, 1 / 32, chunks=8)
    ref = oracle.advance_block(_pad(C, ("periodic",) * 3), (32, 24, 8), (1, 1, 1), 1e-3, 1 / 32)
    got = workloads.unpatchify(out.numpy(), npx, npy, npz)
    assert cons_rel_err(got.reshape(5, -1), ref["out"].reshape(5, -1)).max() <= 1e-12
    assert abs(dn / oracle.cfl_dt(ref["out"], 1 / 32) - 1) <= 1e-12
    # an empty range still reports the CFL bound of nothing (+inf); ranges
    # outside the grid and foreign tensors are refused
    Ud = U.cuda()
    dd = torch.tensor([[1e-3, 1 / 32]] * 12, dtype=torch.float64, device="cuda")
    dnd = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.advance_uniform(Ud, npx, npy, npz, dd, p0=5, n=0, dt_next=dnd)
    assert dnd.item() == float("inf")
    with pytest.raises(Exception, match="range"):
        ctx.advance_uniform(Ud, npx, npy, npz, dd, p0=10, n=3)
    with pytest.raises(Exception):
        ctx.advance_uniform(Ud, npx, npy, npz + 1, dd)


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
def test_full_size_host_step_equals_device_step(oracle, prec):
    # The end-to-end configuration bench.py times: the 256^3 advection grid
    # (32768 patches) in pinned host memory, 32 z-slab chunks on four
    # streams. Its output, dt_next and statuses are bitwise those of the
    # device-resident gathering step (srhd_advance_uniform) of the same
    # state, which the full-size sampled test of test_gpu_runs.py compares
    # with the oracle.
    torch, srhd = require_gpu()
    N = 256
    npx = N // 8
    Wf = workloads.advection_prims(N)
    C, _ = oracle.prim2con(Wf.reshape(5, -1))
    C = C.reshape(5, N, N, N)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    U = workloads.patchify(C.astype(np.float64 if prec == "fp64" else np.float32))
    dh = 1.0 / N
    dt = 0.4 * dh
    ctx = srhd.Context()
    H = _host(U, dtype)
    out_h = torch.empty_like(H).pin_memory()
    st_h = torch.empty(npx ** 3, dtype=torch.int32).pin_memory()
    _, dn_h = ctx.advance_uniform_host(H, npx, npx, npx, dt, dh, cons_out=out_h,
                                       patch_status=st_h, prec=prec)
    D = H.to("cuda")
    dd = torch.tensor([[dt, dh]], dtype=torch.float64, device="cuda").repeat(npx ** 3, 1)
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(npx ** 3, dtype=torch.int32, device="cuda")
    out_d = ctx.advance_uniform(D, npx, npx, npx, dd, dt_next=dn, patch_status=st, prec=prec)
    torch.cuda.synchronize()
    assert _same_bits(out_h, out_d.cpu())
    assert np.array_equal(st_h.numpy(), st.cpu().numpy()) and int(st_h.abs().max()) == 0
    assert dn_h == dn.item()
