"""The uniform-grid gather with tensor-map staging: on grids with several
patches per CTA, the tiles of the second and later patches of each CTA come
from seven tensor copies (interior and face slabs of the neighbours, issued
during the previous patch's update) instead of plain loads. The result must
equal the ghost fill followed by srhd_advance_patches bitwise: whole grids
and patch ranges, periodic boundaries (every later patch staged) and outflow
ones (boundary patches keep plain loads), a field that makes patches retry
(a retry waits for the copies before it rewrites the stage), and the
host-resident step, whose slabs are launched one by one. The cached step
(primitive cache, mode 3) stages variables 0..4 of the cache the same way
and must equal the same step taken in ranges too small to stage."""
import numpy as np
import pytest

from gpu_common import require_gpu
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

NPX, NPY, NPZ = 32, 16, 4      # 2048 patches: several per CTA in every launch variant
NP = NPX * NPY * NPZ


def _grid(oracle):
    nz, ny, nx = 8 * NPZ, 8 * NPY, 8 * NPX
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                          indexing="ij")
    W = np.stack([1 + 0.3 * np.sin(2 * np.pi * (x + 2 * y)),
                  0.6 * np.sin(2 * np.pi * (x + z)),
                  0.6 * np.cos(2 * np.pi * (x - y)),
                  0.6 * np.sin(2 * np.pi * z),
                  1 + 0.3 * np.sin(2 * np.pi * (y - z))]).reshape(5, nz, ny, nx)
    # a rough block (uncorrelated cells) in a few patches, so that they retry
    rough = workloads.rough_patch_prims(1, seed=4, spread=0.5, lg_gamma_max=0.7, edge=8)[0]
    for (pz, py, px) in ((1, 3, 5), (2, 9, 20), (0, 15, 31)):
        W[:, 8 * pz:8 * pz + 8, 8 * py:8 * py + 8, 8 * px:8 * px + 8] = rough
    C, st = oracle.prim2con(W.reshape(5, -1))
    assert np.all(st == 0)
    return workloads.patchify(C.reshape(5, nz, ny, nx))


def _same(a, b):
    it = {8: "int64", 4: "int32"}[a.element_size()]
    import torch
    return a.dtype == b.dtype and torch.equal(a.view(getattr(torch, it)),
                                              b.view(getattr(torch, it)))


@pytest.mark.parametrize("prec", ["fp64", "mixed_cf"])
@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow")])
def test_staged_gather_equals_fill_and_advance(oracle, prec, bc):
    torch, srhd = require_gpu()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    U = torch.from_numpy(_grid(oracle)).to(dtype).cuda()
    dd = torch.tensor([[0.004, 1 / 32]] * NP, dtype=torch.float64, device="cuda")
    for variant in (0, 1):
        ctx = srhd.Context(srhd.Params(patch_variant=variant))
        G = ctx.fill_ghosts_uniform(U, NPX, NPY, NPZ, bc=bc)
        for p0, n in ((0, NP), (700, 1000)):
            outs = []
            for gather in (False, True):
                st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
                dn = torch.empty(1, dtype=torch.float64, device="cuda")
                pf = torch.zeros((n, 6, 5, 64), dtype=dtype, device="cuda")
                if gather:
                    o = ctx.advance_uniform(U, NPX, NPY, NPZ, dd[p0:p0 + n].contiguous(), bc=bc,
                                            p0=p0, n=n, patch_face_flux=pf, dt_next=dn,
                                            patch_status=st, prec=prec)
                else:
                    o = ctx.advance_patches(G[p0:p0 + n].contiguous(),
                                            dd[p0:p0 + n].contiguous(), patch_face_flux=pf,
                                            dt_next=dn, patch_status=st, prec=prec)
                torch.cuda.synchronize()
                outs.append((o, pf, dn, st))
            (o0, f0, d0, s0), (o1, f1, d1, s1) = outs
            assert torch.equal(s0, s1) and int(s0.min()) >= 0
            assert _same(o1, o0) and _same(f1, f0) and _same(d1, d0)
            if p0 == 0:
                assert int((s0 & 255).max()) > 0      # some patches retried


def test_host_step_with_staged_slabs(oracle):
    torch, srhd = require_gpu()
    U = torch.from_numpy(_grid(oracle)).float()
    ctx = srhd.Context(srhd.Params(patch_variant=1))
    dt, dh = 0.004, 1 / 32
    out, dn = ctx.advance_uniform_host(U.pin_memory(), NPX, NPY, NPZ, dt, dh, chunks=NPZ)
    Ud = U.cuda()
    G = ctx.fill_ghosts_uniform(Ud, NPX, NPY, NPZ)
    dd = torch.tensor([[dt, dh]] * NP, dtype=torch.float64, device="cuda")
    dnd = torch.empty(1, dtype=torch.float64, device="cuda")
    want = ctx.advance_patches(G, dd, dt_next=dnd)
    torch.cuda.synchronize()
    assert _same(out, want.cpu()) and dn == dnd.item()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_cf"])
@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow")])
def test_staged_cached_step_equals_unstaged(oracle, prec, bc):
    # mode 3 (primitive cache): variables 0..4 of the cached tile come from
    # the tensor copies on the second and later patches of each CTA. The
    # whole-grid step must equal the same step taken in ranges of 128
    # patches, fewer than the CTAs of a launch, so that nothing is staged.
    torch, srhd = require_gpu()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    U = torch.from_numpy(_grid(oracle)).to(dtype).cuda()
    dd = torch.tensor([[0.004, 1 / 32]] * NP, dtype=torch.float64, device="cuda")
    ctx = srhd.Context(srhd.Params(patch_variant=1 if prec != "fp64" else 0))
    P = ctx.con2pri_patches(U, prec=prec)
    st = torch.full((NP,), -1, dtype=torch.int32, device="cuda")
    whole_u, whole_p = ctx.advance_uniform_prim(U, P, NPX, NPY, NPZ, dd, bc=bc, patch_status=st,
                                                prec=prec)
    part_u, part_p = torch.empty_like(whole_u), torch.empty_like(whole_p)
    st2 = torch.full((NP,), -1, dtype=torch.int32, device="cuda")
    for p0 in range(0, NP, 128):
        ctx.advance_uniform_prim(U, P, NPX, NPY, NPZ, dd[p0:p0 + 128].contiguous(), bc=bc,
                                 p0=p0, n=128, cons_out=part_u[p0:p0 + 128],
                                 prim_out=part_p[p0:p0 + 128], patch_status=st2[p0:p0 + 128],
                                 prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(st, st2) and int((st & 255).max()) > 0
    assert _same(whole_u, part_u) and _same(whole_p, part_p)
