"""A patch's result does not depend on where it sits in the batch.

For a ghosted batch the fused kernel copies each CTA's next tile into shared
memory with the bulk-copy engine while the current patch is updated, and
phase 1 of the next patch reads it from there; a limiter retry waits for
that copy before it rewrites the slots. A pool of rough patches (which retry,
Section 3.3 (1)) and smooth ones is first advanced alone, with fewer patches
than CTAs, so that no tile is staged; then a batch that repeats pool patches
in random order, several per CTA, must give bitwise the same outputs and
statuses, directly, through a worklist, and from an input that is not 16-byte
aligned (no staging)."""
import numpy as np
import pytest

from gpu_common import require_gpu, to_dev, to_np, torch_dtype
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu

N_ROUGH, N_SMOOTH = 48, 64   # pool of 112 patches: fewer than the CTAs of any launch
N_BATCH = 1500


@pytest.fixture(scope="module")
def pool(oracle):
    Wr = workloads.rough_patch_prims(N_ROUGH, seed=5, spread=1.0)
    Ws = workloads.smooth_patch_prims(N_SMOOTH, seed=23)
    W = np.concatenate([Wr, Ws])
    n = W.shape[0]
    C, st = oracle.prim2con(W.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    assert np.all(st == 0)
    C = C.reshape(5, n, 12, 12, 12).transpose(1, 0, 2, 3, 4).copy()
    dt_dh = np.empty((n, 2))
    dt_dh[:, 1] = 1 / 64
    dt_dh[:, 0] = [oracle.cfl_dt(C[q].reshape(5, -1), 1 / 64) for q in range(n)]
    return C, dt_dh


@pytest.mark.parametrize("prec,variant", [("fp64", 0), ("fp64", 2), ("mixed", 0),
                                          ("mixed_cf", 0), ("mixed_cf", 1)])
def test_batch_position_does_not_change_results(pool, prec, variant):
    torch, srhd = require_gpu()
    C, dt_dh = pool
    dtype = torch_dtype(torch, prec)
    ctx = srhd.Context(srhd.Params(patch_variant=variant))
    n = C.shape[0]

    def run(g, dd, worklist=None, npatch=None):
        m = g.shape[0]
        st = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        dn = torch.empty(1, dtype=torch.float64, device="cuda")
        out = ctx.advance_patches(g, dd, worklist=worklist, npatch=npatch, dt_next=dn,
                                  patch_status=st, prec=prec)
        torch.cuda.synchronize()
        return to_np(out), st.cpu().numpy(), dn.item()

    ref_out, ref_st, ref_dt = run(to_dev(torch, C, dtype), to_dev(torch, dt_dh, torch.float64))
    assert (ref_st & 255).max() > 0, "the pool must contain retried patches"
    assert np.all(ref_st >= 0)

    rng = np.random.default_rng(77)
    idx = rng.integers(0, n, N_BATCH)
    g = to_dev(torch, C[idx], dtype)
    dd = to_dev(torch, dt_dh[idx], torch.float64)
    out, st, dt = run(g, dd)
    assert np.array_equal(st, ref_st[idx])
    assert np.array_equal(out, ref_out[idx])
    assert len(np.unique(idx)) == n  # every pool patch is in the batch
    assert dt == ref_dt or (np.isnan(dt) and np.isnan(ref_dt))

    # through a worklist: a permuted subset, the other patches untouched
    wl = rng.permutation(N_BATCH)[:1100].astype(np.int32)
    out_w = torch.full((N_BATCH, 5, 8, 8, 8), 7.0, dtype=dtype, device="cuda")
    st_w = torch.full((N_BATCH,), -1, dtype=torch.int32, device="cuda")
    ctx.advance_patches(g, dd, cons_out=out_w, worklist=torch.as_tensor(wl, device="cuda"),
                        patch_status=st_w, prec=prec)
    torch.cuda.synchronize()
    ow, sw = to_np(out_w), st_w.cpu().numpy()
    mask = np.zeros(N_BATCH, bool)
    mask[wl] = True
    assert np.array_equal(sw[mask], ref_st[idx[mask]])
    assert np.array_equal(ow[mask], ref_out[idx[mask]])
    assert np.all(ow[~mask] == 7.0) and np.all(sw[~mask] == -1)

    # an input 8 (double) or 4 (float) bytes off a 16-byte boundary
    flat = torch.empty(N_BATCH * 5 * 1728 + 1, dtype=dtype, device="cuda")
    g_off = flat[1:].view(N_BATCH, 5, 12, 12, 12)
    g_off.copy_(g)
    assert g_off.data_ptr() % 16 != 0
    out_o, st_o, _ = run(g_off, dd)
    assert np.array_equal(st_o, ref_st[idx])
    assert np.array_equal(out_o, ref_out[idx])
