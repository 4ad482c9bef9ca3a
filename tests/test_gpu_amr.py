"""Batched AMR on the GPU: a small off-centre blast hierarchy (3 levels of
uneven size) through one fused launch per level substep. The CUDA-graph
replay of a coarse step equals the eager launches bitwise, and sampled
patches of every level equal the oracle's step from the same inputs; the
same sampled check on the full-size blast the benchmark times."""
import numpy as np
import pytest

from gpu_common import cons_rel_err, require_gpu, to_dev, to_np, torch_dtype
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu


def _hierarchy(oracle, prec):
    lev = workloads.amr_blast_hierarchy(base=32, levels=3, widths=(0.06, 0.03))
    parts = []
    for l, coords in enumerate(lev):
        Wp = workloads.amr_patch_prims(coords, l, base=32)
        n = Wp.shape[0]
        C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
        assert np.all(st == 0)
        parts.append(C.reshape(5, n, 12, 12, 12).transpose(1, 0, 2, 3, 4))
    G = np.concatenate(parts)
    if prec != "fp64":
        G = G.astype(np.float32).astype(np.float64)
    return lev, G


@pytest.mark.parametrize("prec", ["mixed_cf", "fp64"])
def test_amr_graph_equals_eager_and_oracle(oracle, prec):
    torch, srhd = require_gpu()
    from paper_2012_11130_gb300 import amr
    lev, G = _hierarchy(oracle, prec)
    counts = [len(c) for c in lev]
    assert counts[0] == 64 and len(set(counts)) == 3
    ctx = srhd.Context(srhd.Params())
    batch = amr.AmrBatch(ctx, to_dev(torch, G, torch_dtype(torch, prec)), counts, 1.0 / 32,
                         prec=prec)
    assert batch.launches_per_step == 7
    batch.step()
    torch.cuda.synchronize()
    eager = to_np(batch.out).copy()
    dt_eager = batch.dt_next.cpu().numpy().copy()
    st_eager = batch.status.cpu().numpy().copy()
    assert np.all((st_eager >> 8) == 0)
    batch.out.fill_(0)
    batch.dt_next.fill_(0)
    batch.capture()
    batch.replay()
    torch.cuda.synchronize()
    assert np.array_equal(to_np(batch.out), eager)
    assert np.array_equal(batch.dt_next.cpu().numpy(), dt_eager)
    # every patch against the oracle, and the per-level CFL minimum of the
    # updated state (C dh_l / S_max over the level's cells)
    dd = batch.dt_dh.cpu().numpy()
    ref = oracle.advance_patches(G, dd)
    assert np.all(ref["status"] == 0)
    # the sharp shell of the coarse levels makes some patches retry with a
    # smaller limiter coefficient (Section 3.3 (1)); in FP64 the GPU takes
    # the same retries, and every patch whose retry count matches agrees
    same = (st_eager & 255) == ref["retries"]
    if prec == "fp64":
        assert same.all(), (st_eager[~same], ref["retries"][~same])
    assert same.mean() > 0.97
    err = cons_rel_err(eager[same].transpose(1, 0, 2, 3, 4),
                       ref["out"][same].transpose(1, 0, 2, 3, 4))
    # FP64: 1e-12, relaxed to 1e-10 on a patch recomputed after a retry (its
    # discontinuous data amplify rounding differences); mixed: 1e-5
    retried = ref["retries"][same] > 0
    tol = np.where(retried, 1e-10, 1e-12) if prec == "fp64" else 1e-5
    assert np.all(err.reshape(-1, 512).max(axis=1) <= tol), err.max()
    off = np.cumsum([0] + counts)
    for l in range(3):
        if not same[off[l]:off[l + 1]].all():
            continue
        cells = ref["out"][off[l]:off[l + 1]].transpose(1, 0, 2, 3, 4).reshape(5, -1)
        want = oracle.cfl_dt(cells, 1.0 / 32 / 2 ** l)
        assert abs(dt_eager[l] / want - 1) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["mixed_cf", "fp64"])
def test_full_size_blast_step_sampled(oracle, prec):
    # The batched AMR blast the benchmark times (5 levels, base 64^3, about
    # 38 000 patches, 31 fused launches per coarse step): one coarse step,
    # then sampled patches of every level recomputed by the oracle from the
    # same ghosted inputs (each level's last substep wrote the output).
    torch, srhd = require_gpu()
    from paper_2012_11130_gb300 import amr
    ctx = srhd.Context(srhd.Params())
    batch, lev = amr.blast_batch(ctx, prec=prec)
    assert batch.launches_per_step == 31 and sum(batch.counts) > 30000
    batch.step()
    torch.cuda.synchronize()
    st = batch.status.cpu().numpy()
    assert np.all((st >> 8) == 0)
    rng = np.random.default_rng(4)
    off = np.cumsum([0] + batch.counts)
    pick = np.concatenate([off[l] + rng.choice(batch.counts[l], min(6, batch.counts[l]),
                                               replace=False) for l in range(batch.nlev)])
    idx = torch.as_tensor(pick, device="cuda")
    G = to_np(batch.G[idx]).astype(np.float64)
    dd = batch.dt_dh[idx].cpu().numpy()
    ref = oracle.advance_patches(G, dd)
    same = (st[pick] & 255) == ref["retries"]
    if prec == "fp64":
        assert same.all()
    got = to_np(batch.out[idx])
    err = cons_rel_err(got[same].transpose(1, 0, 2, 3, 4), ref["out"][same].transpose(1, 0, 2, 3, 4))
    retried = ref["retries"][same] > 0
    tol = np.where(retried, 1e-10, 1e-12) if prec == "fp64" else 1e-5
    assert np.all(err.reshape(-1, 512).max(axis=1) <= tol), err.max()
