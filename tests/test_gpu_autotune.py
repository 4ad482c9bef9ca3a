"""The launch variants of the fused patch kernel compute the same step
(same per-cell arithmetic; only the thread mapping differs), and the
autotuner returns one of them with its timings."""
import numpy as np
import pytest

from gpu_common import cons_rel_err, require_gpu, to_dev, to_np, torch_dtype
from paper_2012_11130_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["mixed_cf", "mixed", "fp64"])
def test_variants_agree_and_tuner_picks_one(oracle, prec):
    torch, srhd = require_gpu()
    from paper_2012_11130_gb300 import autotune
    npatch = 200
    Wp = workloads.rough_patch_prims(npatch, seed=8, spread=0.5, lg_gamma_max=1.0)
    C, st = oracle.prim2con(Wp.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    C = C.reshape(5, npatch, 12, 12, 12).transpose(1, 0, 2, 3, 4).copy()
    g = to_dev(torch, C, torch_dtype(torch, prec))
    dd = torch.tensor([[2e-4, 1 / 64]] * npatch, dtype=torch.float64, device="cuda")
    outs, stats = [], []
    for v in range(autotune.N_VARIANTS):
        ctx = srhd.Context(srhd.Params(patch_variant=v))
        s = torch.empty(npatch, dtype=torch.int32, device="cuda")
        outs.append(to_np(ctx.advance_patches(g, dd, patch_status=s, prec=prec)))
        stats.append(s.cpu().numpy())
    # identical per-cell arithmetic up to the compiler's FMA contraction in
    # the paired code; retried rough patches amplify that rounding
    for o, s in zip(outs[1:], stats[1:]):
        assert np.array_equal(s, stats[0])
        err = cons_rel_err(o.transpose(1, 0, 2, 3, 4), outs[0].transpose(1, 0, 2, 3, 4))
        assert err.max() <= (1e-10 if prec == "fp64" else 1e-5), err.max()
    best, times = autotune.tune(g, dd, prec=prec, steps=2)
    assert best.patch_variant in times and len(times) == autotune.N_VARIANTS
    assert all(t > 0 for t in times.values())
    with pytest.raises(Exception, match="patch_variant"):
        srhd.Context(srhd.Params(patch_variant=autotune.N_VARIANTS))
