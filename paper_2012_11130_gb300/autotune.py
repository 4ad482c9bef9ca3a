"""Autotuner of the fused patch kernel's launch variant.

Each precision has kPatchVariants instantiations of the patch kernel that
differ in threads per CTA, CTAs per SM and in whether a thread runs one or
two Newton solves in lockstep (include/srhd.h, srhd_params.patch_variant).
Which is fastest depends on the workload (Newton iteration counts, retry
rate, batch size), so the tuner times every variant on the caller's own
batch (CUDA events, after warm-up) and returns the fastest. Results are
cached per (device, precision, batch size) for the life of the process.
"""
from __future__ import annotations

import dataclasses

import torch

from . import srhd as S

N_VARIANTS = 4
_cache: dict = {}


def time_variant(params: S.Params, cons_ghosted, dt_dh, prec=None, steps: int = 3,
                 warmup: int = 1, worklist=None, npatch=None) -> float:
    """Mean milliseconds of one srhd_advance_patches launch (with the fused
    CFL) in the variant params.patch_variant."""
    ctx = S.Context(params)
    n = cons_ghosted.shape[0]
    out = torch.empty((n, 5, 8, 8, 8), dtype=cons_ghosted.dtype, device=cons_ghosted.device)
    dn = torch.empty(1, dtype=torch.float64, device=cons_ghosted.device)
    kw = dict(cons_out=out, dt_next=dn, prec=prec, worklist=worklist, npatch=npatch)
    for _ in range(warmup):
        ctx.advance_patches(cons_ghosted, dt_dh, **kw)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.advance_patches(cons_ghosted, dt_dh, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.close()
    return e0.elapsed_time(e1) / steps


def tune(cons_ghosted, dt_dh, prec=None, params: S.Params | None = None, steps: int = 3,
         warmup: int = 1, variants=range(N_VARIANTS)):
    """Returns (best Params, {variant: ms}). The best Params equal `params`
    with patch_variant set to the fastest variant."""
    params = params or S.Params()
    key = (torch.cuda.get_device_name(cons_ghosted.device), prec or str(cons_ghosted.dtype),
           cons_ghosted.shape[0], dataclasses.astuple(dataclasses.replace(params, patch_variant=0)))
    if key in _cache:
        return _cache[key]
    times = {}
    for v in variants:
        p = dataclasses.replace(params, patch_variant=v)
        times[v] = time_variant(p, cons_ghosted, dt_dh, prec, steps, warmup)
    best = min(times, key=times.get)
    res = (dataclasses.replace(params, patch_variant=best), times)
    _cache[key] = res
    return res
