"""Batched AMR driver: many 8^3 patches of uneven refinement level through
one persistent srhd_advance_patches launch per level substep.

A hierarchy is given as per-level lists of ghosted patches (all in one
[npatch][5][12^3] batch on the device). One coarse step advances level l
2^l times with its own (dt, dh) (Section 3.1-3.2: level l has a 2^l times
finer cell and takes 2^l substeps), i.e. sum_l 2^l launches, each processing
the level's worklist. The launches of a coarse step contain no host
synchronisation and no allocation, so the step can be captured once into a
CUDA graph and replayed. Ghost zones are static here (the caller fills them
once); exchanging them between substeps is the AMR layer above this path.
"""
from __future__ import annotations

import torch

from . import srhd as S


class AmrBatch:
    def __init__(self, ctx: S.Context, cons_ghosted: torch.Tensor, level_counts, dh0: float,
                 cfl_dt_factor: float = 0.4, prec: str | None = None):
        """cons_ghosted: [npatch][5][12][12][12] on the device, level 0 patches
        first, then level 1, ...; level_counts: patches per level; dh0: cell
        size of level 0; each level steps with dt_l = cfl_dt_factor * dh_l."""
        self.ctx = ctx
        self.prec = prec
        self.G = cons_ghosted
        dev = cons_ghosted.device
        self.counts = [int(n) for n in level_counts]
        assert sum(self.counts) == cons_ghosted.shape[0]
        self.nlev = len(self.counts)
        self.out = torch.empty((cons_ghosted.shape[0], 5, 8, 8, 8), dtype=cons_ghosted.dtype,
                               device=dev)
        self.status = torch.zeros(cons_ghosted.shape[0], dtype=torch.int32, device=dev)
        self.dt_next = torch.empty(self.nlev, dtype=torch.float64, device=dev)
        dd = torch.empty((cons_ghosted.shape[0], 2), dtype=torch.float64, device=dev)
        self.worklists = []
        off = 0
        for l, n in enumerate(self.counts):
            dh = dh0 / 2 ** l
            dd[off:off + n, 0] = cfl_dt_factor * dh
            dd[off:off + n, 1] = dh
            self.worklists.append(torch.arange(off, off + n, dtype=torch.int32, device=dev))
            off += n
        self.dt_dh = dd
        self.graph = None

    @property
    def launches_per_step(self) -> int:
        return sum(2 ** l for l in range(self.nlev))

    @property
    def cell_updates_per_step(self) -> int:
        return sum(n * 512 * 2 ** l for l, n in enumerate(self.counts))

    def step(self, stream=None):
        """One coarse step: every level substep is one fused launch over the
        level's worklist; the fused CFL minimum of level l goes to dt_next[l]."""
        for l, n in enumerate(self.counts):
            if n == 0:
                continue
            for _ in range(2 ** l):
                self.ctx.advance_patches(self.G, self.dt_dh, cons_out=self.out,
                                         worklist=self.worklists[l], npatch=n,
                                         dt_next=self.dt_next[l:l + 1],
                                         patch_status=self.status, stream=stream, prec=self.prec)

    def capture(self, warmup: int = 2):
        """Record one coarse step into a CUDA graph (after eager warm-ups on
        the capture stream)."""
        s = torch.cuda.Stream(device=self.G.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()


def blast_batch(ctx: S.Context, prec: str = "mixed_cf", base: int = 64, levels: int = 5,
                device="cuda", **hier):
    """The off-centre blast hierarchy of workloads.amr_blast_hierarchy with
    its ghosted inputs converted on the device (srhd_prim2con in FP64, then
    stored in the precision's type)."""
    from . import workloads as W
    lev = W.amr_blast_hierarchy(base=base, levels=levels, **hier)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    parts = []
    for l, coords in enumerate(lev):
        for a in range(0, len(coords), 4096):
            Wp = W.amr_patch_prims(coords[a:a + 4096], l, base=base, xp=torch, device=device)
            n = Wp.shape[0]
            C = ctx.prim2con(Wp.permute(1, 0, 2, 3, 4).reshape(5, -1).contiguous())
            parts.append(C.reshape(5, n, 12, 12, 12).permute(1, 0, 2, 3, 4).to(dtype))
    G = torch.cat(parts).contiguous()
    return AmrBatch(ctx, G, [len(c) for c in lev], 1.0 / base, prec=prec), lev
