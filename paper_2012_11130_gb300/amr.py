"""Batched AMR drivers: many 8^3 patches of uneven refinement level through
one persistent srhd_advance_patches launch per level substep.

AmrBatch: a hierarchy given as per-level lists of ghosted patches (all in one
[npatch][5][12^3] batch on the device) with static ghost zones. One coarse
step advances level l 2^l times with its own (dt, dh) (Section 3.1-3.2: level
l has a 2^l times finer cell and takes 2^l substeps), i.e. sum_l 2^l
launches, each processing the level's worklist.

Hierarchy + AmrRun: the same with the data exchange between levels on the
GPU (srhd_amr_fill_ghosts, srhd_amr_restrict, srhd_amr_flux_correct), the
maps built here on the host from the patch coordinates.

The launches of a coarse step contain no host synchronisation and no
allocation, so a step can be captured once into a CUDA graph and replayed.
"""
from __future__ import annotations

import numpy as np
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


# ---- hierarchy with ghost exchange, restriction and flux correction --------
# Section 3.1: levels of 8^3 patches, level l with cells 2^l times finer than
# level 0, advanced with two substeps per step of level l - 1. A level is
# refined in groups of eight patches (the 2x2x2 children of a coarser patch),
# and every level-l patch has its ghost zones covered by level l or l - 1
# (proper nesting). The maps below tell the srhd_amr_* calls where each ghost
# cell, restricted cell and corrected face takes its data from.

class Hierarchy:
    """Static patch hierarchy and its data maps.

    base: level-0 patch counts (px, py, pz); levels[l]: int array (n_l, 3) of
    patch coordinates at level l (a level-l patch covers cells 8X..8X+7);
    bc: per-axis "periodic" or "outflow"; inflow: optional dict(axis, side,
    center, radius, index) giving the special-state index used for ghost
    cells beyond that domain face within `radius` (in level-0 cell units) of
    `center` (the two transverse coordinates, level-0 cell units); those cells
    take special state `index` instead of the outflow copy.
    Patches are numbered level by level in the given order.
    prolong: how a level takes the ghost cells that lie on the coarser level:
    "constant" (map entries with SRHD_AMR_COARSE: the coarse cell containing
    the ghost cell) or "linear" (Section 3.3 (3): limited linear
    interpolation with the primitive-variable fallback, srhd_amr_prolong).
    With "linear", every distinct such ghost cell of level l is a row of
    prolong_tables[l] ([rows][8] int32, the format of srhd_amr_prolong) and
    the map entries that read it are special states nspecial +
    prolong_offsets[l] + row: the caller's special array holds its nspecial
    fixed states (inflow) followed by the prolongation rows of all levels,
    which srhd_amr_prolong rewrites before each substep of the level.
    """

    def __init__(self, base, levels, bc=("periodic",) * 3, inflow=None, prolong="constant",
                 nspecial=None):
        if prolong not in ("constant", "linear"):
            raise ValueError("prolong must be 'constant' or 'linear'")
        self.prolong = prolong
        self.nspecial = (int(nspecial) if nspecial is not None else
                         (int(inflow["index"]) + 1 if inflow is not None else 0))
        self.prolong_tables = []
        self.prolong_offsets = []
        self._prolong_rows = 0
        self.base = tuple(int(b) for b in base)
        self.coords = [np.asarray(c, dtype=np.int64).reshape(-1, 3) for c in levels]
        self.nlev = len(self.coords)
        self.counts = [len(c) for c in self.coords]
        self.offsets = list(np.cumsum([0] + self.counts[:-1]))
        self.ntotal = int(sum(self.counts))
        self.bc = tuple(bc)
        self.inflow = inflow
        self.grids = []
        for l, c in enumerate(self.coords):
            g = np.full(tuple(b << l for b in self.base)[::-1], -1, dtype=np.int64)  # [z][y][x]
            if len(c):
                if np.any(c < 0) or np.any(c >= np.array([b << l for b in self.base])):
                    raise ValueError(f"level {l}: patch outside the domain")
                if len(np.unique(c, axis=0)) != len(c):
                    raise ValueError(f"level {l}: duplicate patches")
                g[c[:, 2], c[:, 1], c[:, 0]] = self.offsets[l] + np.arange(len(c))
            self.grids.append(g)
        self.map = np.concatenate([self._level_map(l) for l in range(self.nlev)]).astype(np.int32)
        self.children = [self._children(l) for l in range(self.nlev)]
        self.faces = [self._faces(l) for l in range(self.nlev)]

    def cells(self, l):
        return tuple(8 * (b << l) for b in self.base)

    def _level_map(self, l):
        c = self.coords[l]
        n = len(c)
        if n == 0:
            if self.prolong == "linear":
                self.prolong_offsets.append(self._prolong_rows)
                self.prolong_tables.append(np.zeros((0, 8), np.int32))
            return np.zeros((0, 1728), np.int64)
        N = self.cells(l)
        g = np.arange(12) - 2
        # tile cell (k, j, i) -> level-l cell coordinates, arrays [n][12][12][12]
        x = (8 * c[:, 0])[:, None, None, None] + g[None, None, None, :]
        y = (8 * c[:, 1])[:, None, None, None] + g[None, None, :, None]
        z = (8 * c[:, 2])[:, None, None, None] + g[None, :, None, None]
        x, y, z = np.broadcast_arrays(x, y, z)
        x, y, z = x.copy(), y.copy(), z.copy()
        special = np.full(x.shape, -1, dtype=np.int64)
        if self.inflow is not None:
            ax, side = self.inflow["axis"], self.inflow["side"]
            co = (x, y, z)
            beyond = co[ax] < 0 if side == 0 else co[ax] >= N[ax]
            t = [a for a in range(3) if a != ax]
            s = 2.0 ** -l
            r2 = sum(((co[a] + 0.5) * s - cen) ** 2 for a, cen in zip(t, self.inflow["center"]))
            special[beyond & (r2 < self.inflow["radius"] ** 2)] = self.inflow["index"]
        for a, arr in enumerate((x, y, z)):
            if self.bc[a] == "periodic":
                arr %= N[a]
            else:
                np.clip(arr, 0, N[a] - 1, out=arr)
        cell = ((z % 8) * 8 + (y % 8)) * 8 + (x % 8)
        idx = self.grids[l][z // 8, y // 8, x // 8]
        src = np.where(idx >= 0, idx * 512 + cell, -1)
        need = (idx < 0) & (special < 0)
        if np.any(need):
            if l == 0:
                raise ValueError("level 0 must cover the domain")
            xc, yc, zc = x[need] // 2, y[need] // 2, z[need] // 2
            ic = self.grids[l - 1][zc // 8, yc // 8, xc // 8]
            if np.any(ic < 0):
                raise ValueError(f"level {l}: ghost zones not covered by level {l - 1} "
                                 "(proper nesting violated)")
            cc = ((zc % 8) * 8 + (yc % 8)) * 8 + (xc % 8)
            if self.prolong == "constant":
                src[need] = (ic * 512 + cc) | (1 << 30)
            else:
                rows, which = self._prolong_table(l, x[need], y[need], z[need])
                src[need] = -1 - (self.nspecial + self._prolong_rows + which)
                self.prolong_offsets.append(self._prolong_rows)
                self.prolong_tables.append(rows)
                self._prolong_rows += len(rows)
        if self.prolong == "linear" and len(self.prolong_tables) <= l:
            self.prolong_offsets.append(self._prolong_rows)
            self.prolong_tables.append(np.zeros((0, 8), np.int32))
        out = np.where(special >= 0, -1 - special, src)
        return out.reshape(n, 1728)

    def _coarse_flat(self, l, x, y, z):
        """Flat index patch * 512 + cell of level-l cells (x, y, z) after the
        boundary rule (periodic wrap, outflow clamp), -1 where level l does
        not cover the cell."""
        N = self.cells(l)
        co = [np.array(v, dtype=np.int64) for v in (x, y, z)]
        for a in range(3):
            if self.bc[a] == "periodic":
                co[a] %= N[a]
            else:
                np.clip(co[a], 0, N[a] - 1, out=co[a])
        x, y, z = co
        idx = self.grids[l][z // 8, y // 8, x // 8]
        cell = ((z % 8) * 8 + (y % 8)) * 8 + (x % 8)
        return np.where(idx >= 0, idx * 512 + cell, -1)

    def _prolong_table(self, l, x, y, z):
        """Rows of srhd_amr_prolong for the level-l ghost cells (x, y, z)
        (boundary rule already applied) taken from level l - 1, one row per
        distinct cell; returns (rows [m][8] int32, row of each input cell)."""
        # rows ordered by (z, y, x), so that neighbouring rows read
        # neighbouring coarse cells
        key = np.stack([z, y, x], axis=1)
        uniq, which = np.unique(key, axis=0, return_inverse=True)
        zf, yf, xf = uniq[:, 0], uniq[:, 1], uniq[:, 2]
        xc, yc, zc = xf // 2, yf // 2, zf // 2
        rows = np.empty((len(uniq), 8), np.int64)
        rows[:, 0] = self._coarse_flat(l - 1, xc, yc, zc)
        for k, (dx, dy, dz) in enumerate(((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                                          (0, 0, -1), (0, 0, 1))):
            rows[:, 1 + k] = self._coarse_flat(l - 1, xc + dx, yc + dy, zc + dz)
        rows[:, 7] = (xf % 2) | ((yf % 2) << 1) | ((zf % 2) << 2)
        assert np.all(rows[:, 0] >= 0)
        return rows.astype(np.int32), which.reshape(-1)

    def _child_index(self, l, X, Y, Z):
        g = self.grids[l + 1]
        return g[Z, Y, X]

    def _children(self, l):
        if l + 1 >= self.nlev or self.counts[l + 1] == 0:
            return np.zeros((0, 9), np.int32)
        rows = []
        for r, (X, Y, Z) in enumerate(self.coords[l]):
            ch = [self._child_index(l, 2 * X + (o & 1), 2 * Y + ((o >> 1) & 1),
                                    2 * Z + (o >> 2)) for o in range(8)]
            if all(v < 0 for v in ch):
                continue
            if any(v < 0 for v in ch):
                raise ValueError(f"level {l + 1} must be refined in groups of 8 children")
            rows.append([self.offsets[l] + r] + ch)
        return np.asarray(rows, np.int32).reshape(-1, 9)

    def _refined(self, l, X, Y, Z):
        return self._child_index(l, 2 * X, 2 * Y, 2 * Z) >= 0

    def _faces(self, l):
        if l + 1 >= self.nlev or self.counts[l + 1] == 0:
            return np.zeros((0, 25), np.int32)
        P = [b << l for b in self.base]
        rows = []
        for r, pc in enumerate(self.coords[l]):
            if self._refined(l, *pc):
                continue
            row = [self.offsets[l] + r] + [-1] * 24
            hit = False
            for f in range(6):
                d, high = f >> 1, f & 1
                q = list(pc)
                q[d] += 1 if high else -1
                if q[d] < 0 or q[d] >= P[d]:
                    if self.bc[d] != "periodic":
                        continue
                    q[d] %= P[d]
                if self.grids[l][q[2], q[1], q[0]] < 0 or not self._refined(l, *q):
                    continue
                ta, tb = [a for a in range(3) if a != d]
                for qa in range(2):
                    for qb in range(2):
                        ch = [2 * v for v in q]
                        ch[d] += 0 if high else 1
                        ch[ta] += qa
                        ch[tb] += qb
                        row[1 + 4 * f + qa + 2 * qb] = int(self._child_index(l, *ch))
                hit = True
            if hit:
                rows.append(row)
        return np.asarray(rows, np.int32).reshape(-1, 25)


class AmrRun:
    """Advance a Hierarchy on the GPU: one coarse step advances level l
    2^l times (dt_l = cfl_dt_factor * dh_l), each substep = a copy of the
    level's state (for the finer levels' time interpolation) and one fused
    launch over the level's patches that reads each tile through the source
    map (srhd_advance_amr; with fused=False a separate ghost fill into a
    ghosted batch and srhd_advance_patches, which give the same bits), and
    after the two substeps of level l + 1 the restriction of l + 1 onto l and
    the coarse-fine flux correction of l. With a hierarchy built with
    prolong="linear", each substep of a level l >= 1 first computes the
    level's coarse-sourced ghost cells by srhd_amr_prolong (counting the
    primitive-variable fallbacks in prolong_fallbacks). A coarse step has no host
    synchronisation or allocation and can be captured into a CUDA graph
    (capture / replay)."""

    def __init__(self, ctx: S.Context, hier: Hierarchy, cons0: torch.Tensor, dh0: float,
                 cfl_dt_factor: float = 0.4, prec: str | None = None, special=None,
                 fused: bool = True):
        self.ctx, self.h, self.prec = ctx, hier, prec
        dev = cons0.device
        dt = cons0.dtype
        n = hier.ntotal
        assert cons0.shape == (n, 5, 8, 8, 8)
        self.fused = fused
        self.cur = cons0.clone()
        self.prev = cons0.clone()
        self.ghosted = (None if fused else
                        torch.zeros((n, 5, 12, 12, 12), dtype=dt, device=dev))
        self.flux = [torch.zeros((n, 6, 5, 64), dtype=dt, device=dev) for _ in range(2)]
        self.status = torch.zeros(n, dtype=torch.int32, device=dev)
        # cells whose flux correction was skipped because it left them
        # unphysical (Section 3.3 (4)), summed over all steps so far
        self.skipped = torch.zeros(1, dtype=torch.int32, device=dev)
        self.map = torch.from_numpy(hier.map).to(dev)
        self.children = [torch.from_numpy(c).to(dev) for c in hier.children]
        self.faces = [torch.from_numpy(f).to(dev) for f in hier.faces]
        self.special = None if special is None else special.to(device=dev, dtype=dt).contiguous()
        # limited linear prolongation (Section 3.3 (3)): the special-state
        # array holds the fixed states, then one row per coarse-sourced ghost
        # cell of every level, rewritten by srhd_amr_prolong before each
        # substep of the level
        self.prolong_tables = None
        self.prolong_fallbacks = torch.zeros(1, dtype=torch.int32, device=dev)
        if hier.prolong == "linear":
            nfix = hier.nspecial
            if nfix and (self.special is None or self.special.shape[0] < nfix):
                raise ValueError(f"the hierarchy's maps use {nfix} fixed special states")
            rows = sum(len(t) for t in hier.prolong_tables)
            sp = torch.zeros((nfix + rows, 5), dtype=dt, device=dev)
            if nfix:
                sp[:nfix] = self.special[:nfix]
            self.special = sp
            self.prolong_tables = [torch.from_numpy(t).to(dev) for t in hier.prolong_tables]
        dd = torch.empty((n, 2), dtype=torch.float64)
        for l in range(hier.nlev):
            o, c = hier.offsets[l], hier.counts[l]
            dh = dh0 / 2 ** l
            dd[o:o + c, 0] = cfl_dt_factor * dh
            dd[o:o + c, 1] = dh
        self.dt_dh = dd.to(dev)
        self.worklists = [torch.arange(o, o + c, dtype=torch.int32, device=dev)
                          for o, c in zip(hier.offsets, hier.counts)]
        self.graph = None
        self.timer = None   # optional list of (event, event) pairs around the updates

    @property
    def cell_updates_per_step(self) -> int:
        return sum(c * 512 * 2 ** l for l, c in enumerate(self.h.counts))

    @property
    def launches_per_step(self) -> int:
        return sum(2 ** l for l, c in enumerate(self.h.counts) if c)

    def _advance(self, l, w, parity, stream):
        h, ctx = self.h, self.ctx
        o, c = h.offsets[l], h.counts[l]
        if self.prolong_tables is not None and len(self.prolong_tables[l]):
            r0 = h.nspecial + h.prolong_offsets[l]
            nr = len(self.prolong_tables[l])
            ctx.amr_prolong(self.cur, self.prev, self.prolong_tables[l],
                            self.special[r0:r0 + nr], w=w, fallbacks=self.prolong_fallbacks,
                            stream=stream, prec=self.prec)
        if not self.fused:
            ctx.amr_fill_ghosts(self.cur, self.prev, self.ghosted, self.map, o, c, w,
                                self.special, stream=stream, prec=self.prec)
        self.prev[o:o + c].copy_(self.cur[o:o + c])
        ev = None
        if self.timer is not None:
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record()
        if self.fused:
            # same-level sources from prev (the level's state before this
            # substep), coarse ones interpolated between the coarser level's
            # states before (prev) and after (cur) its step
            ctx.advance_amr(self.prev, self.prev, self.cur, self.map, self.dt_dh, self.cur, w=w,
                            special=self.special, patch_face_flux=self.flux[parity],
                            worklist=self.worklists[l], npatch=c, patch_status=self.status,
                            stream=stream, prec=self.prec)
        else:
            ctx.advance_patches(self.ghosted, self.dt_dh, cons_out=self.cur,
                                patch_face_flux=self.flux[parity], worklist=self.worklists[l],
                                npatch=c, patch_status=self.status, stream=stream,
                                prec=self.prec)
        if ev is not None:
            ev[1].record()
            self.timer.append(ev)
        if l + 1 < h.nlev and h.counts[l + 1]:
            self._advance(l + 1, 0.0, 0, stream)
            self._advance(l + 1, 0.5, 1, stream)
            ctx.amr_restrict(self.cur, self.children[l], stream=stream, prec=self.prec)
            ctx.amr_flux_correct(self.cur, self.flux[parity], self.flux[0], self.flux[1],
                                 self.faces[l], self.dt_dh, stream=stream, prec=self.prec,
                                 skipped=self.skipped)

    def step(self, stream=None):
        """One coarse step (every level advanced by dt_0), on `stream` (or the
        current stream)."""
        if stream is not None:
            with torch.cuda.stream(stream):
                self._advance(0, 0.0, 0, None)
        else:
            self._advance(0, 0.0, 0, None)

    def capture(self, warmup: int = 1):
        s = torch.cuda.Stream(device=self.cur.device)
        s.wait_stream(torch.cuda.current_stream())
        saved = (self.cur.clone(), self.prev.clone())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.cur.copy_(saved[0])
        self.prev.copy_(saved[1])
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
