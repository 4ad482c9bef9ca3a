"""FP64 CPU oracle of the AMR exchange around the per-patch update (test
infrastructure: only tests/, the package's smoke check and bench.py's CPU
baseline use it; it shares no code with the CUDA path or its host-side map
builder).

Section 3.1 of arXiv 2012.11130: the data live in 8^3 patches on levels
l = 0, 1, ... (level l has cells 2^l times finer than level 0); level l
takes two substeps per step of level l - 1; ghost zones of a patch come from
its own level where that level covers them, otherwise from the coarser level
(the ghost-zone passage of Section 3.3); after the fine substeps the coarse
level is replaced by the average of the fine one where refined, and the
coarse cells next to the fine region are corrected with the fine fluxes
(the flux-correction passage of Section 3.3), which makes the composite
update conservative.

Written as the plain definitions: each ghost cell is looked up cell by cell
(same-level patch, else the coarse cell containing it, taken linearly in time
between the coarse states before and after the coarse step: piecewise-constant
prolongation, or, with prolong="linear", the limited linear interpolation of
the conserved variables with the primitive-variable fallback of the
ghost-zone passage of Section 3.3); restriction is the mean of the eight child
cells; the flux correction replaces, for a coarse cell on a coarse-fine face,
the coarse face flux by the mean of the fine face fluxes over the 2x2 fine
faces and the two substeps, and is ignored on a cell that it would leave
unphysical. The per-patch step is oracle.advance_patches.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


class OracleAmr:
    """levels[l]: list of patch coordinates (X, Y, Z) at level l; base: level-0
    patch counts; bc per axis "periodic" | "outflow"; inflow: dict(axis, side,
    center, radius, state) -- ghost cells beyond that face within `radius`
    (level-0 cell units) of `center` take the conserved `state`.
    data[l][(X, Y, Z)] = conserved [5][8][8][8] (z, y, x order)."""

    def __init__(self, base, levels, data, dh0, cfl_dt_factor=0.4, bc=("periodic",) * 3,
                 inflow=None, flux_correction=True, prolong="constant"):
        self.base = tuple(base)
        self.levels = [[tuple(int(v) for v in c) for c in lev] for lev in levels]
        self.data = [{c: np.array(data[l][c], dtype=np.float64) for c in self.levels[l]}
                     for l in range(len(self.levels))]
        self.old = [{c: v.copy() for c, v in d.items()} for d in self.data]
        self.dh0 = dh0
        self.cfl = cfl_dt_factor
        self.bc = bc
        self.inflow = inflow
        self.flux_correction = flux_correction
        self.face_flux = [dict() for _ in self.levels]   # [l][coord] -> list per substep
        self.skipped = 0     # cells whose flux correction was ignored (Section 3.3 (4))
        # ghost cells taken from the coarser level: "constant" (the coarse cell
        # containing the ghost cell) or "linear" (limited linear interpolation
        # of the conserved variables, primitive variables where that is
        # unphysical: Section 3.3 (3))
        assert prolong in ("constant", "linear")
        self.prolong = prolong
        self.prim_fallbacks = 0   # linear ghost cells interpolated in primitive variables

    def ncell(self, l):
        return [8 * (b << l) for b in self.base]

    # -- ghost zones ------------------------------------------------------
    def _value(self, l, x, y, z, w):
        """Conserved state that the ghost fill of level l assigns to level-l
        cell (x, y, z) (may lie outside the domain)."""
        N = self.ncell(l)
        co = [x, y, z]
        if self.inflow is not None:
            a = self.inflow["axis"]
            beyond = co[a] < 0 if self.inflow["side"] == 0 else co[a] >= N[a]
            if beyond:
                t = [b for b in range(3) if b != a]
                s = 2.0 ** -l
                r2 = sum(((co[b] + 0.5) * s - c) ** 2 for b, c in zip(t, self.inflow["center"]))
                if r2 < self.inflow["radius"] ** 2:
                    return np.asarray(self.inflow["state"], dtype=np.float64)
        for a in range(3):
            if co[a] < 0 or co[a] >= N[a]:
                co[a] = co[a] % N[a] if self.bc[a] == "periodic" else min(max(co[a], 0), N[a] - 1)
        x, y, z = co
        key = (x // 8, y // 8, z // 8)
        if key in self.data[l]:
            return self.data[l][key][:, z % 8, y % 8, x % 8]
        assert l > 0, "level 0 must cover the domain"
        xc, yc, zc = x // 2, y // 2, z // 2
        U = self._coarse(l - 1, xc, yc, zc, w)
        assert U is not None, "proper nesting violated"
        if self.prolong == "constant":
            return U
        return self._prolong_linear(l - 1, (xc, yc, zc), (x % 2, y % 2, z % 2), w)

    def _coarse(self, l, x, y, z, w):
        """State of level-l cell (x, y, z) between its level's states before
        (w = 0) and after (w = 1) its step, after the boundary rule (periodic
        wrap, outflow clamp); None where level l does not cover the cell."""
        N = self.ncell(l)
        co = [x, y, z]
        for a in range(3):
            if co[a] < 0 or co[a] >= N[a]:
                co[a] = co[a] % N[a] if self.bc[a] == "periodic" else min(max(co[a], 0), N[a] - 1)
        x, y, z = co
        kc = (x // 8, y // 8, z // 8)
        if kc not in self.data[l]:
            return None
        new = self.data[l][kc][:, z % 8, y % 8, x % 8]
        old = self.old[l][kc][:, z % 8, y % 8, x % 8]
        return (1.0 - w) * old + w * new

    @staticmethod
    def _minmod(a, b):
        """minmod of the one-sided differences (elementwise): the one of
        smaller magnitude if they have the same sign, else 0."""
        return np.where(a * b > 0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)

    def _prolong_linear(self, lc, c, parity, w):
        """Section 3.3 (3): the state of a fine ghost cell in coarse cell c
        (level lc) by limited linear interpolation, the fine cell centre lying
        at a quarter of a coarse cell from the coarse centre along each axis
        (parity 0: below, 1: above). Per axis the slope is the minmod of the
        two one-sided differences of the coarse cell with its neighbours (0
        where a neighbour is not on level lc). The conserved variables are
        interpolated; if the result fails Eq. (Unphysical result), the
        primitive variables (rho, U^x, U^y, U^z, p) of the same coarse cells
        are interpolated instead and converted to conserved variables."""
        x, y, z = c
        Uc = self._coarse(lc, x, y, z, w)
        nb = []
        for d in range(3):
            pair = []
            for s in (-1, 1):
                q = [x, y, z]
                q[d] += s
                pair.append(self._coarse(lc, *q, w))
            nb.append(pair)

        def interp(center, nbs):
            out = center.copy()
            for d in range(3):
                m, p = nbs[d]
                lo = center - m if m is not None else np.zeros(5)
                hi = p - center if p is not None else np.zeros(5)
                out = out + (0.25 if parity[d] else -0.25) * self._minmod(lo, hi)
            return out

        U = interp(Uc, nb)
        if self.physical(U.reshape(5, 1))[0]:
            return U
        self.prim_fallbacks += 1

        def prim(u):
            if u is None:
                return None
            r = O.con2pri(u.reshape(5, 1))
            assert r["status"][0] != O.UNPHYSICAL, "unphysical coarse state"
            return r["prim"][:, 0]
        Wf = interp(prim(Uc), [[prim(m), prim(p)] for m, p in nb])
        C, st = O.prim2con(Wf.reshape(5, 1))
        assert st[0] == 0
        return C[:, 0]

    def ghosted(self, l, c, w):
        X, Y, Z = c
        g = np.empty((5, 12, 12, 12))
        for k in range(12):
            for j in range(12):
                for i in range(12):
                    g[:, k, j, i] = self._value(l, 8 * X + i - 2, 8 * Y + j - 2, 8 * Z + k - 2, w)
        return g

    # -- restriction and flux correction ------------------------------------
    def children(self, l, c):
        X, Y, Z = c
        ch = [(2 * X + (o & 1), 2 * Y + ((o >> 1) & 1), 2 * Z + (o >> 2)) for o in range(8)]
        if l + 1 >= len(self.levels):
            return None
        have = [k in self.data[l + 1] for k in ch]
        return ch if all(have) else None

    def restrict(self, l):
        for c in self.levels[l]:
            ch = self.children(l, c)
            if ch is None:
                continue
            u = self.data[l][c]
            for o, k in enumerate(ch):
                f = self.data[l + 1][k]   # [5][8][8][8]
                m = f.reshape(5, 4, 2, 4, 2, 4, 2).mean(axis=(2, 4, 6))
                cx, cy, cz = o & 1, (o >> 1) & 1, o >> 2
                u[:, 4 * cz:4 * cz + 4, 4 * cy:4 * cy + 4, 4 * cx:4 * cx + 4] = m

    @staticmethod
    def patch_face(flux, d, high):
        """[5][8][8] face flux (a along the lower transverse axis, b the other:
        indexed [v][b][a]) on the low/high face of a patch, from the face fluxes
        [3][5][576] of oracle.advance_patches."""
        fd = 8 if high else 0
        F = flux[d]
        out = np.empty((5, 8, 8))
        for b in range(8):
            for a in range(8):
                if d == 0:
                    q = (b * 8 + a) * 9 + fd          # (k*8 + j)*9 + fd, a = j, b = k
                elif d == 1:
                    q = (b * 9 + fd) * 8 + a          # (k*9 + fd)*8 + i, a = i, b = k
                else:
                    q = (fd * 8 + b) * 8 + a          # (fd*8 + j)*8 + i, a = i, b = j
                out[:, b, a] = F[:, q]
        return out

    @staticmethod
    def physical(u):
        """Eq. (Unphysical result) of conserved states u [5][...]: D > 0 and
        A = eD (eD + 2) - m2 > 2e-16, eD = Etilde/D, m2 = |M|^2/D^2."""
        D = u[0]
        with np.errstate(divide="ignore", invalid="ignore"):
            m2 = (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / (D * D)
            eD = u[4] / D
            A = eD * (eD + 2.0) - m2
        return (D > 0) & (A > 2e-16)

    def flux_correct(self, l, coarse_flux):
        """Correct the unrefined coarse patches of level l next to level
        l + 1; a cell whose corrected state fails Eq. (Unphysical result)
        keeps its uncorrected state (Section 3.3 (4)) and is counted in
        self.skipped."""
        P = [b << l for b in self.base]
        dt, dh = self.cfl * self.dh0 / 2 ** l, self.dh0 / 2 ** l
        for c in self.levels[l]:
            if self.children(l, c) is not None:
                continue
            u0 = self.data[l][c]
            u = u0.copy()
            touched = np.zeros((8, 8, 8), bool)
            for d in range(3):
                for high in (0, 1):
                    q = list(c)
                    q[d] += 1 if high else -1
                    if q[d] < 0 or q[d] >= P[d]:
                        if self.bc[d] != "periodic":
                            continue
                        q[d] %= P[d]
                    q = tuple(q)
                    if q not in self.data[l] or self.children(l, q) is None:
                        continue
                    t = [a for a in range(3) if a != d]
                    fine_mean = np.zeros((5, 8, 8))
                    for qb in range(2):
                        for qa in range(2):
                            ch = [2 * v for v in q]
                            ch[d] += 0 if high else 1
                            ch[t[0]] += qa
                            ch[t[1]] += qb
                            for sub in self.face_flux[l + 1][tuple(ch)]:
                                F = self.patch_face(sub, d, not high)  # [5][b][a], fine
                                m = F.reshape(5, 4, 2, 4, 2).mean(axis=(2, 4))
                                fine_mean[:, 4 * qb:4 * qb + 4, 4 * qa:4 * qa + 4] += m / 2
                    Fc = self.patch_face(coarse_flux[c], d, high)
                    du = (dt / dh) * (Fc - fine_mean)
                    e = 7 if high else 0
                    sl = [slice(None)] * 3      # (z, y, x)
                    sl[2 - d] = e
                    view = u[(slice(None),) + tuple(sl)]   # [5][.][.] over the two transverse axes
                    # view axes: for d=0 (z, y) = (b, a); d=1 (z, x) = (b, a); d=2 (y, x) = (b, a)
                    if high:
                        view += du
                    else:
                        view -= du
                    touched[tuple(sl)] = True
            # Section 3.3 (4): the correction is ignored on cells it leaves
            # unphysical
            bad = touched & ~self.physical(u)
            u[:, bad] = u0[:, bad]
            self.skipped += int(bad.sum())
            u0[...] = u

    # -- time stepping --------------------------------------------------------
    def _advance(self, l, w):
        coords = self.levels[l]
        dt, dh = self.cfl * self.dh0 / 2 ** l, self.dh0 / 2 ** l
        G = np.stack([self.ghosted(l, c, w) for c in coords])
        r = O.advance_patches(G, np.tile([dt, dh], (len(coords), 1)), want_flux=True)
        for c in coords:
            self.old[l][c] = self.data[l][c].copy()
        for n, c in enumerate(coords):
            self.data[l][c] = r["out"][n].copy()
            self.face_flux[l].setdefault(c, []).append(r["flux"][n])
        coarse_flux = {c: r["flux"][n] for n, c in enumerate(coords)}
        if l + 1 < len(self.levels) and self.levels[l + 1]:
            for c in self.levels[l + 1]:
                self.face_flux[l + 1][c] = []
            self._advance(l + 1, 0.0)
            self._advance(l + 1, 0.5)
            self.restrict(l)
            if self.flux_correction:
                self.flux_correct(l, coarse_flux)
        return r["status"]

    def step(self):
        for c in self.levels[0]:
            self.face_flux[0][c] = []
        self._advance(0, 0.0)

    def totals(self):
        """Level-0 sums of D, M, Etilde times the cell volume."""
        v = self.dh0 ** 3
        return sum(u.reshape(5, -1).sum(axis=1) for u in self.data[0].values()) * v
