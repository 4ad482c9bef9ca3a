"""CPU pins of the AMR exchange oracle (oracle/amr_oracle.py) and CPU checks
of the host-side map builder (paper_2012_11130_gb300/amr.py Hierarchy).

Pins (against what the method fixes, not against the oracle itself):
* a hierarchy whose level 1 covers the whole domain evolves level 1 exactly
  like the uniform grid at that resolution, and level 0 becomes its
  restriction (Section 3.1: the coarse level is the average of the fine one);
* with restriction and flux correction the composite update conserves D, M
  and Etilde to round-off on a periodic domain; without the flux correction
  it does not (the correction is what makes it conservative);
* a uniform state stays bitwise uniform on every level.
"""
import numpy as np
import pytest

from oracle import amr_oracle
from paper_2012_11130_gb300 import workloads as Wk
from paper_2012_11130_gb300.amr import Hierarchy

DH0 = 1.0 / 32


def _level_data(oracle, lev, fn, dh0):
    data = []
    for l, coords in enumerate(lev):
        W = Wk.level_prims(coords, l, fn, dh0)
        C, st = oracle.prim2con(W.transpose(1, 0, 2, 3, 4).reshape(5, -1))
        assert np.all(st == 0)
        C = C.reshape(5, len(coords), 8, 8, 8).transpose(1, 0, 2, 3, 4)
        data.append({tuple(c): C[n] for n, c in enumerate(coords)})
    return data


def _consistent(amr):
    """Make every coarse cell the restriction of the finer level (t = 0)."""
    for l in range(len(amr.levels) - 2, -1, -1):
        amr.restrict(l)
    for l, d in enumerate(amr.data):
        amr.old[l] = {c: v.copy() for c, v in d.items()}


def test_fully_refined_level_equals_uniform_fine_grid(oracle):
    base = (2, 2, 2)
    lev0 = [(x, y, z) for z in range(2) for y in range(2) for x in range(2)]
    lev1 = [(x, y, z) for z in range(4) for y in range(4) for x in range(4)]
    fn = lambda x, y, z: Wk.bump_prims(x * 2, y * 2, z * 2)  # noqa: E731  (domain is [0, 0.5]^3)
    data = _level_data(oracle, [np.array(lev0), np.array(lev1)], fn, DH0)
    amr = amr_oracle.OracleAmr(base, [lev0, lev1], data, DH0)
    _consistent(amr)
    fine0 = np.zeros((5, 32, 32, 32))
    for (X, Y, Z), u in amr.data[1].items():
        fine0[:, 8 * Z:8 * Z + 8, 8 * Y:8 * Y + 8, 8 * X:8 * X + 8] = u
    amr.step()
    # uniform grid at level-1 resolution, two steps of dt_1
    dh1 = DH0 / 2
    ref = fine0
    for _ in range(2):
        ref = oracle.advance_block(oracle.fill_ghosts(ref, (1, 1, 1), "periodic"), (32, 32, 32),
                                   (1, 1, 1), 0.4 * dh1, dh1)["out"]
    got = np.zeros_like(ref)
    for (X, Y, Z), u in amr.data[1].items():
        got[:, 8 * Z:8 * Z + 8, 8 * Y:8 * Y + 8, 8 * X:8 * X + 8] = u
    assert np.max(np.abs(got - ref) / (np.abs(ref) + 1e-300)) <= 1e-14
    # level 0 is the average of level 1
    for (X, Y, Z), u in amr.data[0].items():
        blk = got[:, 16 * Z:16 * Z + 16, 16 * Y:16 * Y + 16, 16 * X:16 * X + 16]
        m = blk.reshape(5, 8, 2, 8, 2, 8, 2).mean(axis=(2, 4, 6))
        assert np.allclose(u, m, rtol=1e-15, atol=0)


def _two_level():
    lev = Wk.nested_hierarchy(base=(4, 4, 4), nlev=2)
    return [[tuple(c) for c in l] for l in lev], lev


@pytest.mark.parametrize("corrected", [True, False])
def test_composite_conservation_needs_flux_correction(oracle, corrected):
    levs, lev = _two_level()
    data = _level_data(oracle, lev, Wk.bump_prims, DH0)
    amr = amr_oracle.OracleAmr((4, 4, 4), levs, data, DH0, flux_correction=corrected)
    _consistent(amr)
    t0 = amr.totals()
    amr.step()
    t1 = amr.totals()
    scale = np.array([abs(t0[0]), abs(t0[1]) + abs(t0[4]), abs(t0[2]) + abs(t0[4]),
                      abs(t0[3]) + abs(t0[4]), abs(t0[4])])
    rel = np.abs(t1 - t0) / scale
    if corrected:
        assert rel.max() <= 1e-13, rel
    else:
        assert rel.max() >= 1e-9, rel   # the coarse-fine flux mismatch is visible


def test_uniform_state_stays_uniform(oracle):
    levs, lev = _two_level()
    data = _level_data(oracle, lev, lambda x, y, z: (2.0, 0.3, -0.1, 0.2, 0.7), DH0)
    amr = amr_oracle.OracleAmr((4, 4, 4), levs, data, DH0)
    u0 = next(iter(amr.data[0].values()))[:, 0, 0, 0].copy()
    amr.step()
    for d in amr.data:
        for u in d.values():
            assert np.array_equal(u, np.broadcast_to(u0[:, None, None, None], u.shape))


def _apply_map(h, cur, prev, w, special):
    """Ghost fill by the host map (numpy restatement of srhd_amr_fill_ghosts)."""
    n = h.ntotal
    flat_c = cur.reshape(n, 5, 512).transpose(1, 0, 2).reshape(5, -1)
    flat_p = prev.reshape(n, 5, 512).transpose(1, 0, 2).reshape(5, -1)
    m = h.map.astype(np.int64)
    out = np.empty((5,) + m.shape)
    sp = m < 0
    co = (m >= 0) & ((m & (1 << 30)) != 0)
    same = (m >= 0) & ~co
    q = m & ~(1 << 30)
    out[:, same] = flat_c[:, q[same]]
    out[:, co] = (1 - w) * flat_p[:, q[co]] + w * flat_c[:, q[co]]
    out[:, sp] = np.asarray(special)[-1 - m[sp]].T
    return out.transpose(1, 0, 2).reshape(n, 5, 12, 12, 12)


@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow")])
def test_host_map_matches_oracle_lookup(oracle, bc):
    lev = Wk.nested_hierarchy(base=(4, 4, 4), nlev=3)
    inflow = dict(axis=2, side=0, center=(16.0, 16.0), radius=5.0, index=0)
    h = Hierarchy((4, 4, 4), lev, bc=bc,
                  inflow=inflow if bc[2] == "outflow" else None)
    rng = np.random.default_rng(3)
    cur = rng.uniform(1, 2, (h.ntotal, 5, 8, 8, 8))
    prev = rng.uniform(1, 2, (h.ntotal, 5, 8, 8, 8))
    special = [[7.0, 0.1, 0.2, 0.3, 9.0]]
    levs = [[tuple(c) for c in l] for l in lev]
    data = [{c: cur[h.offsets[l] + n] for n, c in enumerate(levs[l])} for l in range(3)]
    amr = amr_oracle.OracleAmr((4, 4, 4), levs, data, DH0, bc=bc,
                               inflow=None if inflow is None or bc[2] != "outflow" else
                               dict(inflow, state=special[0]))
    amr.old = [{c: prev[h.offsets[l] + n] for n, c in enumerate(levs[l])} for l in range(3)]
    for w in (0.0, 0.5):
        G = _apply_map(h, cur, prev, w, special)
        for l in range(3):
            for n, c in enumerate(levs[l][::9]):
                p = h.offsets[l] + 9 * n
                assert np.allclose(G[p], amr.ghosted(l, c, w), rtol=1e-15, atol=0), (l, c, w)


def test_host_tables_match_hierarchy():
    lev = Wk.nested_hierarchy(base=(4, 4, 4), nlev=3)
    h = Hierarchy((4, 4, 4), lev)
    # restriction rows: parents are the refined block; children by octant
    for l in range(2):
        ch = h.children[l]
        assert len(ch) == 8
        for row in ch:
            X, Y, Z = h.coords[l][row[0] - h.offsets[l]]
            for o in range(8):
                cx, cy, cz = h.coords[l + 1][row[1 + o] - h.offsets[l + 1]]
                assert (cx, cy, cz) == (2 * X + (o & 1), 2 * Y + ((o >> 1) & 1), 2 * Z + (o >> 2))
    # flux-correction rows: the 24 unrefined neighbours of the 2x2x2 block,
    # one bordering face each
    for l in range(2):
        f = h.faces[l]
        assert len(f) == 24
        assert np.all((f[:, 1:] >= 0).reshape(-1, 6, 4).all(axis=2).sum(axis=1) == 1)
    # level-2 patches under a level-1 patch that does not exist: their ghost
    # zones are covered by neither level 2 nor level 1
    with pytest.raises(ValueError, match="nesting"):
        Hierarchy((4, 4, 4), [lev[0], lev[1], np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0],
                                                       [1, 1, 0], [0, 0, 1], [1, 0, 1],
                                                       [0, 1, 1], [1, 1, 1]])])


def test_flux_correction_skips_cells_left_unphysical(oracle):
    # Section 3.3 (4): the correction is ignored on a cell whose corrected
    # state fails Eq. (Unphysical result). Coarse patch (0, 1, 1) is
    # unrefined and its +x face borders the refined block. With zero fine
    # fluxes every cell on that face gets U += (dt/dh) F_coarse; one face
    # cell gets a flux that turns its Etilde negative and must keep its
    # state, the other 63 take the correction exactly.
    levs, lev = _two_level()
    data = _level_data(oracle, lev, Wk.bump_prims, DH0)
    amr = amr_oracle.OracleAmr((4, 4, 4), levs, data, DH0)
    zero = np.zeros((3, 5, 576))
    for c in levs[1]:
        amr.face_flux[1][c] = [zero, zero]
    coarse_flux = {c: np.zeros((3, 5, 576)) for c in levs[0]}
    c0 = (0, 1, 1)
    before = {c: v.copy() for c, v in amr.data[0].items()}
    coef = 0.4   # dt/dh of level 0
    rng = np.random.default_rng(1)
    u = before[c0]
    F = coarse_flux[c0]
    for k in range(8):
        for j in range(8):
            # a physical correction: a few per cent of each variable
            F[0, :, (k * 8 + j) * 9 + 8] = 0.03 * rng.uniform(-1, 1, 5) * \
                np.abs(u[:, k, j, 7]).max() / coef
    F[0, 4, (5 * 8 + 3) * 9 + 8] = -2.0 * u[4, 5, 3, 7] / coef    # Etilde -> -Etilde
    amr.flux_correct(0, coarse_flux)
    assert amr.skipped == 1
    for c, v in amr.data[0].items():
        if c != c0:
            assert np.array_equal(v, before[c])
    got = amr.data[0][c0]
    want = before[c0].copy()
    for k in range(8):
        for j in range(8):
            if (j, k) != (3, 5):
                want[:, k, j, 7] = want[:, k, j, 7] + coef * F[0, :, (k * 8 + j) * 9 + 8]
    assert np.array_equal(got, want)
    assert amr_oracle.OracleAmr.physical(got.reshape(5, -1)).all()


def _one_patch_amr(oracle, prims_fn):
    """A one-patch level 0 (outflow) whose 8^3 conserved cells come from
    prims_fn(i, j, k) -> (rho, Ux, Uy, Uz, p); for direct prolongation calls."""
    W = np.array([[[prims_fn(i, j, k) for i in range(8)] for j in range(8)] for k in range(8)])
    W = W.transpose(3, 0, 1, 2).reshape(5, -1)
    C, st = oracle.prim2con(W)
    assert np.all(st == 0)
    data = [{(0, 0, 0): C.reshape(5, 8, 8, 8)}, {}]
    return amr_oracle.OracleAmr((1, 1, 1), [[(0, 0, 0)], []], data, DH0,
                                bc=("outflow",) * 3, prolong="linear")


def test_linear_prolongation_is_exact_for_linear_data(oracle):
    # Section 3.3 (3), limited linear interpolation: for conserved variables
    # that are linear in the cell coordinates, both one-sided differences
    # are equal, the limiter keeps them, and the fine ghost value is the
    # linear function at the fine cell centre, a quarter of a coarse cell
    # from the coarse centre along each axis.
    amr = _one_patch_amr(oracle, lambda i, j, k: (1.0, 0.0, 0.0, 0.0, 1.0))
    u = amr.data[0][(0, 0, 0)]
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    lin = np.array([2.0 + 0.01 * i - 0.02 * j + 0.03 * k, 0.1 + 0.005 * i, -0.05 + 0.004 * k,
                    0.02 * j, 3.0 + 0.01 * i + 0.01 * j - 0.02 * k])
    u[...] = lin
    amr.old[0][(0, 0, 0)] = u.copy()
    for c in ((3, 4, 2), (1, 6, 5), (6, 1, 1)):
        for par in ((0, 0, 0), (1, 0, 1), (1, 1, 1), (0, 1, 0)):
            got = amr._prolong_linear(0, c, par, 0.0)
            x = [c[a] + (0.25 if par[a] else -0.25) for a in range(3)]
            want = np.array([2.0 + 0.01 * x[0] - 0.02 * x[1] + 0.03 * x[2], 0.1 + 0.005 * x[0],
                             -0.05 + 0.004 * x[2], 0.02 * x[1],
                             3.0 + 0.01 * x[0] + 0.01 * x[1] - 0.02 * x[2]])
            assert np.allclose(got, want, rtol=1e-14, atol=1e-16), (c, par, got - want)
    assert amr.prim_fallbacks == 0


def test_linear_prolongation_conserves_and_limits(oracle):
    # The eight fine cells of a coarse cell average to the coarse state
    # (offsets +-1/4 cancel), and at a local extremum the slope is zero
    # (minmod of one-sided differences of opposite sign).
    rng = np.random.default_rng(4)
    R = rng.uniform(0.5, 2.0, (8, 8, 8))
    amr = _one_patch_amr(oracle, lambda i, j, k: (R[k, j, i], 0.1 * R[j, i, k], 0.0, 0.0,
                                                  1.0 + 0.5 * R[i, k, j]))
    for c in ((3, 4, 2), (1, 1, 6)):
        kids = [amr._prolong_linear(0, c, ((o & 1), (o >> 1) & 1, o >> 2), 0.0)
                for o in range(8)]
        Uc = amr.data[0][(0, 0, 0)][:, c[2], c[1], c[0]]
        assert np.allclose(np.mean(kids, axis=0), Uc, rtol=1e-15, atol=1e-16)
    u = amr.data[0][(0, 0, 0)]
    u[:, 3, 3, 3] = 2.0 * u.reshape(5, -1).max(axis=1)   # a local maximum of every variable
    amr.old[0][(0, 0, 0)] = u.copy()
    peak = [amr._prolong_linear(0, (3, 3, 3), (o & 1, (o >> 1) & 1, o >> 2), 0.0)
            for o in range(8)]
    for p in peak:
        assert np.array_equal(p, u[:, 3, 3, 3])
    assert amr.prim_fallbacks == 0


def test_linear_prolongation_falls_back_to_primitives(oracle):
    # Cold gas (T = 1e-6) moving at U^x = 9, 10, 12 in three neighbouring
    # cells: cold states lie on the boundary of the physical cone
    # E^2 >= D^2 + |M|^2, so extrapolating the conserved variables from the
    # middle cell towards the right (1.25 C - 0.25 L, the minmod picks the
    # smaller left difference) leaves the cone: Eq. (Unphysical result)
    # fails and the primitive variables are interpolated instead
    # (U^x = 10 + 0.25 * 1), which Eq. (Unphysical result) always accepts.
    ux = {2: 9.0, 3: 10.0, 4: 12.0}
    amr = _one_patch_amr(oracle, lambda i, j, k: (1.0, ux.get(i, 10.0), 0.0, 0.0, 1e-6))
    c = (3, 4, 4)
    Cc = amr.data[0][(0, 0, 0)][:, 4, 4, 3]
    Cl = amr.data[0][(0, 0, 0)][:, 4, 4, 2]
    cons_interp = Cc + 0.25 * (Cc - Cl)
    assert not amr_oracle.OracleAmr.physical(cons_interp.reshape(5, 1))[0]
    got = amr._prolong_linear(0, c, (1, 0, 0), 0.0)
    assert amr.prim_fallbacks == 1
    want, _ = oracle.prim2con(np.array([[1.0], [10.25], [0.0], [0.0], [1e-6]]))
    assert np.allclose(got, want[:, 0], rtol=1e-7, atol=0)
    assert amr_oracle.OracleAmr.physical(got.reshape(5, 1))[0]
    # towards the left the conserved interpolation (1.25 C - 0.25 L again,
    # the same minmod side) fails too; at parity 0 along an axis with equal
    # neighbours nothing changes
    same = amr._prolong_linear(0, c, (0, 0, 0), 0.0)
    assert amr_oracle.OracleAmr.physical(same.reshape(5, 1))[0]


def test_linear_prolongation_reduces_interface_error(oracle):
    # A two-level run of a smooth field against the uniform grid at the fine
    # resolution: taking the fine level's ghost zones by limited linear
    # interpolation instead of the containing coarse cell makes the fine
    # level's error after one coarse step markedly smaller (the ghost values
    # are second- instead of first-order accurate).
    base = (4, 4, 4)
    lev = Wk.nested_hierarchy(base=base, nlev=2)
    levs = [[tuple(c) for c in l] for l in lev]
    data = _level_data(oracle, lev, Wk.bump_prims, DH0)
    # uniform fine-grid reference from the same smooth field
    W = Wk.level_prims([(x, y, z) for z in range(8) for y in range(8) for x in range(8)], 1,
                       Wk.bump_prims, DH0)
    C, _ = oracle.prim2con(W.transpose(1, 0, 2, 3, 4).reshape(5, -1))
    C = C.reshape(5, 8, 8, 8, 8, 8, 8)   # [v][Z][Y][X][k][j][i] for patches (X, Y, Z) in z,y,x order
    fine = np.zeros((5, 64, 64, 64))
    n = 0
    for z in range(8):
        for y in range(8):
            for x in range(8):
                fine[:, 8 * z:8 * z + 8, 8 * y:8 * y + 8, 8 * x:8 * x + 8] = \
                    C.reshape(5, 512, 8, 8, 8)[:, n]
                n += 1
    dh1 = DH0 / 2
    ref = fine
    for _ in range(2):
        ref = oracle.advance_block(oracle.fill_ghosts(ref, (1, 1, 1), "periodic"), (64, 64, 64),
                                   (1, 1, 1), 0.4 * dh1, dh1)["out"]
    errs = {}
    for mode in ("constant", "linear"):
        amr = amr_oracle.OracleAmr(base, levs, data, DH0, prolong=mode)
        _consistent(amr)
        amr.step()
        e = []
        for (X, Y, Z), u in amr.data[1].items():
            r = ref[:, 8 * Z:8 * Z + 8, 8 * Y:8 * Y + 8, 8 * X:8 * X + 8]
            e.append(np.abs(u[0] - r[0]) / r[0])
        errs[mode] = float(np.max(e))
    assert errs["linear"] < 0.6 * errs["constant"], errs


def prolong_rows_coords(h, l):
    """One fine-level cell (x, y, z) of level l (boundary rule applied) per
    row of h.prolong_tables[l], found through the map."""
    t = h.prolong_tables[l]
    coords = np.full((len(t), 3), -1, np.int64)
    base = h.nspecial + h.prolong_offsets[l]
    N = h.cells(l)
    for n, (X, Y, Z) in enumerate(h.coords[l]):
        m = h.map[h.offsets[l] + n].astype(np.int64)
        r = -1 - m - base
        sel = (m < 0) & (r >= 0) & (r < len(t))
        for c in np.nonzero(sel)[0]:
            k, j, i = c // 144, (c // 12) % 12, c % 12
            co = [8 * X + i - 2, 8 * Y + j - 2, 8 * Z + k - 2]
            for a in range(3):
                co[a] = co[a] % N[a] if h.bc[a] == "periodic" else min(max(co[a], 0), N[a] - 1)
            coords[r[c]] = co
    assert np.all(coords >= 0), "a table row that no map entry reads"
    return coords


@pytest.mark.parametrize("bc", [("periodic",) * 3, ("outflow", "periodic", "outflow")])
def test_host_prolong_tables_match_oracle_neighbours(oracle, bc):
    # The host tables of limited linear prolongation name, for every
    # coarse-sourced ghost cell, the coarse cell the oracle's geometric
    # lookup finds, its six neighbours (or -1 where the coarse level does
    # not cover one) and the fine cell's parity along each axis.
    lev = Wk.nested_hierarchy(base=(4, 4, 4), nlev=3)
    h = Hierarchy((4, 4, 4), lev, bc=bc, prolong="linear")
    rng = np.random.default_rng(5)
    cur = rng.uniform(1, 2, (h.ntotal, 5, 8, 8, 8))
    levs = [[tuple(c) for c in l] for l in lev]
    data = [{c: cur[h.offsets[l] + n] for n, c in enumerate(levs[l])} for l in range(3)]
    amr = amr_oracle.OracleAmr((4, 4, 4), levs, data, DH0, bc=bc, prolong="linear")
    flat = cur.transpose(1, 0, 2, 3, 4).reshape(5, -1)
    for l in (1, 2):
        t = h.prolong_tables[l]
        xyz = prolong_rows_coords(h, l)
        for r in range(0, len(t), 17):
            x, y, z = xyz[r]
            xc, yc, zc = x // 2, y // 2, z // 2
            assert np.array_equal(flat[:, t[r, 0]], amr._coarse(l - 1, xc, yc, zc, 1.0))
            for k, (dx, dy, dz) in enumerate(((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                                              (0, 0, -1), (0, 0, 1))):
                want = amr._coarse(l - 1, xc + dx, yc + dy, zc + dz, 1.0)
                if t[r, 1 + k] < 0:
                    assert want is None
                else:
                    assert np.array_equal(flat[:, t[r, 1 + k]], want)
            assert t[r, 7] == (x % 2) | ((y % 2) << 1) | ((z % 2) << 2)
