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
