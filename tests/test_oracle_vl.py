"""CPU pins of the oracle's VL integrator (Section 3.1: GAMER-SR supports
MUSCL-Hancock and VL; a first-order unsplit predictor to the half step,
then a PLM corrector for the full step) against special cases, symmetries,
conservation, smooth convergence and the exact Riemann solution."""
import numpy as np


def _cons(oracle, W):
    C, st = oracle.prim2con(np.asarray(W, float).reshape(5, -1))
    assert np.all(st == 0)
    return C


def _smooth_block(oracle, rng, shape, amp=0.3):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(*(np.arange(s) / s for s in shape), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 5)
    W = np.stack([1 + amp * np.sin(2 * np.pi * (x + 2 * y) + ph[0]),
                  0.5 * np.sin(2 * np.pi * (x + z) + ph[2]),
                  0.5 * np.cos(2 * np.pi * (x - y) + ph[3]),
                  0.5 * np.sin(2 * np.pi * z + ph[4]),
                  1 + amp * np.sin(2 * np.pi * (y - z) + ph[1])]).reshape(5, -1)
    return _cons(oracle, W).reshape(5, nz, ny, nx)


def test_uniform_state_unchanged(oracle):
    for W in ([1.0, 0.0, 0.0, 0.0, 1.0], [1e-3, 3.0, -4.0, 5.0, 1e-7]):
        C = _cons(oracle, W)[:, 0]
        G = np.broadcast_to(C[:, None, None, None], (5, 14, 14, 14)).copy()
        r = oracle.advance_block_vl(G, (8, 8, 8), (1, 1, 1), 1e-3, 1e-2)
        assert r["status"] == 0 and r["retries"] == 0
        assert np.array_equal(r["out"], G[:, 3:-3, 3:-3, 3:-3])


def test_mirror_symmetry_and_periodic_conservation(oracle):
    rng = np.random.default_rng(5)
    C = _smooth_block(oracle, rng, (14, 14, 14))
    Cm = C[:, :, :, ::-1].copy()
    Cm[1] *= -1
    a = oracle.advance_block_vl(C, (8, 8, 8), (1, 1, 1), 2e-3, 1 / 14)
    b = oracle.advance_block_vl(Cm, (8, 8, 8), (1, 1, 1), 2e-3, 1 / 14)
    bm = b["out"][:, :, :, ::-1].copy()
    bm[1] *= -1
    scale = np.abs(a["out"]).max(axis=(1, 2, 3))[:, None, None, None]
    assert np.all(np.abs(a["out"] - bm) <= 1e-13 * scale)
    # periodic conservation over a few steps
    C = _smooth_block(oracle, rng, (16, 16, 16))
    tot0 = C.reshape(5, -1).sum(1)
    for _ in range(3):
        dt = oracle.cfl_dt(C, 1 / 16)
        r = oracle.advance_block_vl(oracle.fill_ghosts(C, (1, 1, 1), "periodic", 3),
                                    (16, 16, 16), (1, 1, 1), dt, 1 / 16)
        assert r["status"] == 0
        C = r["out"]
    scale = np.abs(C.reshape(5, -1)).sum(1)
    assert np.all(np.abs(C.reshape(5, -1).sum(1) - tot0) <= 1e-13 * scale)


def test_direction_permutation(oracle):
    N = 24
    x = (np.arange(N) + 0.5) / N
    W = np.vstack([1 + 0.5 * (x > 0.5), 0.2 * np.sin(2 * np.pi * x), np.zeros(N), np.zeros(N),
                   1 + (x < 0.3)])
    res = []
    for d in range(3):
        Wd = W.copy()
        Wd[[1, 1 + d]] = Wd[[1 + d, 1]]
        C = _cons(oracle, Wd)
        shape = [1, 1, 1]
        shape[2 - d] = N
        act = [0, 0, 0]
        act[d] = 1
        G = oracle.fill_ghosts(C.reshape(5, *shape), act, "outflow", 3)
        n = [1, 1, 1]
        n[d] = N
        out = oracle.advance_block_vl(G, tuple(n), tuple(act), 4e-3, 1 / N)["out"].reshape(5, N)
        out[[1, 1 + d]] = out[[1 + d, 1]]
        res.append(out)
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_smooth_advection_second_order_and_close_to_mh(oracle):
    # hot gas, gamma = 10: the wave is translated exactly; VL converges at
    # second order and its error is of the size of MUSCL-Hancock's
    Ux = np.sqrt(99.0)
    v = Ux / 10.0
    t_end = 1.0 / v
    errs = {"vl": [], "mh": []}
    for N in (32, 64, 128):
        dh = 1.0 / N
        x = (np.arange(N) + 0.5) * dh
        W = np.vstack([1 + 0.5 * np.sin(2 * np.pi * x), np.full(N, Ux), np.zeros(N), np.zeros(N),
                       np.ones(N)])
        C = _cons(oracle, W).reshape(5, 1, 1, N)
        exact = 1 + 0.5 * np.sin(2 * np.pi * (x - v * t_end))
        for integ in ("vl", "mh"):
            res = oracle.evolve(C, (1, 0, 0), dh, t_end, "periodic", integrator=integ)
            prim = oracle.con2pri(res["cons"].reshape(5, -1))["prim"]
            errs[integ].append(np.mean(np.abs(1 - prim[0] / exact)))
    assert np.log2(errs["vl"][1] / errs["vl"][2]) > 1.7, errs
    assert 0.2 < errs["vl"][2] / errs["mh"][2] < 5, errs


def test_shock_tube_converges_to_exact(oracle):
    # the tube of the MUSCL-Hancock pin: the thin blast shell dominates the
    # relative L1 until it is resolved, so convergence is judged from 256 to
    # 1024 cells, at about first order, and VL's error is close to
    # MUSCL-Hancock's
    errs = {"vl": [], "mh": []}
    for N in (256, 512, 1024):
        dh = 1.0 / N
        x = (np.arange(N) + 0.5) * dh
        W = np.vstack([np.ones(N), np.zeros(N), np.zeros(N), np.zeros(N),
                       np.where(x < 0.5, 1e3, 1e-2)])
        rho, _, _, _ = oracle.exact_riemann((1, 0, 1e3), (1, 0, 1e-2), 0.5, 0.4, x)
        for integ in ("vl", "mh"):
            res = oracle.evolve(_cons(oracle, W).reshape(5, 1, 1, N), (1, 0, 0), dh, 0.4,
                                "outflow", integrator=integ)
            prim = oracle.con2pri(res["cons"].reshape(5, -1))["prim"]
            errs[integ].append(np.mean(np.abs(1 - prim[0] / rho)))
    e = errs["vl"]
    assert e[2] < e[1] < e[0], errs
    assert 0.5 < np.log2(e[0] / e[2]) / 2 < 1.3, errs
    assert 0.7 < e[2] / errs["mh"][2] < 1.5, errs


def test_patch_batch_matches_block_and_bad_input(oracle):
    rng = np.random.default_rng(2)
    P = np.stack([_smooth_block(oracle, rng, (14, 14, 14)) for _ in range(3)])
    dt_dh = np.array([[1e-3, 0.1], [2e-3, 0.05], [5e-4, 0.2]])
    r = oracle.advance_patches_vl(P, dt_dh, want_flux=True)
    for i in range(3):
        b = oracle.advance_block_vl(P[i], (8, 8, 8), (1, 1, 1), dt_dh[i, 0], dt_dh[i, 1],
                                    want_flux=True)
        assert np.array_equal(b["out"], r["out"][i])
        assert np.array_equal(b["flux"], r["flux"][i].reshape(-1))
    # an unphysical cell in the predictor's stencil (third ghost layer, on an
    # axis line of the interior) is bad input; a corner far from every
    # stencil is not read
    Q = P[0].copy()
    Q[0, 0, 5, 5] = -1.0
    assert oracle.advance_block_vl(Q, (8, 8, 8), (1, 1, 1), 1e-3, 0.1)["status"] == 2
    Q = P[0].copy()
    Q[0, 0, 0, 0] = -1.0
    assert oracle.advance_block_vl(Q, (8, 8, 8), (1, 1, 1), 1e-3, 0.1)["status"] == 0
