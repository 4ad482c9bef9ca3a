"""CPU pins of the oracle's polytropic (constant-Gamma) EoS option, the EoS
the paper keeps for pure non-relativistic or ultra-relativistic gas
(Section 2.2: h = 1 + Gamma/(Gamma-1) T), against closed forms derived
independently of the oracle's code:
* the TM EoS tends to Gamma = 5/3 for T -> 0 and Gamma = 4/3 for T -> inf;
* c_s^2 = (dp/de)_s = Gamma T / h from p = K rho^Gamma and de = h drho;
* the rarefaction rapidity integral has the closed form
  (2/sqrt(Gamma-1)) [artanh(c_s/sqrt(Gamma-1))] between its limits
  (d/dT of it equals c_s / ((Gamma-1) T));
* conversions round-trip, Newton equals bisection, the scheme conserves,
  converges at second order on a smooth wave and at about first order to the
  exact polytropic shock-tube solution, and a cold shock tube barely
  notices the difference between TM and Gamma = 5/3.
"""
import numpy as np
import pytest

GAMMAS = (5.0 / 3.0, 4.0 / 3.0)


@pytest.fixture
def poly(oracle):
    def use(g):
        return oracle.eos(oracle.EOS_POLYTROPIC, g)
    return use


def test_tm_limits_are_the_polytropic_eos(oracle, poly):
    T_lo, T_hi = np.array([1e-9]), np.array([1e9])
    tm_lo, tm_hi = oracle.htilde_of_T(T_lo), oracle.htilde_of_T(T_hi)
    with poly(5 / 3):
        p_lo = oracle.htilde_of_T(T_lo)
    with poly(4 / 3):
        p_hi = oracle.htilde_of_T(T_hi)
    assert abs(tm_lo[0] / p_lo[0] - 1) < 1e-8
    assert abs(tm_hi[0] / p_hi[0] - 1) < 1e-8
    # closed form
    for g in GAMMAS:
        with poly(g):
            T = np.logspace(-8, 6, 50)
            assert np.allclose(oracle.htilde_of_T(T), g / (g - 1) * T, rtol=1e-15)
            assert np.allclose(oracle.T_of_htilde(g / (g - 1) * T), T, rtol=1e-15)


def test_sound_speed_from_isentrope(oracle, poly):
    # along p = K rho^Gamma, e = rho h - p and c_s^2 = dp/de, by central
    # differences in ln rho
    for g in GAMMAS:
        with poly(g):
            for T0 in (1e-6, 1e-2, 1.0, 1e3):
                rho0 = 1.0
                K = rho0 * T0 / rho0 ** g

                def pe(lnr):
                    r = np.exp(lnr)
                    p = K * r ** g
                    T = p / r
                    return p, r * (1 + oracle.htilde_of_T(np.array([T]))[0]) - p
                e = 1e-5
                p1, e1 = pe(np.log(rho0) + e)
                p0, e0 = pe(np.log(rho0) - e)
                cs2_fd = (p1 - p0) / (e1 - e0)
                cs2 = oracle.cs2_of_T(np.array([T0]))[0]
                assert abs(cs2 / cs2_fd - 1) < 1e-8, (g, T0)
                h = 1 + g / (g - 1) * T0
                assert abs(cs2 / (g * T0 / h) - 1) < 1e-14


def test_rapidity_integral_closed_form(oracle, poly):
    for g in GAMMAS:
        with poly(g):
            s = np.sqrt(g - 1)
            for T1, T2 in ((1e-6, 1e-3), (1e-2, 10.0), (0.5, 3e4)):
                c1 = np.sqrt(oracle.cs2_of_T(np.array([T1]))[0])
                c2 = np.sqrt(oracle.cs2_of_T(np.array([T2]))[0])
                closed = 2 / s * (np.arctanh(c2 / s) - np.arctanh(c1 / s))
                assert abs(oracle.rapidity_integral(T1, T2) / closed - 1) < 1e-12


def test_conversion_round_trip_and_bisection(oracle, poly):
    rng = np.random.default_rng(5)
    n = 4000
    rho = 10 ** rng.uniform(-4, 2, n)
    T = 10 ** rng.uniform(-8, 4, n)
    U = 10 ** rng.uniform(-3, 3, n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    W = np.vstack([rho, U * d, rho * T])
    for g in GAMMAS:
        with poly(g):
            C, st = oracle.prim2con(W)
            assert np.all(st == 0)
            r = oracle.con2pri(C)
            ok = r["status"] == 0
            assert ok.mean() > 0.99
            ht0 = g / (g - 1) * T
            err = np.abs(r["htilde"][ok] / ht0[ok] - 1)
            # the round trip tracks the conditioning (1 + Mach^2) eps
            cs2 = oracle.cs2_of_T(T)
            mach2 = U * U * (1 - cs2) / cs2
            assert np.all(err <= 64 * (1 + mach2[ok]) * 2.2e-16 + 1e-15)
            for q in range(0, n, 97):
                m2 = (C[1, q] ** 2 + C[2, q] ** 2 + C[3, q] ** 2) / C[0, q] ** 2
                hb = oracle.lib().or_htilde_bisect(r["A"][q], m2)
                if ok[q]:
                    assert abs(r["htilde"][q] / hb - 1) < 1e-13


def _shock_tube(oracle, N, L=(1.0, 0.0, 1e3), R=(1.0, 0.0, 1e-2), t=0.4):
    x = (np.arange(N) + 0.5) / N
    W = np.where(x < 0.5, np.array(L)[[0, 1, 2]][:, None], np.array(R)[[0, 1, 2]][:, None])
    W5 = np.vstack([W[0], W[1], 0 * x, 0 * x, W[2]])
    C, st = oracle.prim2con(W5)
    res = oracle.evolve(C.reshape(5, 1, 1, N), (1, 0, 0), 1.0 / N, t, "outflow")
    prim = oracle.con2pri(res["cons"].reshape(5, -1))["prim"]
    rho_ex, _, _, _ = oracle.exact_riemann(L, R, 0.5, t, x)
    return np.mean(np.abs(1 - prim[0] / rho_ex)), res


SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)   # mildly relativistic (T_L = 1)


@pytest.mark.parametrize("g", GAMMAS)
def test_polytropic_shock_tube_converges_to_exact(oracle, poly, g):
    with poly(g):
        errs = [_shock_tube(oracle, N, SOD_L, SOD_R)[0] for N in (128, 256, 512)]
        assert errs[1] < errs[0] and errs[2] < errs[1], errs
        order = np.log2(errs[0] / errs[2]) / 2
        assert 0.5 < order < 1.3, errs
        # the exact solution conserves mass: shock mass-flux continuity
        _, _, _, info = oracle.exact_riemann(SOD_L, SOD_R, 0.5, 0.4, np.array([0.5]))
        Us = info["Ushock_R"]
        gs = np.sqrt(1 + Us * Us)
        j_u = SOD_R[0] * (0.0 * gs - 1.0 * Us)
        j_d = info["rho_CR"] * (info["U_CR"] * gs - np.sqrt(1 + info["U_CR"] ** 2) * Us)
        assert abs(j_d / j_u - 1) < 1e-9


def test_cold_shock_tube_tm_equals_five_thirds(oracle, poly):
    # a non-relativistic shock tube (T ~ 1e-4): TM behaves as Gamma = 5/3
    L, R = (1.0, 0.0, 1e-4), (0.125, 0.0, 1e-5)
    x = np.linspace(0.01, 0.99, 99)
    rho_tm, _, _, _ = oracle.exact_riemann(L, R, 0.5, 20.0, x)
    with poly(5 / 3):
        rho_53, _, _, _ = oracle.exact_riemann(L, R, 0.5, 20.0, x)
    with poly(4 / 3):
        rho_43, _, _, _ = oracle.exact_riemann(L, R, 0.5, 20.0, x)
    d53 = np.mean(np.abs(rho_tm / rho_53 - 1))
    d43 = np.mean(np.abs(rho_tm / rho_43 - 1))
    assert d53 < 1e-3 and d43 > 10 * d53, (d53, d43)


def test_polytropic_scheme_conserves_and_is_second_order(oracle, poly):
    for g in GAMMAS:
        with poly(g):
            errs = []
            Ux = 3.0
            v = Ux / np.sqrt(1 + Ux * Ux)
            t_end = 1.0 / v
            for N in (32, 64, 128):
                dh = 1.0 / N
                x = (np.arange(N) + 0.5) * dh
                W = np.vstack([1 + 0.5 * np.sin(2 * np.pi * x), np.full(N, Ux), np.zeros(N),
                               np.zeros(N), np.ones(N)])
                C, _ = oracle.prim2con(W)
                res = oracle.evolve(C.reshape(5, 1, 1, N), (1, 0, 0), dh, t_end, "periodic")
                tot0 = C.sum(axis=1)
                tot1 = res["cons"].reshape(5, -1).sum(axis=1)
                assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.abs(C).sum(axis=1))
                prim = oracle.con2pri(res["cons"].reshape(5, -1))["prim"]
                exact = 1 + 0.5 * np.sin(2 * np.pi * (x - v * t_end))
                errs.append(np.mean(np.abs(1 - prim[0] / exact)))
            assert np.log2(errs[1] / errs[2]) > 1.7, (g, errs)


def test_invalid_gamma_is_refused(oracle):
    for g in (1.0, 0.5, 2.0):
        with pytest.raises(ValueError):
            oracle.set_eos(oracle.EOS_POLYTROPIC, g)
    oracle.set_eos(oracle.EOS_TM)
