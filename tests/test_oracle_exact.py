"""Pins of the oracle's exact TM Riemann solver (Appendix C of arXiv
2012.11130): the paper's printed exact-solution table, jump conditions and
invariants. CPU only."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "exact_mixed_limits_t80.txt")
MIXED_L = (1e2, 1e-3, 1e-4)
MIXED_R = (1e-12, -1e2, 1e-10)


def test_exact_table_mixed_limits(oracle):
    tab = np.loadtxt(GOLDEN)
    rho, U, p, info = oracle.exact_riemann(MIXED_L, MIXED_R, 0.05, 80.0, tab[:, 0])
    assert info["shock_L"] == 0 and info["shock_R"] == 1  # rarefaction - contact - shock
    # The table prints 16 digits. Its left- and right-contact four-velocities
    # (rows 15-16 vs 17-18) differ from each other by 4.6e-10 relative,
    # which is the accuracy of the printed root; elsewhere the rows agree
    # with this solver to about 1e-12.
    rel = lambda a, b: np.abs(a / b - 1)
    assert np.all(rel(rho, tab[:, 1]) < 2e-12)
    assert np.all(rel(p, tab[:, 3]) < 2e-12)
    right_contact = np.array([16, 17])
    others = np.setdiff1d(np.arange(20), right_contact)
    assert np.all(rel(U[others], tab[others, 2]) < 2e-12)
    assert np.all(rel(U[right_contact], tab[right_contact, 2]) < 1e-9)
    # internal consistency of the printed table itself
    assert abs(tab[16, 2] / tab[15, 2] - 1) < 1e-9


def test_contact_velocity_continuous(oracle):
    for L, R in ((MIXED_L, MIXED_R), ((1.0, 0.0, 1e3), (1.0, 0.0, 1e-2))):
        _, _, _, info = oracle.exact_riemann(L, R, 0.5, 0.4, np.array([0.5]))
        assert abs(info["U_CL"] / info["U_CR"] - 1) < 1e-10


def test_shock_mass_flux_continuity(oracle):
    # Across a shock moving with four-velocity Us, the rest-mass flux
    # rho (U gamma_s - gamma U_s) is the same on both sides.
    for L, R in ((MIXED_L, MIXED_R), ((1.0, 0.0, 1e3), (1.0, 0.0, 1e-2))):
        _, _, _, info = oracle.exact_riemann(L, R, 0.5, 0.4, np.array([0.5]))
        Us = info["Ushock_R"]
        gs = np.sqrt(1 + Us * Us)
        rho_u, U_u = R[0], R[1]
        rho_d, U_d = info["rho_CR"], info["U_CR"]
        j_u = rho_u * (U_u * gs - np.sqrt(1 + U_u ** 2) * Us)
        j_d = rho_d * (U_d * gs - np.sqrt(1 + U_d ** 2) * Us)
        assert abs(j_d / j_u - 1) < 1e-9


def test_shock_speed_from_table(oracle):
    # The table brackets the shock between x = 26.90929 and 26.91026 at t=80.
    _, _, _, info = oracle.exact_riemann(MIXED_L, MIXED_R, 0.05, 80.0, np.array([1.0]))
    Us = info["Ushock_R"]
    xs = 0.05 + 80.0 * Us / np.sqrt(1 + Us * Us)
    assert 26.909288248391281 < xs < 26.910264810891281


def test_isentrope_constant_in_fan(oracle):
    # Eq. (entropy): p (h - T) / rho^{5/3} is constant through the fan.
    x = np.linspace(0.027, 0.2, 40)
    rho, U, p, info = oracle.exact_riemann(MIXED_L, MIXED_R, 0.05, 80.0, x)
    T = p / rho
    h = 1 + oracle.htilde_of_T(T)
    K = p * (h - T) / rho ** (5 / 3)
    TL = MIXED_L[2] / MIXED_L[0]
    KL = MIXED_L[2] * (1 + oracle.htilde_of_T(TL) - TL) / MIXED_L[0] ** (5 / 3)
    assert np.max(np.abs(K / KL - 1)) < 1e-12


def test_head_on_collision_symmetric(oracle):
    # Ultra-relativistic head-on collision (Table tb:IC_RiemannProblems, row 1):
    # two shocks, gas at rest between them, symmetric.
    L = (1e-5, 1e6, 1.0)
    R = (1e-5, -1e6, 1.0)
    x = np.array([0.2, 0.5, 0.8])
    rho, U, p, info = oracle.exact_riemann(L, R, 0.5, 1.0, x)
    assert info["shock_L"] == 1 and info["shock_R"] == 1
    assert abs(info["U_CL"]) < 1e-6 * 1e6 * 1e-9
    assert abs(info["Ushock_L"] + info["Ushock_R"]) < 1e-9 * abs(info["Ushock_R"])
    assert abs(info["rho_CL"] / info["rho_CR"] - 1) < 1e-9


def test_rapidity_integral_additive(oracle):
    a = oracle.rapidity_integral(1e-6, 1e-2)
    b = oracle.rapidity_integral(1e-2, 1e3)
    c = oracle.rapidity_integral(1e-6, 1e3)
    assert abs((a + b) / c - 1) < 1e-14
    assert oracle.rapidity_integral(1e3, 1e-6) == -c


def _fixture_keys(path):
    keys = {}
    for line in open(path):
        if line.startswith("# key "):
            k, v = line[6:].split("=")
            keys[k.strip()] = float(v)
    return keys


def test_mixed_limits_cell_fixture(oracle):
    # tests/golden/mixed_limits_cells_t80.txt (the mixed-limits solution at
    # the cell centres of the paper's 102 400-cell grid, for the GPU run of
    # Section 4.2.2 in bench.py) is this solver's output, and its constants
    # are the paper's table: the right plateau's density and pressure, the
    # contact four-velocity (to the table's 1e-9), and the shock inside the
    # table's bracket; the rows run from the cold left state through the fan
    # to the right plateau, ending at x < 0.3.
    path = os.path.join(os.path.dirname(__file__), "golden", "mixed_limits_cells_t80.txt")
    cells = np.loadtxt(path)
    keys = _fixture_keys(path)
    tab = np.loadtxt(GOLDEN)
    x = cells[:, 0]
    dx = 100.0 / 102400
    assert np.allclose(x, (np.arange(x.size) + 0.5) * dx, rtol=0, atol=1e-15) and x[-1] < 0.3 <= x[-1] + dx
    rho, U, p, _ = oracle.exact_riemann(MIXED_L, MIXED_R, 0.05, 80.0, x)
    assert np.all(np.abs(cells[:, 1] / rho - 1) < 1e-14) and np.all(np.abs(cells[:, 3] / p - 1) < 1e-14)
    assert abs(keys["rho_right_plateau"] / tab[17, 1] - 1) < 2e-12
    assert abs(keys["p_star"] / tab[17, 3] - 1) < 2e-12
    assert abs(keys["U_right_plateau"] / tab[17, 2] - 1) < 1e-9
    assert tab[17, 0] < keys["x_shock"] < tab[18, 0]
    assert cells[0, 1] == MIXED_L[0] and abs(cells[-1, 1] / keys["rho_right_plateau"] - 1) < 1e-12
