"""Writes mixed_limits_cells_t80.txt: the exact TM solution (Appendix C of
arXiv 2012.11130, computed by the oracle's exact Riemann solver) of the
mixed-limits Riemann problem of Section 4.2.2 (Table "tb:IC_RiemannProblems",
second row: (rho, U, p) = (1e2, 1e-3, 1e-4) | (1e-12, -1e2, 1e-10), the
discontinuity at x = 5e-2) at t = 80, on the paper's grid of 102 400 cells
of [0, 100]. The rows are the cells with centres below x = 0.3 (the cold
left state, the rarefaction fan, the left plateau and the contact); beyond
them the solution is the right plateau up to the shock and the right state
after it, whose values and the shock position are the header's key lines.

Usage: python tests/golden/make_mixed_limits_exact.py   (calls only oracle/)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import oracle as O  # noqa: E402

LEFT, RIGHT, X0, T_END, N, LENGTH = (1e2, 1e-3, 1e-4), (1e-12, -1e2, 1e-10), 5e-2, 80.0, 102400, 100.0


def main():
    x = (np.arange(N) + 0.5) * (LENGTH / N)
    x = x[x < 0.3]
    rho, U, p, info = O.exact_riemann(LEFT, RIGHT, X0, T_END, x)
    # the right-moving shock: four-velocity Ushock_R, speed Ushock_R / sqrt(1 + Ushock_R^2)
    vs = info["Ushock_R"] / np.sqrt(1.0 + info["Ushock_R"] ** 2)
    hdr = ("exact TM solution of the mixed-limits Riemann problem (1e2,1e-3,1e-4)|(1e-12,-1e2,1e-10), "
           "x0 = 5e-2, t = 80, 102400 cells of [0,100]; written by "
           "tests/golden/make_mixed_limits_exact.py (oracle, Appendix C)\n"
           f"key rho_right_plateau = {info['rho_CR']:.17g}\n"
           f"key U_right_plateau = {info['U_CR']:.17g}\n"
           f"key p_star = {info['pstar']:.17g}\n"
           f"key x_shock = {X0 + vs * T_END:.17g}\n"
           "columns (cells with centres below 0.3): x rho U_x p")
    np.savetxt(os.path.join(HERE, "mixed_limits_cells_t80.txt"), np.column_stack([x, rho, U, p]),
               fmt="%.17e", header=hdr)


if __name__ == "__main__":
    main()
