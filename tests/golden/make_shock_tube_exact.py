"""Writes shock_tube_exact_1024.txt: the exact TM solution (Appendix C of
arXiv 2012.11130, computed by the oracle's exact Riemann solver) of the 1-D
shock tube (rho, v, p) = (1, 0, 1e3) | (1, 0, 1e-2) with the diaphragm at
x = 0.5, at t = 0.4, sampled at the 1024 cell centres of [0, 1].

Usage: python tests/golden/make_shock_tube_exact.py   (calls only oracle/)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import oracle as O  # noqa: E402


def main():
    n = 1024
    x = (np.arange(n) + 0.5) / n
    rho, U, p, info = O.exact_riemann((1.0, 0.0, 1e3), (1.0, 0.0, 1e-2), 0.5, 0.4, x)
    hdr = ("exact TM solution of the shock tube (1,0,1e3)|(1,0,1e-2), x0 = 0.5, t = 0.4, "
           "written by tests/golden/make_shock_tube_exact.py (oracle, Appendix C)\n"
           f"p* = {info['pstar']:.17g}, U* = {info['U_CL']:.17g}\ncolumns: x rho U_x p")
    np.savetxt(os.path.join(HERE, "shock_tube_exact_1024.txt"), np.column_stack([x, rho, U, p]),
               fmt="%.17e", header=hdr)


if __name__ == "__main__":
    main()
