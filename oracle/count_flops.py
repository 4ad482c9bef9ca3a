"""Algorithmic operation count of one cell update of the benchmark workload
(3-D smooth advection, gamma = 10 along the diagonal, hot gas T ~ 1), from
the operation-counting instantiation of the oracle.

TEST INFRASTRUCTURE: runs only the oracle. One MUSCL-Hancock step of an
n^3 periodic block is counted for n = 16, 32, 64; the count per interior
cell is c(n) = a + b/n + c/n^2 (halo work scales with the surface), and
a, the limit n -> infinity, is the algorithmic count of one cell update
(ghost recomputation excluded). The CFL bound of the updated cell (one
con2pri and S_max) is counted separately and added. The same count is made
for the VL integrator (key "vl") and for the MUSCL-Hancock step under the
polytropic EoS with Gamma = 4/3 (key "polytropic_gamma_4_3"), the two other
workloads the benchmark times on this state.

Usage: python oracle/count_flops.py   (prints JSON)
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import oracle as O  # noqa: E402
from paper_2012_11130_gb300 import workloads  # noqa: E402


def per_cell(n, N=256, vl=False):
    W = workloads.advection_prims(N)
    C, _ = O.prim2con(W.reshape(5, -1))
    g = 6 if vl else 4  # ghost cells of both sides
    C = C.reshape(5, N, N, N)[:, :n + g, :n + g, :n + g].copy()  # n^3 block with ghosts
    dh = 1.0 / N
    count = O.count_advance_block_vl if vl else O.count_advance_block
    c = count(C, (n, n, n), (1, 1, 1), 0.4 * dh, dh)
    return {k: v / n ** 3 for k, v in c.items()}


def count(vl=False):
    """Per cell update: the step's count in the large-block limit plus the
    CFL bound of the updated cell, under the EoS currently selected."""
    sizes = (16, 32, 64)
    rows = [per_cell(n, vl=vl) for n in sizes]
    kinds = ("add", "mul", "div", "sqrt")
    A = np.array([[1.0, 1.0 / n, 1.0 / n ** 2] for n in sizes])
    limit = {k: float(np.linalg.solve(A, np.array([r[k] for r in rows]))[0]) for k in kinds}
    W = workloads.advection_prims(32)
    C, _ = O.prim2con(W.reshape(5, -1))
    cfl = {k: v / C.shape[1] for k, v in O.count_cfl(C).items()}
    step = {k: limit[k] + cfl[k] for k in kinds}
    return {
        "per_cell_update_step": limit,
        "per_cell_cfl": cfl,
        "per_cell_update_with_cfl": step,
        "flops_per_cell_update": sum(step.values()),
        "measured_per_cell_at_n": {str(n): r for n, r in zip(sizes, rows)},
    }


def main():
    out = {"workload": "smooth advection, gamma 10 along (1,1,1), T ~ 1"}
    out.update(count())  # MUSCL-Hancock, Taub-Mathews EoS
    out["vl"] = count(vl=True)
    with O.eos(O.EOS_POLYTROPIC, 4.0 / 3.0):
        out["polytropic_gamma_4_3"] = count()
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
