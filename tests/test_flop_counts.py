"""The algorithmic flop counts behind bench.py's ALU rooflines are the
oracle's operation counts (oracle/count_flops.py) of one cell update of the
benchmark state: MUSCL-Hancock under the Taub-Mathews EoS, the VL
integrator, and MUSCL-Hancock under the polytropic EoS with Gamma = 4/3.
CPU only (oracle)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_flop_constants_are_the_oracle_counts(oracle):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "oracle", "count_flops.py")],
                         capture_output=True, text=True, check=True, cwd=ROOT)
    counts = json.loads(out.stdout)
    sys.path.insert(0, ROOT)
    import bench
    for got, want in ((counts["flops_per_cell_update"], bench.FLOPS_PER_CELL_UPDATE),
                      (counts["vl"]["flops_per_cell_update"], bench.FLOPS_PER_CELL_UPDATE_VL),
                      (counts["polytropic_gamma_4_3"]["flops_per_cell_update"],
                       bench.FLOPS_PER_CELL_UPDATE_POLY)):
        assert abs(got / want - 1) < 5e-4, (got, want)
    # the counts scale with the block as a + b/n + c/n^2 (halo work on the
    # surface): the large-block limit lies below every measured size
    for key in (None, "vl", "polytropic_gamma_4_3"):
        c = counts if key is None else counts[key]
        limit = sum(c["per_cell_update_step"].values())
        assert all(limit < sum(r.values()) for r in c["measured_per_cell_at_n"].values())
