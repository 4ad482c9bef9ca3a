"""CPU check of the register budget of the headline kernels: the 448-thread
float patch kernels run two CTAs per SM at the 72-register limit of
__launch_bounds__(448, 2), and a spill there costs local-memory traffic in
the hot loops. Compiles the mixed_cf translation unit with ptxas statistics
(nvcc only, no GPU) and checks that the ghosted-batch (mode 0), uniform
gather (mode 1) and primitive-cache (mode 3) kernels of that variant use 72
registers and spill nothing."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_headline_kernels_do_not_spill(tmp_path):
    from paper_2012_11130_gb300 import build
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    cmd = [nvcc, *build.ARCH, *build.NVCC_FLAGS, "-Xptxas", "-v", "-I", build.INCLUDE, "-I",
           build.CSRC, "-c", os.path.join(build.CSRC, "srhd_mixed_cf.cu"), "-o",
           str(tmp_path / "cf.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    stats = {}
    cur = None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\w+)'", line)
        if m:
            cur = m.group(1)
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            stats.setdefault(cur, {})["spill"] = (int(m.group(1)), int(m.group(2)))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            stats.setdefault(cur, {})["regs"] = int(m.group(1))
    for mode in (0, 1, 3):
        key = f"patch_kernelINS_11PrecMixedCFELi448ELi2ELb1ENS_5EosTMELi{mode}E"
        found = [k for k in stats if key in k]
        assert len(found) == 1, (key, list(stats)[:5])
        s = stats[found[0]]
        assert s["regs"] <= 72 and s["spill"] == (0, 0), (mode, s)
