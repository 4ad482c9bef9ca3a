"""CPU check of the register budget of the headline kernels. The 384-thread
float patch kernels (the autotuner's usual choice) run two CTAs per SM at the
80-register limit of __launch_bounds__(384, 2), and the 512-thread FP64
kernels one CTA per SM at 128; a spill costs local-memory traffic in the hot
loops. Compiles the mixed_cf and FP64 translation units with ptxas
statistics (nvcc only, no GPU, both at once) and checks that the
ghosted-batch (mode 0), uniform gather (mode 1) and primitive-cache (mode 3)
kernels of those variants, and the float VL kernel, stay within their limit
and spill at most the few words recorded here (the float kernels keep the
packed limiter's operands of two variables live; measured 4 to 12 bytes of
spill stores in modes 0 and 3, 24 in mode 1), nothing in FP64."""
import os
import re
import shutil
import subprocess

import pytest


def _ptxas_stats(stderr):
    stats, cur = {}, None
    for line in stderr.splitlines():
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
    return stats


def _check(stats, key, max_regs, max_spill=0):
    found = [k for k in stats if key in k]
    assert len(found) == 1, (key, sorted(stats)[:5])
    s = stats[found[0]]
    assert s["regs"] <= max_regs and max(s["spill"]) <= max_spill, (key, s)


def test_headline_kernels_do_not_spill(tmp_path):
    from paper_2012_11130_gb300 import build
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    procs = {}
    for tu in ("srhd_mixed_cf", "srhd_fp64"):
        cmd = [nvcc, *build.ARCH, *build.NVCC_FLAGS, "-Xptxas", "-v", "-I", build.INCLUDE, "-I",
               build.CSRC, "-c", os.path.join(build.CSRC, tu + ".cu"), "-o",
               str(tmp_path / (tu + ".o"))]
        procs[tu] = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                     text=True)
    stats = {}
    for tu, p in procs.items():
        _, err = p.communicate()
        assert p.returncode == 0, (tu, err[-2000:])
        stats.update(_ptxas_stats(err))
    for mode, spill in ((0, 8), (1, 24), (3, 16)):
        _check(stats, f"patch_kernelINS_11PrecMixedCFELi384ELi2ELb1ENS_5EosTMELi{mode}E", 80,
               spill)
        _check(stats, f"patch_kernelINS_8PrecFP64ELi512ELi1ELb0ENS_5EosTMELi{mode}E", 128)
    _check(stats, "vl_patch_kernelINS_11PrecMixedCFELi384ELi2ENS_5EosTME", 80)
