"""CPU checks of bench.py: the reference arm (the oracle timed on the host
cores) prints one JSON line with the fields the benchmark contract asks for,
and the kernel-source hash that guards the ncu traffic table ignores
comments but not code."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "cell updates/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_source_hash_ignores_comments_only():
    sys.path.insert(0, ROOT)
    import bench
    code = "int f(int a) { return a + 1; }  // add one\n/* block\n comment */ int g;\n"
    same = "int f(int a) {\n  return a + 1;  // add one to a\n}\n/* other */ int g;\n"
    other = "int f(int a) { return a + 2; }\nint g;\n"
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)
    assert len(bench.kernel_sources_sha()) == 16
