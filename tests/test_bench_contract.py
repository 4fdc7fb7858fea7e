"""The benchmark's reference arm (the CPU oracle timed on the host cores) prints
one JSON line with the contract's keys.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-depth-max", "6"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "contractions/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["n"] == 50 and d["steps"] == 1
    # the value is the uniform mix over the depths sampled, each depth measured
    per = d["cpu_baseline"]["per_depth"]
    assert sorted(int(k) for k in per) == [2, 3, 4, 5, 6]
    rates = [v["pairs_per_s"] for v in per.values()]
    assert abs(d["value"] - 1.0 / (sum(1.0 / r for r in rates) / len(rates))) < 1e-9 * d["value"]
