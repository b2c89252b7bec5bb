"""bench.py's host-side contract without a GPU: the reference arm (the CPU
oracle as it stands, on the host cores) prints one JSON line with the keys
the benchmark contract asks for, other ranks print nothing, and the ALU
roofline arithmetic (152 SMs x the maximum SM clock / issue slots per
simulated day) gives the peak the JSON line reports."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_arm(env=None):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    return [line for line in out.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_prints_the_contract_line(oracle_lib):
    lines = _reference_arm()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "accepted samples/s" and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "sample" in d["cpu_baseline"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_runs_on_rank_0_only(oracle_lib):
    assert _reference_arm(env=dict(os.environ, RANK="1")) == []


def test_alu_roofline_arithmetic():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    peak = 152 * 2070e6 / (144.0 / 128.0)   # simulated days/s: issue-bound, 144 slots per day
    r = bench.roofline(2.8e8, 1.0, 152, 2070.0, traffic=123)
    assert r["bound"] == "alu" and r["unit"] == "Gsim*days/s" and r["traffic"] == 123
    assert r["peak"] == pytest.approx(peak / 1e9)
    assert r["achieved"] == pytest.approx(280.0)
    assert r["frac"] == pytest.approx(2.8e11 / peak)
    # the SFU bound (18 transcendentals per day at 16 per clock) ties with issue
    assert 18.0 / 16.0 == pytest.approx(144.0 / 128.0)


def test_roofline_counts_each_samples_own_work():
    """A sample's prior draw and initial state (104 issue slots) count as
    104/144 of a simulated day on the issue pipe; days_only_frac leaves them
    out."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    peak = 152 * 2070e6 / (144.0 / 128.0)
    r = bench.roofline(2.8e8, 1.0, 152, 2070.0, samples_per_launch=1.44e6)
    assert r["achieved"] == pytest.approx((2.8e8 + 1.04e6) / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx((2.8e11 + 1.04e9) / peak)
    assert r["days_only_frac"] == pytest.approx(2.8e11 / peak)
    assert bench.OPS_PER_SAMPLE["sfu"] == 0.0
