"""Host logic of bench.py that needs no GPU: the reference arm's JSON line (the oracle
timed on the host cores), its behaviour on non-zero ranks, the Clopper-Pearson
interval behind the FER checks and the parsing of the clock samples."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(extra_env):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--ref-frames-per-point", "8"],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_contract_line():
    p = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d
    assert d["unit"] == "frames/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # 8 frames x 11 points x 2 codes per step
    assert d["config"]["frames_per_point"] == 8 and d["config"]["points"] == 11


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_clopper_pearson_closed_forms():
    # k = 0: upper bound 1 - (a/2)^(1/n); k = n: lower bound (a/2)^(1/n)
    n, a = 50, 0.05
    lo, hi = bench.clopper_pearson(0, n, a)
    assert lo == 0.0 and hi == pytest.approx(1 - (a / 2) ** (1 / n), rel=1e-9)
    lo, hi = bench.clopper_pearson(n, n, a)
    assert hi == 1.0 and lo == pytest.approx((a / 2) ** (1 / n), rel=1e-9)
    lo, hi = bench.clopper_pearson(10, 100, a)
    assert lo < 0.1 < hi


def test_clock_samples_are_parsed_and_reasons_collected():
    s = bench.ClockSampler(0)
    s.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: None})()
    s.lines = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 1350.0, Not Active, Not Active, Not Active, Active",
               "garbage",
               "2070, 2070, 1380.2, Not Active, Not Active, Not Active, Active"]
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
