"""Host side of bench.py without a GPU: the reference arm's JSON line (the
FP64 oracle on the host cores), its silence on ranks other than 0, and the
parsing of the clock and throttle-reason samples taken during a timed region."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run_reference(env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run_reference()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["dtype"] == "f64"
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"],
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value is the 181 x 61 pair count over the step time
    from paper_1709_08803_gb300 import workloads as W
    mesh = W.config_paper_scale(0.7)[0]
    assert d["value"] == pytest.approx(mesh.pair_evals() / (d["ms_per_step"] * 1e-3), rel=1e-9)


def test_reference_arm_is_silent_off_rank_zero():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_give_median_max_and_active_reasons():
    import bench
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
               "2040, 2070, 1300.0, Not Active, Not Active, Not Active, Active",
               "1995, 2070, 1390.5, Not Active, Not Active, Not Active, Active",
               "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active",
               "short line"]
    c = s.stop()
    assert c["sm_mhz"] == 2040.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_samples_report_thermal_slowdown():
    import bench
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = ["1500, 2070, 1000.0, Not Active, Active, Active, Not Active"]
    assert s.stop()["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    import bench
    c = bench.ClockSampler(0).stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
