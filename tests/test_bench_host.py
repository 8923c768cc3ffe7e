"""Host logic of bench.py, on the CPU: the reference arm's JSON line (the FP64
oracle timed on the host cores) and the clock sampler's summary of
nvidia-smi's CSV lines."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line(oracle_mod):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "dtype", "data"):
        assert key in line, key
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and line["dtype"] == "f64"
    assert "bounded sample per step" in line["config"]["workload"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary():
    """Median SM clock under load, the largest maximum clock, and the reasons
    seen active in any sample; lines that do not parse are skipped."""
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "[N/A]",
    ]
    out = cs.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.lines.append("0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active")
    out = cs.stop()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and out["samples"] == 4
    assert cs.__class__(0).stop()["reasons"] == ["nvidia-smi unavailable"]
