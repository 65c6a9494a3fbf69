"""CPU checks of bench.py's output contract: the reference arm (the float64 oracle timed on the
host cores) prints one JSON line with the fields the benchmark's readers expect, ranks other than
0 print nothing, and the clock sampler turns nvidia-smi rows into the median SM clock and the set
of active throttle reasons."""
import json
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          env=e, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    out = run_bench("--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "1")
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("stereo 64x48")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # value is units per second: 64 x 48 pixels x 16 labels per step
    assert abs(d["value"] - 64 * 48 * 16 / (d["ms_per_step"] / 1e3) / 1e6) <= 1e-9 * d["value"]


def test_reference_arm_other_ranks_exit_quietly():
    out = run_bench("--impl", "reference", "--workload", "small", "--steps", "1", "--warmup", "0",
                    env={"RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_rows_and_reasons():
    sys.path.insert(0, ROOT)
    import bench
    rows = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = bench.ClockSampler(0)
    s.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.file.write("\n".join(rows) + "\n")
    s.proc = _Done()
    c = s.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 4

    s = bench.ClockSampler(0)
    s.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.file.write("0, 1200, 2070, 700, 0x8, Active, Not Active, Active, Not Active\n")
    s.proc = _Done()
    c = s.stop()
    assert c["sm_mhz"] == 1200.0 and c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_reference_sample_and_fp32_peak():
    """The reference arm times the whole workload when its steps fit the time budget (10 steps
    of the 450x375 / 60-label workload) and a proportional centred crop otherwise (the 20 + 5
    steps of a typical short run, and 305); the FP32 peak follows the SM count and clock it is
    given."""
    sys.path.insert(0, ROOT)
    import bench
    w = bench.WORKLOADS["quarter"]
    assert bench.reference_crop(w, 10) == (450, 375)
    for steps in (25, 305):
        cw, ch = bench.reference_crop(w, steps)
        assert cw < 450 and ch < 375 and abs(cw / ch - 450 / 375) < 0.05
        assert cw * ch * 60 * steps <= bench.REFERENCE_BUDGET_S * bench.ORACLE_MPLS_ESTIMATE * 1e6
    # the default line's CPU baseline: about CPU_SAMPLE_S of oracle work in two repetitions
    cw, ch = bench.cpu_sample_crop(w)
    assert cw <= 450 and ch <= 375
    t = 2 * cw * ch * 60 / (bench.ORACLE_MPLS_ESTIMATE * 1e6)
    assert 0.8 * bench.CPU_SAMPLE_S <= t <= bench.CPU_SAMPLE_S
    assert bench.cpu_sample_crop(bench.WORKLOADS["small"]) == (64, 48)
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert abs(bench.fp32_peak_tflops(148, 1800.0) - 148 * 128 * 2 * 1.8e9 / 1e12) < 1e-9
