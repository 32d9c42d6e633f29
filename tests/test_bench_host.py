"""Host-side logic of the benchmark, on the CPU: the reference arm (the FP64 oracle on the host
cores, one bounded step of the 13,824-atom workload) prints one JSON line of the benchmark's form
on rank 0 and nothing on the other ranks; the clock samples taken during the timed region are
reduced to the median and maximum SM clock and the set of active slowdown reasons."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def run_bench(args, env):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=900, env=dict(os.environ, **env))


def test_reference_arm_line_on_rank_0():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert all(k in d for k in KEYS), sorted(set(KEYS) - set(d))
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["vs_baseline"] is None
    assert d["config"]["workload"] == "si13824_dc1728_72cube_ns528_m20"
    assert d["config"]["subdomains"] == 1728 and d["config"]["points_per_subdomain"] == 72 ** 3
    assert d["config"]["states"] == 528 and d["config"]["degree"] == 20
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_silent_on_other_ranks():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


class _Stopped:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _parse(tmp_path, text):
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    with open(cs.path, "w") as f:
        f.write(text)
    cs.proc = _Stopped()
    cs.f = open(os.devnull, "w")
    return cs.stop()


def test_clock_samples_reduced(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits rows: index, sm, max sm, power, active mask, then the
    # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown and sw_power_cap flags
    rows = ["0, 1980, 2070, 905.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1935, 2070, 1391.20, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1950, 2070, 1200.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 1200.00, 0x0, Not Active, Not Active, Not Active, Not Active",
            "short line"]
    out = _parse(tmp_path, "\n".join(rows) + "\n")
    assert out["sm_mhz"] == 1950.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_samples_report_thermal_and_hardware_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1100.00, 0x08, Active, Not Active, Not Active, Not Active",
            "0, 1400, 2070, 1100.00, 0x48, Not Active, Not Active, Active, Not Active"]
    out = _parse(tmp_path, "\n".join(rows) + "\n")
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1450.0


def test_clock_sampler_without_nvidia_smi():
    sys.path.insert(0, ROOT)
    import bench
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
