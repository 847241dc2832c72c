"""Host logic of bench.py, CPU only: the reference arm (the FP64 oracle timed on the host
cores) prints one JSON line with the keys the benchmark line carries, on the same metric,
unit and workload as the GPU arm, and ranks other than 0 print nothing and exit 0; the
clock sampler reduces nvidia-smi rows to the median SM clock and the throttle reasons
seen."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_line_contract():
    lines = _run(None, "--steps", "2", "--warmup", "1")
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.HEADLINE_METRIC and d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"].startswith("thgem_cell N=9996 images=25 points=1000000")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["vs_baseline"] is None


def test_reference_other_ranks_silent():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "0") == []


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_reduces_rows():
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    na, act = "Not Active", "Active"
    cs.rows = [
        ["0", "2070", "2070", "900.1", "0x0", na, na, na, na],
        ["0", "2055", "2070", "1390.0", "0x4", na, na, na, act],
        ["0", "2070", "2070", "1400.0", "0x4", na, na, na, act],
        ["0", "[N/A]", "2070", "1.0", "0x0", na, na, na, na],
    ]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 4
    assert out["reasons"] == ["sw_power_cap"]
    cs.rows.append(["0", "1500", "2070", "700.0", "0x48", act, na, act, na])
    assert bench.ClockSampler.stop(cs)["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    none = bench.ClockSampler(0)
    assert none.stop()["reasons"] == ["nvidia-smi unavailable"]
