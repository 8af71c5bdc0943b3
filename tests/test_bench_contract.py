"""bench.py's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys a benchmark consumer reads, on the same metric and
unit as the GPU arm; runs on the CPU in a few seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "3", "--cpu-budget", "0.5"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "samples/s"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.WORKLOADS["qnn12"]["desc"]
    assert d["config"]["per_gpu_batch"] == bench.WORKLOADS["qnn12"]["B"]


def test_roofline_fields_from_launch_times():
    """bench.roofline on a synthetic timing record: achieved = the plan's
    adjoint flops x B / reverse passes / launch time; frac against the
    derived FP32 peak (SMs x 128 lanes x 2 flop x clock); the measured
    ceiling of the complex-pair arithmetic, when given, reported beside it
    with its own fraction; the HBM figure as the other bound."""
    import bench
    info = {"adj_flops": 1.0e7, "adj_state_bytes": 32768.0, "adj_passes": 1}
    r = {"info": info, "B": 1000, "n_rev_pass": 10, "pass_rev_ms": 2.5, "sm_count": 152,
         "workload": "qnn12", "kernels": "cpx"}
    peaks = {"sm_max_mhz": 2000.0, "hbm_gbs": 6000.0}
    rl = bench.roofline(r, peaks, "test", ceiling=50.0)
    t = 2.5 / 10 / 1e3
    achieved = 1.0e7 * 1000 / t / 1e12
    assert rl["bound"] == "alu" and abs(rl["achieved"] - achieved) < 1e-9
    assert abs(rl["peak"] - 152 * 128 * 2 * 2000e6 / 1e12) < 1e-9
    assert abs(rl["frac"] - achieved / rl["peak"]) < 1e-12
    assert abs(rl["launch_ms"] - 0.25) < 1e-12 and rl["launches_timed"] == 10
    mc = rl["measured_ceiling"]
    assert mc["value"] == 50.0 and abs(mc["frac"] - achieved / 50.0) < 1e-12
    assert rl["other"]["bound"] == "hbm" and abs(rl["other"]["achieved"] - 32768.0 * 1000 / t / 1e9) < 1e-6
    assert rl["traffic"] == bench.PROFILED_TRAFFIC[("qnn12", "cpx")][0]
    # no ceiling for the general kernels or when none was measured
    assert "measured_ceiling" not in bench.roofline(dict(r, kernels="general"), peaks, "test", ceiling=50.0)
    assert "measured_ceiling" not in bench.roofline(r, peaks, "test")
