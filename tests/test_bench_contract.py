"""bench.py's reference arm (the FP64 oracle on the host cores) without a GPU: one JSON
line with the keys the benchmark contract names, on the workload asked for, and
rank 0 alone printing under a multi-rank launch."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra, env=None):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "small_n65536_d16", "--steps", "2", "--warmup", "1", *extra],
                         capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run()
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["unit"] == "nnz/s" and j["higher_is_better"] is True
    assert j["steps"] == 2 and j["warmup"] == 1 and j["n_gpus"] == 1
    assert j["value"] > 0 and j["ms_per_step"] > 0 and j["dtype"] == "f64"
    assert j["config"]["workload"] == "small_n65536_d16" and j["config"]["d"] == 16
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] == bench_cores()
    assert j["cpu_baseline"]["value"] == j["value"]
    assert 0 < j["config"]["fraction_per_step"] <= 1 / 16
    assert j["e2e"] == {"value": j["value"], "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def bench_cores():
    sys.path.insert(0, ROOT)
    import bench
    return bench.host_cores()


def test_oracle_fraction_step_does_that_fraction_of_the_work():
    """A reference step on fraction f runs the sketch of the first f n rows and the
    contraction over the first f B columns of G: its nonzero count is that of those rows."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1606_05732_gb300 import synth
    X, w = synth.workload_csr("small_n65536_d16")
    dt, k1 = bench.oracle_fraction_step(X, w, 0.25, 2)
    assert dt > 0 and k1 == int(X.row_ptr[X.n // 4])


def test_cpu_baselines_time_the_oracle_and_the_plain_product():
    """The bench's cpu_baseline: the oracle on all host cores and on one, and the plain
    product's oracle on a sample of output rows, labelled as extrapolated to all m rows."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1606_05732_gb300 import synth
    X, w = synth.workload_csr("small_n65536_d16")
    r = bench.cpu_baselines(X, w)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] == bench.host_cores()
    assert r["one_core"]["cores"] == 1 and r["one_core"]["value"] > 0
    p = r["plain_one_core"]
    assert p["extrapolated"] is True and p["cores"] == 1 and p["value"] > 0
    assert "scaled to all 8 rows" in p["sample"]


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT="29511")
    assert _run("--gpus", "2", env=env) == []


def test_clock_record_names_the_throttle_reasons():
    """The clocks record: NVML's event-reason bits mapped to names, median SM clock under
    load, and the error itself in place of reasons where NVML cannot be opened."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(None)
    c.samples, c.max_mhz = [2070.0, 1995.0, 2070.0], 2070.0
    c.reasons = 0x4 | 0x40
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap", "hw_thermal_slowdown"]
    c.reasons = 0
    assert c.summary()["reasons"] == []
    c.error = "nvml unavailable: test"
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvml unavailable: test"]}
