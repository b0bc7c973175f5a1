"""bench.py's JSON contract on CPU: the reference arm (the oracle on host cores) prints
one line with the keys the contract names, and the roofline helpers compute what they
state."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-sweeps", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [x for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["gpus_used"] == 0
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("pt_L64")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roof_is_measured_generator_rate():
    import bench
    # a sweep kernel at 2e12 attempts/s: 16 attempts per Philox block of 20 multiplies is
    # 1.25 multiplies per attempt; against a measured 5.45e11 blocks/s (10.9 T multiplies/s)
    r = bench._roof(2.0e12, 16, bench.hbm_views(32), 5.45e11, 152, 2070.0, 6800.0, "measured")
    assert r["bound"] == "alu" and r["peak_source"].startswith("measured")
    assert r["peak"] == pytest.approx(5.45e11 * 20 / 1e12)
    assert r["achieved"] == pytest.approx(2.0e12 * 1.25 / 1e12)
    assert r["frac"] == pytest.approx(2.0e12 / (16 * 5.45e11))
    assert r["peak_attempts_per_s"] == pytest.approx(16 * 5.45e11)
    assert r["nominal_peak"]["value"] == pytest.approx(152 * 32 * 2070e6 / 1e12)
    v = r["hbm_views"]
    assert v["int8_layout"]["bytes_per_attempt"] == pytest.approx(2 + 3 / 32)
    assert v["bit_packed"]["bytes_per_attempt"] == pytest.approx(0.25 + 3 / 32)
    assert v["bit_packed"]["frac"] == pytest.approx(2.0e12 * (0.25 + 3 / 32) / 1e9 / 6800.0)
    # without the measurement the nominal peak stands in, and says so
    d = bench._roof(2.0e12, 16, {}, None, 152, 2070.0, 6800.0, "measured")
    assert d["peak_source"].startswith("derived") and d["peak"] == pytest.approx(d["nominal_peak"]["value"])


def test_censored_percentiles_count_capped_requests_as_not_reached():
    import bench
    # 10 requests, 6 reached: p50 is the 5th smallest time, p95 and p99 fall among the capped
    r = bench._pcts_censored([6.0, 1.0, 5.0, 2.0, 4.0, 3.0], 10)
    assert r["p50"] == 5.0 and r["p95"] is None and r["p99"] is None
    assert r["censored"] == ["p95", "p99"] and r["censored_fraction"] == pytest.approx(0.4)
    # more than half capped: the median itself is censored
    assert bench._pcts_censored([1.0, 2.0], 10)["p50"] is None
    full = bench._pcts_censored([float(x) for x in range(1, 101)], 100)
    assert (full["p50"], full["p95"], full["p99"]) == (50.0, 95.0, 99.0)
