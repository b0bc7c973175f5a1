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


def test_roof_picks_the_binding_roof():
    import bench
    # 152 SMs at 2070 MHz: 10.07 T multiplies/s = 8.05e12 attempts/s at 1.25 per attempt;
    # HBM at 6800 GB/s and 0.344 B/attempt allows 1.98e13, so the multiply roof binds
    r = bench._roof(2.0e12, 0.34375, 152, 2070.0, 6800.0, "measured")
    assert r["bound"] == "alu" and r["other_roof"]["bound"] == "hbm"
    assert r["peak"] == pytest.approx(152 * 32 * 2070e6 / 1e12)
    assert r["frac"] == pytest.approx(2.0e12 * 1.25 / 1e12 / r["peak"])
    assert r["other_roof"]["frac"] == pytest.approx(2.0e12 * 0.34375 / 1e9 / 6800.0)
    # 3 B per attempt: HBM allows 2.27e12 attempts/s, below the multiply roof
    assert bench._roof(1.0e12, 3.0, 152, 2070.0, 6800.0, "measured")["bound"] == "hbm"


def test_rng_roof_scales_the_measured_block_rate():
    import bench

    class Fake:
        @staticmethod
        def philox_rate():
            return 5.0e11

    r = bench._rng_roof(Fake, 2.0e12, 16)
    assert r["attempts_per_s"] == pytest.approx(8.0e12) and r["frac"] == pytest.approx(0.25)

    class Broken:
        @staticmethod
        def philox_rate():
            raise RuntimeError("no device")

    assert "error" in bench._rng_roof(Broken, 1.0, 16)
