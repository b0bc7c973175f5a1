"""Sweep launches with and without programmatic dependent launch (SG_PDL, read once per
process): graph-captured SA and PT runs give bit-identical results either way, and the
plain launches match the oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as o

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (kind, L, instance seed, replicas or temperatures, sweeps, run seed, instance id)
CASES = [
    ("pt", 4, 7600, 8, 230, 17, 5),     # three graph chunks, the last one shorter
    ("pt", 64, 2 ** 32, 32, 20, 0, 0),  # the L = 64, 32-temperature geometry, one chunk
    ("pt", 16, 7801, 128, 20, 29, 6),   # four words per site
    ("sa", 6, 7601, 40, 251, 19, 2),    # SA through the row kernel
]

_CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, ".")
from paper_2501_17267_gb300 import sg
cases = eval(sys.argv[2])
out = {}
for n, (kind, L, iseed, width, S, seed, iid) in enumerate(cases):
    inst = sg.Instance.create(L, iseed)
    out[f"{n}_J3"] = inst.get()[0]
    if kind == "pt":
        r = sg.pt_run(inst, width, S, 0.2, 3.0, seed, iid, spins="host")
        keys = ("spins", "E", "perm", "accepts", "minE")
    else:
        r = sg.sa_run(inst, width, S, 0.1, 3.0, "geometric", seed, iid, spins="host")
        keys = ("spins", "E")
    for k in keys:
        out[f"{n}_{k}"] = np.asarray(r[k])
np.savez(sys.argv[1], **out)
"""


def _run_child(tmp_path, pdl):
    path = str(tmp_path / f"pdl{pdl}.npz")
    env = dict(os.environ, SG_PDL=str(pdl), SG_SA_CLUSTER="0", SG_PT_CLUSTER="0")
    p = subprocess.run([sys.executable, "-c", _CHILD, path, repr(CASES)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    return np.load(path)


def test_dependent_launch_changes_no_result(tmp_path):
    from paper_2501_17267_gb300 import build
    build.build()
    plain = _run_child(tmp_path, 0)
    overlapped = _run_child(tmp_path, 1)
    assert sorted(plain.files) == sorted(overlapped.files)
    for k in plain.files:
        assert np.array_equal(plain[k], overlapped[k]), k
    # the plain launches against the oracle: both PT cases with one ladder (the L = 64,
    # 32-temperature geometry included) and the SA case, the oracle runs side by side
    from oracle import pool
    pt_cases = (0, 1)
    refs = pool.pt_runs([(CASES[n][1], plain[f"{n}_J3"], CASES[n][5], CASES[n][6], CASES[n][3], CASES[n][4],
                          0.2, 3.0) for n in pt_cases])
    for n, ref in zip(pt_cases, refs):
        for k in ("spins", "E", "perm", "accepts"):
            assert np.array_equal(plain[f"{n}_{k}"], ref[k]), (n, k)
        assert int(plain[f"{n}_minE"]) == ref["minE"], n
    kind, L, iseed, width, S, seed, iid = CASES[3]
    ospins, oE = o.sa_run(L, plain["3_J3"], seed, iid, S, 0.1, 3.0, True, R=width)
    assert np.array_equal(plain["3_spins"], ospins)
    assert np.array_equal(plain["3_E"], oE)


def test_generator_rate_is_measured():
    """sg_philox_rate: a positive, finite block rate; invalid arguments rejected."""
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg
    rate = sg.philox_rate(256)
    assert np.isfinite(rate) and rate > 1e9
    for bad in (0, 1, 3, -2):
        with pytest.raises(sg.SGError) as e:
            sg.philox_rate(bad)
        assert e.value.code == sg.SG_EINVAL
