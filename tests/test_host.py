"""Host-side tests of libsg (no GPU): the C ABI loads and exports every declared
symbol, the host tile-planting generator agrees byte for byte with the oracle's
independent generator, and invalid arguments are rejected before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as o
from paper_2501_17267_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sg():
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg as mod
    return mod


def test_exports_every_declared_symbol(sg):
    declared = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        declared |= set(re.findall(r"^\s*(?:int32_t|const char\*)\s+(sg_\w+)\s*\(", text, re.M))
    assert {"sg_instance_create", "sg_sa_run", "sg_pt_run", "sg_energy"} <= declared
    lib = ctypes.CDLL(sg.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_kernel_kinds_follow_the_header(sg):
    """The binding's launch-statistics kinds are the header's SG_KERNEL_* in index order,
    and reading the counters (host state only) fills every kind."""
    text = open(os.path.join(ROOT, "include", "sg.h")).read()
    defs = {name: int(v) for name, v in re.findall(r"#define SG_KERNEL_(\w+) (\d+)", text)}
    n = defs.pop("KINDS")
    assert sorted(defs.values()) == list(range(n)) and len(sg.KERNEL_KINDS) == n
    for name, idx in defs.items():
        assert sg.KERNEL_KINDS[idx] == name.lower()
    st = sg.stats_read(reset=True)
    assert list(st) == list(sg.KERNEL_KINDS)
    assert all(v["launches"] == 0 and v["units"] == 0 for v in st.values())


@pytest.mark.parametrize("L", [2, 4, 6, 12, 16])
@pytest.mark.parametrize("cp,gauge", [(wl.UNIFORM, True), ((0, 0, 1), True), ((0.3, 0.7, 0), False),
                                      ((0.5, 0, 0.5), True)])
def test_generator_matches_oracle(sg, L, cp, gauge):
    seed = 2 ** 32 * 3 + 17 * L
    inst = sg.Instance.create(L, seed, cp, gauge)
    J3, planted, egs = inst.get()
    J3o, tauo, egso = o.generate(L, seed, cp, gauge)
    assert egs == egso == inst.e_gs
    assert np.array_equal(J3, J3o)
    assert np.array_equal(planted, tauo)


def test_workload_instances_match_oracle(sg):
    for w in (wl.SA_L4, wl.SA_L16):
        inst = sg.Instance.create(w.L, w.instance_seed(0), w.class_prob, True)
        J3, planted, egs = inst.get()
        J3o, tauo, egso = o.generate(w.L, w.instance_seed(0), w.class_prob, True)
        assert np.array_equal(J3, J3o) and egs == egso


def test_from_couplings_roundtrip(sg):
    L = 6
    J3 = wl.random_couplings(5, L, jmax=2)
    inst = sg.Instance.from_couplings(L, J3, e_gs=-123)
    J3b, planted, egs = inst.get()
    assert np.array_equal(J3, J3b) and egs == -123 and (planted == 1).all()


def test_invalid_arguments(sg):
    with pytest.raises(sg.SGError) as e:
        sg.Instance.create(5, 0)
    assert e.value.code == sg.SG_EINVAL
    assert "even" in sg.last_error_string()
    with pytest.raises(sg.SGError):
        sg.Instance.create(0, 0)
    with pytest.raises(sg.SGError):
        sg.Instance.create(4, 0, (-1, 1, 1))
    with pytest.raises(sg.SGError):
        sg.Instance.create(4, 0, (0, 0, 0))
    bad = np.full((64, 3), 3, dtype=np.int8)
    with pytest.raises(sg.SGError) as e:
        sg.Instance.from_couplings(4, bad)
    assert e.value.code == sg.SG_EINVAL
    inst = sg.Instance.create(4, 1)
    for kw in [dict(replicas=0), dict(sweeps=-1), dict(beta0=0.0), dict(beta1=-1.0),
               dict(beta0=float("nan")), dict(schedule=7)]:
        args = dict(replicas=4, sweeps=1, beta0=0.1, beta1=1.0)
        args.update(kw)
        with pytest.raises(sg.SGError) as e:
            sg.sa_run(inst, **args)
        assert e.value.code == sg.SG_EINVAL
    for kw in [dict(temps=0), dict(temps=300), dict(beta_min=0.0), dict(sweeps=-2)]:
        args = dict(temps=4, sweeps=1, beta_min=0.2, beta_max=3.0)
        args.update(kw)
        with pytest.raises(sg.SGError) as e:
            sg.pt_run(inst, **args)
        assert e.value.code == sg.SG_EINVAL


def test_server_rejects_bad_config_and_null_handles(sg):
    for bad in [dict(hbm_budget_bytes=0), dict(max_active=0), dict(chunk_sweeps=0),
                dict(queue_capacity=0)]:
        args = dict(hbm_budget_bytes=1 << 30, max_active=4, chunk_sweeps=10, queue_capacity=8)
        args.update(bad)
        with pytest.raises(sg.SGError) as e:
            sg.Server(**args)
        assert e.value.code == sg.SG_EINVAL
    lib = sg._lib
    req = sg.request(sg.SG_REQ_SA, 8, 1, 8, 0.1, 3.0, 0.0, 10)
    t = ctypes.c_uint64()
    assert lib.sg_submit(None, ctypes.byref(req), ctypes.byref(t)) == sg.SG_EINVAL
    res = sg.Result()
    assert lib.sg_poll(None, 1, 0, ctypes.byref(res)) == sg.SG_EINVAL
    assert lib.sg_cancel(None, 1) == sg.SG_EINVAL
    assert lib.sg_server_destroy(None) == sg.SG_OK


def test_request_bytes_counts_state(sg):
    small = sg.request_bytes(sg.request(sg.SG_REQ_SA, 8, 1, 8, 0.1, 3.0, 0.0, 10))
    wide = sg.request_bytes(sg.request(sg.SG_REQ_SA, 8, 1, 64, 0.1, 3.0, 0.0, 10))
    # spins are bit-packed: one 32-bit word per site for every 32 replicas
    assert small >= 8 ** 3 * 4 and wide - small >= 8 ** 3 * 4
    pt = sg.request_bytes(sg.request(sg.SG_REQ_PT, 16, 1, 32, 0.2, 3.0, 0.0, 10))
    assert pt >= 16 ** 3 * 4
    with pytest.raises(sg.SGError) as e:
        sg.request_bytes(sg.request(sg.SG_REQ_SA, 7, 1, 8, 0.1, 3.0, 0.0, 10))
    assert e.value.code == sg.SG_EINVAL


class _FakeCudaTensor:
    """Stands in for a CUDA tensor on a machine without a GPU: the binding may look at its
    dtype, size, layout and device, never at its memory."""

    def __init__(self, dtype, numel, device=0, contiguous=True):
        import types
        self.is_cuda = True
        self.dtype = dtype
        self._numel = numel
        self._contiguous = contiguous
        self.device = types.SimpleNamespace(index=device)

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contiguous

    def data_ptr(self):
        raise AssertionError("a rejected call must not reach the library")


def test_noalloc_binding_rejects_bad_tensors_before_any_launch(sg, monkeypatch):
    """energy_noalloc checks dtypes, sizes, layout and device of every tensor and raises
    ValueError before anything reaches the device (a wrong dtype or a short buffer would
    otherwise make the kernels read or write out of bounds)."""
    import torch
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(sg._lib, "sg_energy_noalloc", lambda *a: pytest.fail("library called"))
    L, n = 4, 3
    N = L ** 3

    def args(**over):
        a = dict(J3=_FakeCudaTensor(torch.int8, 3 * N), spins=_FakeCudaTensor(torch.int8, n * N),
                 E=_FakeCudaTensor(torch.int64, n))
        a.update(over)
        return a

    bad = [
        args(E=_FakeCudaTensor(torch.int32, n)),               # 4-byte energies
        args(J3=_FakeCudaTensor(torch.int16, 3 * N)),          # wrong coupling dtype
        args(spins=_FakeCudaTensor(torch.float32, n * N)),     # wrong spin dtype
        args(J3=_FakeCudaTensor(torch.int8, 3 * N - 1)),       # short couplings
        args(spins=_FakeCudaTensor(torch.int8, n * N + 1)),    # ragged spins
        args(spins=_FakeCudaTensor(torch.int8, 0), E=_FakeCudaTensor(torch.int64, 0)),  # nothing
        args(E=_FakeCudaTensor(torch.int64, n + 1)),           # energies of the wrong count
        args(spins=_FakeCudaTensor(torch.int8, n * N, device=1)),  # not the current device
        args(J3=_FakeCudaTensor(torch.int8, 3 * N, contiguous=False)),
        args(E=np.zeros(n, dtype=np.int64)),                   # a host array
    ]
    for a in bad:
        with pytest.raises(ValueError):
            sg.energy_noalloc(L, a["J3"], a["spins"], a["E"])
    for badL in (3, 0, 258):
        with pytest.raises(ValueError):
            a = args()
            sg.energy_noalloc(badL, a["J3"], a["spins"], a["E"])
    # the argument set the others were made from passes the checks
    a = args()
    assert sg._check_noalloc_args(L, a["J3"], a["spins"], a["E"]) == n
