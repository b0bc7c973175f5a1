"""The energy entry point that allocates no device memory.

It serves callers that cannot let the library call cudaMalloc (a server that owns
the device-memory budget through its own pool, a latency-critical loop).  Its
results must equal those of the allocating entry point, call after call, although
every call reuses the same fixed scratch array.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2501_17267_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg
    return sg, torch


def test_noalloc_energy_matches_allocating_entry_point(env):
    sg, torch = env
    L = 16
    inst = sg.Instance.create(L, 31337)
    J3, tau, egs = inst.get()
    J3_dev = torch.from_numpy(J3).cuda()
    # two calls in a row with different sizes and contents: the second must not see the
    # first call's sums left in the shared scratch
    for k, n in enumerate((7, 5)):
        spins = wl.random_spins(100 + k, (n, L ** 3))
        if k == 0:
            spins[0] = tau  # the planted state reaches E_gs
        ref = sg.energy(inst, spins)
        E_dev = torch.zeros(n, dtype=torch.int64, device="cuda")
        spins_dev = torch.from_numpy(spins).cuda()
        # settle every earlier allocation and release (a device-wide synchronisation also
        # trims stream-ordered pools) before looking at free device memory
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        sg.energy_noalloc(L, J3_dev, spins_dev, E_dev)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        got = E_dev.cpu().numpy()
        assert np.array_equal(got, ref)
        if k == 0:
            assert got[0] == egs
        else:
            # the scratch lookup happened on the first call; this one allocates nothing
            assert free_after == free_before


def test_noalloc_energy_rejects_oversized_requests(env):
    sg, torch = env
    # L = 64 with 512 configurations: 9 L^3 + 16 words of 4 L^3 bytes, about 19 MB
    L, n = 64, 512
    J3_dev = torch.zeros((L ** 3, 3), dtype=torch.int8, device="cuda")
    spins = torch.ones((n, L ** 3), dtype=torch.int8, device="cuda")
    E_dev = torch.zeros(n, dtype=torch.int64, device="cuda")
    with pytest.raises(sg.SGError) as e:
        sg.energy_noalloc(L, J3_dev, spins, E_dev)
    assert e.value.code == sg.SG_EINVAL
    assert "scratch" in str(e.value)
