"""GPU parity at the benchmarked workloads, through the calls and launch settings the
benchmark times, against the CPU oracle run on all host cores (a spawn pool, one plain
oracle call per job).

- PT, 16 instances at L = 64, 32 temperatures, geometric beta 0.2 -> 3.0 (App. D.2):
  the batched call over all 16 instances for 101 sweeps, i.e. a CUDA graph of 100
  sweeps and a second one of 1, programmatic dependent launch on, the exchange fused
  into the colour-1 launch; every instance's energies, slot permutation, swap counts
  and minimum energy, and all spins.
- SA, one L = 16 instance, 1024 replicas, 1000 sweeps, beta linear 0.1 -> 3.0
  (App. D.1): every replica, spins and energies (the thread-block-cluster kernel).
- 512 uneven SA instances (L in {8, 12, 16, 24, 32, 48}, 64 replicas): the whole mix
  in one persistent launch of the cluster form (C = 4, the form the autotuner picks
  for this mix), with each instance's sweeps cut to a few so the oracle finishes;
  every replica's energy, and the spins of two instances.

The bar is bit-exact: every value is an integer or an integer compare.
"""
import numpy as np
import pytest

from oracle import oracle as o
from oracle import pool
from paper_2501_17267_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg as mod
    return mod


PT_SWEEPS = 101  # one graph of 100 sweeps, then one of a single sweep


def test_pt_benchmarked_batch_every_instance(sg):
    w = wl.PT_L64
    insts = [sg.Instance.create(w.L, w.instance_seed(k), w.class_prob, True) for k in range(w.instances)]
    params = [dict(temps=w.temps, sweeps=PT_SWEEPS, beta_min=w.beta_min, beta_max=w.beta_max,
                   seed=w.run_seed, instance_id=k) for k in range(w.instances)]
    # exactly the benchmark's call (no spin output), then the same with spins
    timed = sg.pt_run_batch(insts, params)
    full = sg.pt_run_batch(insts, params, spins="host")
    host = [i.get() for i in insts]
    refs = pool.pt_runs([(w.L, J3, w.run_seed, k, w.temps, PT_SWEEPS, w.beta_min, w.beta_max)
                         for k, (J3, _, _) in enumerate(host)])
    for k, (ref, a, b) in enumerate(zip(refs, timed, full)):
        egs = host[k][2]
        for got in (a, b):
            assert np.array_equal(got["E"], ref["E"]), k
            assert np.array_equal(got["perm"], ref["perm"]), k
            assert np.array_equal(got["accepts"], ref["accepts"]), k
            assert got["minE"] == ref["minE"], k
            assert got["min_eps"] == o.epsilon(ref["minE"], egs), k
        assert np.array_equal(b["spins"], ref["spins"]), k
    # the exchange ran: swaps were accepted (at the cold end of the ladder; with L = 64
    # and 32 rungs the hot end's energy gaps make swaps there all but impossible)
    acc = np.sum([r["accepts"] for r in refs], axis=0)
    assert acc.sum() > 0 and (acc[w.temps // 2:] > 0).all()


def test_sa_L16_every_replica(sg):
    w = wl.SA_L16
    inst = sg.Instance.create(w.L, w.instance_seed(0), w.class_prob, True)
    J3, _, egs = inst.get()
    res = sg.sa_run(inst, w.replicas, w.sweeps, w.beta0, w.beta1, "linear", w.run_seed, 0, spins="host")
    chunks = [list(range(r, min(r + 32, w.replicas))) for r in range(0, w.replicas, 32)]
    refs = pool.sa_runs([(w.L, J3, w.run_seed, 0, w.sweeps, w.beta0, w.beta1, False, reps, True)
                         for reps in chunks])
    spins = np.concatenate([s for s, _ in refs])
    E = np.concatenate([e for _, e in refs])
    assert np.array_equal(res["spins"], spins)
    assert np.array_equal(res["E"], E)
    assert all(res["eps"][r] == o.epsilon(int(E[r]), egs) for r in range(w.replicas))


# sweeps of the 512-instance mix cut so that the oracle finishes: 100 -> 2, 1000 -> 3, 10^4 -> 4
BATCH_TRUNC = {100: 2, 1000: 3, 10000: 4}


def test_batched_512_uneven_cluster_form(sg, monkeypatch, tmp_path):
    w = wl.BATCHED
    shapes = [(L, BATCH_TRUNC[S]) for L, S in w.draw()]
    insts = [sg.Instance.create(L, w.instance_seed(k), w.class_prob, True) for k, (L, _) in enumerate(shapes)]
    params = [dict(replicas=w.replicas, sweeps=S, beta0=w.beta0, beta1=w.beta1, schedule="linear", seed=0,
                   instance_id=k) for k, (_, S) in enumerate(shapes)]
    monkeypatch.setenv("SG_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setenv("SG_BATCH_WG", "0")  # one-word planes on thread-block clusters
    got = sg.sa_run_batch(insts, params)
    spin_check = [int(np.argmax([L for L, _ in shapes])), 1]  # a largest instance, and another
    with_spins = sg.sa_run_batch(insts, params, spins=["host" if k in spin_check else None
                                                       for k in range(len(insts))])
    monkeypatch.setenv("SG_BATCH_WG", "")  # the autotuned choice gives the same bytes
    tuned = sg.sa_run_batch(insts, params)
    host = [i.get() for i in insts]
    reps = list(range(w.replicas))
    refs = pool.sa_runs([(L, host[k][0], 0, k, S, w.beta0, w.beta1, False, reps, k in spin_check)
                         for k, (L, S) in enumerate(shapes)])
    for k, (spins, E) in enumerate(refs):
        egs = host[k][2]
        assert np.array_equal(got[k]["E"], E), k
        assert np.array_equal(with_spins[k]["E"], E), k
        assert np.array_equal(tuned[k]["E"], E), k
        assert all(got[k]["eps"][r] == o.epsilon(int(E[r]), egs) for r in range(0, w.replicas, 7)), k
        if k in spin_check:
            assert np.array_equal(with_spins[k]["spins"], spins), k
