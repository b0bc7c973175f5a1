"""Time-to-epsilon protocol (App. D.1): host logic on fakes (CPU), a small run on the GPU."""
import math

import numpy as np
import pytest

from paper_2501_17267_gb300 import tte


class FakeRunner:
    """Mean gap eps_k(S) = c_k / S (falls with S); counts calls and requests."""

    def __init__(self, c):
        self.c = c
        self.calls = 0
        self.requests = 0

    def __call__(self, requests):
        self.calls += 1
        self.requests += len(requests)
        return [self.c[k] / S for (k, S, b0, b1) in requests]


def test_min_sweeps_finds_the_smallest_passing_count():
    c = [0.5, 3.0, 7.7, 40.0, 1e9]
    target = 0.05
    S = tte.min_sweeps(FakeRunner(c), [(k, 1.0, 5.0) for k in range(len(c))], target, s_max=1 << 12)
    for k, s in enumerate(S):
        exact = math.ceil(c[k] / target - 1e-12)
        if exact > 1 << 12:
            assert s is None  # censored at s_max
        else:
            assert s == exact


def test_min_sweeps_when_one_sweep_suffices():
    assert tte.min_sweeps(FakeRunner([0.01]), [(0, 1.0, 5.0)], 0.05) == [1]


def test_fit_alpha_recovers_known_exponents():
    Ls = [20, 30, 40, 50, 56]
    for alpha, a, b in [(0.8, 3.0, 50.0), (1.25, 0.2, -10.0), (1.0, 1.0, 0.0)]:
        T = [a * L ** (3 * alpha) + b for L in Ls]
        al, aa, bb = tte.fit_alpha(Ls, T)
        assert al == pytest.approx(alpha, rel=1e-6)
        assert aa == pytest.approx(a, rel=1e-5)
        assert bb == pytest.approx(b, abs=1e-3 * max(1.0, abs(b)))


def test_tune_beta_range_averages_the_best_ranges():
    """Instance k needs fewest sweeps at (bmin*, bmax*) = optima[k]; the tuned range is
    the mean of the optima."""
    optima = [(0.5, 5.0), (0.9, 7.0), (1.3, 6.0)]

    class RangeRunner:
        def __call__(self, requests):
            out = []
            for k, S, b0, b1 in requests:
                o0, o1 = optima[k]
                need = 10 + 100 * abs(b0 - o0) + 10 * abs(b1 - o1)
                out.append(need / S * 0.05)  # passes 0.05 from S = need on
            return out

    res = tte.tune_beta_range(RangeRunner(), 3, 0.05, bmin_grid=(0.5, 0.7, 0.9, 1.1, 1.3),
                              bmax_grid=(5.0, 6.0, 7.0), s_max=1 << 12)
    assert res["beta_min"] == pytest.approx(np.mean([o[0] for o in optima]))
    assert res["beta_max"] == pytest.approx(np.mean([o[1] for o in optima]))
    assert [(b0, b1) for b0, b1, s in res["per_instance"]] == optima


def test_runner_groups_equal_requests():
    calls = []

    class FakeSG:
        @staticmethod
        def sa_run_batch(insts, params):
            calls.append([p["sweeps"] for p in params])
            return [{"eps": np.full(p["replicas"], 0.01 * p["sweeps"])} for p in params]

    class Inst:
        N = 64

    r = tte.SARunner(FakeSG, [Inst(), Inst(), Inst()], runs=4)
    eps = r([(0, 8, 1.0, 5.0), (1, 8, 1.0, 5.0), (2, 16, 1.0, 5.0)])
    assert eps == [pytest.approx(0.08), pytest.approx(0.08), pytest.approx(0.16)]
    assert sorted(map(sorted, calls)) == [[8, 8], [16]]
    assert r.attempts == 64 * 4 * (8 + 8 + 16)


@pytest.mark.gpu
def test_min_sweeps_on_the_gpu_is_the_first_passing_count():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg
    insts = [sg.Instance.create(6, 5000 + k, tte.F6, True) for k in range(3)]
    runner = tte.SARunner(sg, insts, runs=8, seed=3)
    target = 0.08
    S = tte.min_sweeps(runner, [(k, 0.5, 5.0) for k in range(3)], target, s_max=1 << 10)
    for k, s in enumerate(S):
        assert s is not None
        mean = lambda n: float(np.mean(sg.sa_run(insts[k], 8, n, 0.5, 5.0, "geometric", 3, k)["eps"]))
        assert mean(s) <= target
        if s > 1:
            assert mean(s - 1) > target
    tuned = tte.tune_beta_range(runner, 3, target, bmin_grid=(0.3, 0.9), bmax_grid=(3.0, 5.0), s_max=1 << 10)
    assert 0.3 <= tuned["beta_min"] <= 0.9 and 3.0 <= tuned["beta_max"] <= 5.0


def test_time_runs_times_each_instance_and_the_batch(monkeypatch):
    """time_runs: one call per instance at its own sweep count (censored ones skipped), and
    one batched call of all of them; the batched time is per instance."""
    calls = []

    class FakeSG:
        @staticmethod
        def sa_run_batch(insts, params):
            calls.append([(i, p["sweeps"], p["instance_id"]) for i, p in zip(insts, params)])
            return [{}] * len(insts)

    clock = iter(float(t) for t in range(1000))
    monkeypatch.setattr(tte.time, "perf_counter", lambda: next(clock))
    one, batched = tte.time_runs(FakeSG, ["a", "b", "c"], [5, None, 9], runs=20, beta_min=1.0, beta_max=9.0,
                                 seed=3, repeat=2)
    # every timed call reads the clock twice, one unit apart
    assert one == 1.0 and batched == 0.5
    singles = [c for c in calls if len(c) == 1]
    assert {c[0] for c in singles} == {("a", 5, 0), ("c", 9, 2)} and len(singles) == 2 * 3
    assert [c for c in calls if len(c) == 2] == [[("a", 5, 0), ("c", 9, 2)]] * 3
    # nothing to time when every instance was censored
    o, b = tte.time_runs(FakeSG, ["a"], [None], 20, 1.0, 9.0, 3)
    assert math.isnan(o) and math.isnan(b)
