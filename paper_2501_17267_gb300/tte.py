"""Time-to-epsilon (TTeps) scaling of simulated annealing, the protocol of App. D.1,
run on the GPU path.

TTeps of an instance at a target gap eps: the smallest number of sweeps S at which the
optimality gap (Eq. 2) averaged over `runs` independent SA runs (geometric beta
schedule, one read each) is at or below eps.  The paper times that S in wall-clock
seconds on a CPU.  Here the cost of a run is reported two ways: as its work, S sweeps
of N sites (S * N attempts per run), which is what a CPU wall time measures up to a
constant, and as the wall time of the runs at those S on this GPU -- one instance per
call (its `runs` replicas together), and all instances of a size in one batched call
(per instance) -- with the a L^(3 alpha) + b fit on each.  A small run on the GPU is
bound by launch and barrier latency rather than by its work, so the time exponents
differ from the work exponents.

Steps (App. D.1):
  1. For each target eps, tune the beta range on L = 10 instances: for each instance
     and each (beta_min, beta_max) of the grid (beta_min 0.3 .. 3.3 step 0.2, beta_max
     3 .. 27 step 1) find the smallest S reaching eps; keep each instance's best range
     (fewest sweeps) and average the best ranges over the instances.
  2. With that range, find each instance's smallest S at L = 20, 30, 40, 50, 56, average
     the cost over the instances at each L, and fit cost = a L^(3 alpha) + b for the
     scaling exponent alpha(eps) (Sec. III).

The independent runs of one instance are the replicas of one sg_sa_run: each replica
starts from its own random state and draws its own random numbers.  The smallest S
is found by doubling S until the target is met and then bisecting between the last
failing and the first passing S (the mean gap is taken to fall with S inside that
bracket).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

BMIN_GRID = tuple(round(0.3 + 0.2 * k, 1) for k in range(16))  # 0.3 .. 3.3
BMAX_GRID = tuple(float(b) for b in range(3, 28))               # 3 .. 27
SCALING_L = (20, 30, 40, 50, 56)
TARGETS = (0.03, 0.04, 0.05)
F6 = (0.0, 0.0, 1.0)  # tile-class probabilities of the F6-only class (Sec. II)


class SARunner:
    """Mean gaps of SA runs on the GPU path: instances[k] annealed with `runs` replicas.

    __call__(requests) takes (k, sweeps, beta_min, beta_max) tuples and returns the
    mean gap over the replicas of each, running requests with equal parameters as one
    sg_sa_run_batch call."""

    def __init__(self, sg, instances, runs: int = 20, seed: int = 0):
        self.sg = sg
        self.instances = list(instances)
        self.runs = runs
        self.seed = seed
        self.attempts = 0  # work done so far, in spin-flip attempts
        self.calls = 0

    def __call__(self, requests):
        out = [None] * len(requests)
        groups = {}
        for q, (k, S, b0, b1) in enumerate(requests):
            groups.setdefault((int(S), float(b0), float(b1)), []).append((q, k))
        for (S, b0, b1), members in groups.items():
            insts = [self.instances[k] for _, k in members]
            params = [dict(replicas=self.runs, sweeps=S, beta0=b0, beta1=b1, schedule="geometric",
                           seed=self.seed, instance_id=k) for _, k in members]
            res = self.sg.sa_run_batch(insts, params)
            self.calls += 1
            for (q, k), r in zip(members, res):
                out[q] = float(np.mean(r["eps"]))
                self.attempts += self.instances[k].N * self.runs * S
        return out


def min_sweeps(runner, items, target: float, s_max: int = 1 << 16):
    """Smallest S per item (k, beta_min, beta_max) whose mean gap is <= target, or None
    when even s_max sweeps do not reach it.  All items advance together, one batched
    runner call per round."""
    n = len(items)
    lo = [0] * n        # largest S known to fail (0: none tried)
    hi = [None] * n     # smallest S known to pass
    S = [1] * n         # doubling phase: next S to try
    done = [False] * n
    while not all(done):
        reqs, idx = [], []
        for q in range(n):
            if done[q]:
                continue
            if hi[q] is None:
                s = S[q]
            else:
                s = (lo[q] + hi[q]) // 2
            k, b0, b1 = items[q]
            reqs.append((k, s, b0, b1))
            idx.append((q, s))
        eps = runner(reqs)
        for (q, s), e in zip(idx, eps):
            if e <= target:
                hi[q] = s
            else:
                lo[q] = s
                if hi[q] is None:
                    if s >= s_max:
                        done[q] = True  # censored
                        continue
                    S[q] = min(2 * s, s_max)
            if hi[q] is not None and hi[q] - lo[q] <= 1:
                done[q] = True
    return hi


def tune_beta_range(runner, n_inst: int, target: float, bmin_grid=BMIN_GRID, bmax_grid=BMAX_GRID,
                    s_max: int = 1 << 14):
    """The averaged best (beta_min, beta_max) over instances 0 .. n_inst-1 of the runner
    (step 1 of App. D.1), with each instance's best range and its sweeps."""
    ranges = [(b0, b1) for b0 in bmin_grid for b1 in bmax_grid if b1 > b0]
    items = [(k, b0, b1) for k in range(n_inst) for (b0, b1) in ranges]
    S = min_sweeps(runner, items, target, s_max)
    best = []
    for k in range(n_inst):
        cands = [(S[q], items[q][1], items[q][2]) for q in range(len(items)) if items[q][0] == k and S[q]]
        if not cands:
            continue
        s, b0, b1 = min(cands)  # fewest sweeps; ties: the smallest beta_min, then beta_max
        best.append((b0, b1, s))
    if not best:
        return None
    return dict(beta_min=float(np.mean([b[0] for b in best])), beta_max=float(np.mean([b[1] for b in best])),
                per_instance=best, ranges=len(ranges))


def fit_alpha(Ls, cost):
    """Fit cost = a L^(3 alpha) + b (Sec. III); returns (alpha, a, b).  Starts from the
    log-log slope of the two largest L and refines by least squares."""
    from scipy.optimize import curve_fit
    Ls = np.asarray(Ls, dtype=np.float64)
    T = np.asarray(cost, dtype=np.float64)
    order = np.argsort(Ls)
    Ls, T = Ls[order], T[order]
    slope = math.log(T[-1] / T[-2]) / math.log(Ls[-1] / Ls[-2]) if len(Ls) >= 2 else 3.0
    alpha0 = max(slope / 3.0, 0.1)
    a0 = T[-1] / Ls[-1] ** (3 * alpha0)

    def model(L, a, alpha, b):
        return a * L ** (3 * alpha) + b

    (a, alpha, b), _ = curve_fit(model, Ls, T, p0=(a0, alpha0, 0.0), maxfev=20000)
    return float(alpha), float(a), float(b)


@dataclass
class ScalingPoint:
    L: int
    sweeps: list = field(default_factory=list)   # per instance (None: censored)
    cost: float = 0.0                              # mean of S * N over uncensored instances
    wall_s: float = 0.0                            # the search for the sweep counts
    time_one_s: float = float("nan")               # mean wall time of one instance's runs at its S
    time_batched_s: float = float("nan")           # all instances at their S in one call, per instance


def time_runs(sg, insts, sweeps, runs: int, beta_min: float, beta_max: float, seed: int, repeat: int = 3):
    """Wall time of SA at each instance's sweep count (None: skipped) -- the time to the
    target gap: (mean over instances of one sg_sa_run call of `runs` replicas, the call
    of all of them together in one sg_sa_run_batch divided by their number); each the
    best of `repeat` after one untimed call.  The calls return once their results are on
    the host, so host timers measure what a caller waits."""
    items = [(k, S) for k, S in enumerate(sweeps) if S]
    if not items:
        return float("nan"), float("nan")

    def params(k, S):
        return dict(replicas=runs, sweeps=int(S), beta0=beta_min, beta1=beta_max, schedule="geometric",
                    seed=seed, instance_id=k)

    def best(fn):
        fn()
        t = []
        for _ in range(repeat):
            t0 = time.perf_counter()
            fn()
            t.append(time.perf_counter() - t0)
        return min(t)

    one = [best(lambda k=k, S=S: sg.sa_run_batch([insts[k]], [params(k, S)])) for k, S in items]
    batch = best(lambda: sg.sa_run_batch([insts[k] for k, _ in items], [params(k, S) for k, S in items]))
    return float(np.mean(one)), batch / len(items)


def scaling(sg, target: float, beta_min: float, beta_max: float, Ls=SCALING_L, n_inst: int = 20,
            runs: int = 20, seed_base: int = 0, s_max: int = 1 << 17, timed: bool = False):
    """Step 2 of App. D.1 at one target: mean cost per L and the fitted alpha.  timed:
    also the wall times of the runs at the sweep counts found (time_runs), and the fit
    is then a dict of (alpha, a, b) per cost: "work", "time_one_s", "time_batched_s"."""
    points = []
    for L in Ls:
        insts = [sg.Instance.create(L, seed_base + 1000 * L + k, F6, True) for k in range(n_inst)]
        runner = SARunner(sg, insts, runs=runs, seed=seed_base + L)
        t0 = time.perf_counter()
        S = min_sweeps(runner, [(k, beta_min, beta_max) for k in range(n_inst)], target, s_max)
        p = ScalingPoint(L=L, sweeps=S, wall_s=time.perf_counter() - t0)
        ok = [s for s in S if s]
        p.cost = float(np.mean([s * L ** 3 for s in ok])) if ok else float("nan")
        if timed:
            p.time_one_s, p.time_batched_s = time_runs(sg, insts, S, runs, beta_min, beta_max, seed_base + L)
        points.append(p)
        for i in insts:
            i.close()
    fit = None
    good = [p for p in points if np.isfinite(p.cost)]
    if len(good) >= 3:
        fit = fit_alpha([p.L for p in good], [p.cost for p in good])
    if not timed:
        return points, fit
    fits = {"work": fit}
    for key in ("time_one_s", "time_batched_s"):
        g = [p for p in points if np.isfinite(getattr(p, key))]
        fits[key] = fit_alpha([p.L for p in g], [getattr(p, key) for p in g]) if len(g) >= 3 else None
    return points, fits


def main(argv=None):
    import argparse
    import json

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--targets", type=float, nargs="+", default=list(TARGETS))
    ap.add_argument("--tune-L", type=int, default=10)
    ap.add_argument("--tune-instances", type=int, default=20)
    ap.add_argument("--instances", type=int, default=20)
    ap.add_argument("--runs", type=int, default=20)
    ap.add_argument("--L", type=int, nargs="+", default=list(SCALING_L))
    ap.add_argument("--bmin-step", type=int, default=1, help="use every n-th beta_min of the grid")
    ap.add_argument("--bmax-step", type=int, default=1, help="use every n-th beta_max of the grid")
    args = ap.parse_args(argv)
    from . import sg

    out = []
    for eps in args.targets:
        insts = [sg.Instance.create(args.tune_L, 7 * 10 ** 6 + k, F6, True) for k in range(args.tune_instances)]
        runner = SARunner(sg, insts, runs=args.runs, seed=11)
        t0 = time.perf_counter()
        tuned = tune_beta_range(runner, len(insts), eps, BMIN_GRID[::args.bmin_step], BMAX_GRID[::args.bmax_step])
        t_tune = time.perf_counter() - t0
        row = dict(eps=eps, tuning=dict(L=args.tune_L, instances=len(insts), runs=args.runs, seconds=t_tune,
                                        ranges=tuned["ranges"] if tuned else None, attempts=runner.attempts))
        if tuned is None:
            row["error"] = "no beta range reached the target at the tuning size"
            out.append(row)
            continue
        row["beta_min"], row["beta_max"] = tuned["beta_min"], tuned["beta_max"]
        points, fits = scaling(sg, eps, tuned["beta_min"], tuned["beta_max"], args.L, args.instances, args.runs,
                               timed=True)
        row["points"] = [dict(L=p.L, mean_sweeps=float(np.mean([s for s in p.sweeps if s])) if any(p.sweeps) else None,
                              censored=sum(1 for s in p.sweeps if not s), cost_attempts=p.cost,
                              time_one_s=p.time_one_s, time_batched_per_instance_s=p.time_batched_s,
                              search_seconds=p.wall_s)
                         for p in points]
        if fits["work"]:
            row["alpha"], row["a"], row["b"] = fits["work"]
        for key in ("time_one_s", "time_batched_s"):
            if fits[key]:
                row[f"alpha_{key}"] = fits[key][0]
        out.append(row)
        print(json.dumps(row), flush=True)
    return out


if __name__ == "__main__":
    main()
