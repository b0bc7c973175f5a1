"""Runs oracle jobs side by side on the host cores.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests and the CPU-baseline
leg of ``bench.py`` use it to compare whole workloads (all instances, all replicas)
with the CUDA path in reasonable time.  Each job is one plain sequential oracle call
(``oracle.sa_run`` / ``oracle.pt_run``); nothing is split below what the oracle itself
computes, so the results are the oracle's own.

The pool is always a ``spawn`` pool: a process forked after CUDA has been initialised
in its parent can hang, and the callers are GPU tests.  It is a process-pool executor,
so a worker that dies raises BrokenProcessPool in the caller instead of leaving it
waiting.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor


def _pt_job(args):
    L, J3, seed, iid, K, S, bmin, bmax = args
    from oracle import oracle as o
    return o.pt_run(L, J3, seed, iid, K, S, bmin, bmax)


def _sa_job(args):
    L, J3, seed, iid, S, b0, b1, geometric, reps, keep_spins = args
    from oracle import oracle as o
    spins, E = o.sa_run(L, J3, seed, iid, S, b0, b1, geometric, reps=reps)
    return (spins if keep_spins else None), E


def workers(n_jobs: int) -> int:
    return max(1, min(n_jobs, os.cpu_count() or 1))


def _run(fn, jobs, cost):
    """fn over jobs in a spawn pool, largest cost first (one job at a time per worker);
    results in the order of `jobs`."""
    from oracle import oracle as o
    o.build()  # compile once here, not in every worker
    order = sorted(range(len(jobs)), key=lambda k: -cost[k])
    with ProcessPoolExecutor(workers(len(jobs)), mp_context=mp.get_context("spawn")) as ex:
        got = list(ex.map(fn, [jobs[k] for k in order]))
    out = [None] * len(jobs)
    for k, r in zip(order, got):
        out[k] = r
    return out


def pt_runs(jobs):
    """jobs: tuples (L, J3, seed, instance_id, K, S, beta_min, beta_max) -> the oracle's
    pt_run dicts, in order."""
    return _run(_pt_job, jobs, [j[0] ** 3 * j[4] * j[5] for j in jobs])


def sa_runs(jobs):
    """jobs: tuples (L, J3, seed, instance_id, S, beta0, beta1, geometric, reps,
    keep_spins) -> (spins or None, E) per job, in order."""
    return _run(_sa_job, jobs, [j[0] ** 3 * len(j[8]) * max(j[4], 1) for j in jobs])
