"""Optimality gap of the fragment meta-heuristic vs lattice size (Sec. II, Fig. 2),
with SA fragment anneals on the GPU path.

For each L, `instances` F6-only instances (Sec. II) are solved by sg_fragment_run with
cubic fragments of side l; the gap eps (Eq. 2) of each is averaged, and the mean gaps
are fitted to a / L + b (the paper's form: boundary spins over bulk spins), b being the
asymptotic gap eps_lin.  L must be a multiple of l.
"""
from __future__ import annotations

import time

import numpy as np

F6 = (0.0, 0.0, 1.0)


def fit_inverse_L(Ls, eps):
    """Least squares for eps = a / L + b; returns (a, b)."""
    A = np.stack([1.0 / np.asarray(Ls, dtype=np.float64), np.ones(len(Ls))], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, np.asarray(eps, dtype=np.float64), rcond=None)
    return float(a), float(b)


def gap_vs_L(sg, Ls, l: int = 5, sweeps: int = 20, beta0: float = 0.5, beta1: float = 6.0,
             instances: int = 20, seed_base: int = 9 * 10 ** 6, tropical: bool = False):
    """Mean gap and throughput at each L, and the a / L + b fit.  tropical: exact
    zero-temperature cube marginals (l <= 3) instead of SA anneals; the rate is then in
    enumerated cube states per second."""
    rows = []
    for L in Ls:
        insts = [sg.Instance.create(L, seed_base + 1000 * L + k, F6, True) for k in range(instances)]
        params = [dict(l=l, sweeps=sweeps, beta0=beta0, beta1=beta1, seed=1, instance_id=k)
                  for k in range(instances)]
        sg.fragment_run_batch(insts[:1], params[:1], tropical=tropical)  # warm-up
        t0 = time.perf_counter()
        res = sg.fragment_run_batch(insts, params, tropical=tropical)
        dt = time.perf_counter() - t0
        eps = np.array([r["eps"] for r in res])
        V = l ** 3
        if tropical:
            attempts = instances * (L ** 3 // V) * sum(2 ** (V - w) for w in range(V))
        else:
            attempts = instances * L ** 3 * 32 * sweeps * (V + 1) / 2
        rows.append(dict(L=L, mean_eps=float(eps.mean()), std_eps=float(eps.std()), seconds=dt,
                         attempts_per_s=attempts / dt, instances=instances))
        for i in insts:
            i.close()
    a, b = fit_inverse_L([r["L"] for r in rows], [r["mean_eps"] for r in rows])
    return rows, dict(a=a, eps_lin=b)


def gallus_class_prob(family: str, p6: float):
    """Tile-class probabilities (F22, F42, F6) of the paper's families (Sec. II): gallus_26
    mixes F22 and F6, gallus_46 mixes F42 and F6, p6 being the F6 share."""
    if family == "gallus_26":
        return (1.0 - p6, 0.0, p6)
    if family == "gallus_46":
        return (0.0, 1.0 - p6, p6)
    raise ValueError(family)


def gap_vs_p6(sg, p6s, families=("gallus_26", "gallus_46"), L: int = 30, l: int = 5, sweeps: int = 20,
              beta0: float = 0.5, beta1: float = 6.0, instances: int = 20, seed_base: int = 8 * 10 ** 6):
    """Mean gap per family and p6 at one L (the paper's Fig. 1 experiment)."""
    rows = []
    for fi, fam in enumerate(families):
        for pi, p6 in enumerate(p6s):
            insts = [sg.Instance.create(L, seed_base + 10 ** 5 * fi + 1000 * pi + k, gallus_class_prob(fam, p6), True)
                     for k in range(instances)]
            params = [dict(l=l, sweeps=sweeps, beta0=beta0, beta1=beta1, seed=1, instance_id=k)
                      for k in range(instances)]
            res = sg.fragment_run_batch(insts, params)
            eps = np.array([r["eps"] for r in res])
            rows.append(dict(family=fam, p6=p6, mean_eps=float(eps.mean()), std_eps=float(eps.std())))
            for i in insts:
                i.close()
    return rows


def main(argv=None):
    import argparse
    import json

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--L", type=int, nargs="+", default=[10, 20, 30, 40, 50])
    ap.add_argument("--l", type=int, default=5)
    ap.add_argument("--sweeps", type=int, nargs="+", default=[20])
    ap.add_argument("--beta0", type=float, default=0.5)
    ap.add_argument("--beta1", type=float, default=6.0)
    ap.add_argument("--instances", type=int, default=20)
    ap.add_argument("--gallus", action="store_true", help="gap vs p6 of gallus_26 / gallus_46 at L = 30")
    ap.add_argument("--tropical", action="store_true", help="exact zero-temperature cube marginals (l <= 3)")
    args = ap.parse_args(argv)
    from . import sg

    out = []
    if args.gallus:
        p6s = [round(0.1 * k, 1) for k in range(11)]
        for S in args.sweeps:
            rows = gap_vs_p6(sg, p6s, L=30, l=args.l, sweeps=S, beta0=args.beta0, beta1=args.beta1,
                             instances=args.instances)
            row = dict(l=args.l, sweeps=S, L=30, points=rows)
            print(json.dumps(row), flush=True)
            out.append(row)
        return out
    if args.tropical:
        rows, fit = gap_vs_L(sg, args.L, args.l, 0, 1.0, 1.0, args.instances, tropical=True)
        row = dict(l=args.l, tropical=True, points=rows, fit=fit)
        print(json.dumps(row), flush=True)
        return [row]
    for S in args.sweeps:
        rows, fit = gap_vs_L(sg, args.L, args.l, S, args.beta0, args.beta1, args.instances)
        row = dict(l=args.l, sweeps=S, beta0=args.beta0, beta1=args.beta1, points=rows, fit=fit)
        print(json.dumps(row), flush=True)
        out.append(row)
    return out


if __name__ == "__main__":
    main()
