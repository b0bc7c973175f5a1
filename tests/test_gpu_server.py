"""Serving path (sg_server_*): requests solved to a target gap under continuous batching.

Each result is checked against the one-shot entry points, which are themselves
checked against the oracle: a PT request stopped after n sweeps reports the minimum
energy sg_pt_run reports for n sweeps, an SA request whose chunk is a whole restart
reports the lowest replica energy of sg_sa_run with instance_id = restart, and every
result is identical alone and in a mix of SA (all plane widths) and PT requests."""
import numpy as np
import pytest

from oracle import oracle as o

pytestmark = pytest.mark.gpu

GiB = 1 << 30


@pytest.fixture(scope="module")
def sg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.init()
    from paper_2501_17267_gb300 import build
    build.build()
    from paper_2501_17267_gb300 import sg as mod
    return mod


def _target(e_gs, eps):
    return e_gs + int(np.floor(eps * abs(e_gs)))


def _expected_pt(sg, req, chunk):
    inst = sg.Instance.create(req.instance.L, req.instance.seed, tuple(req.instance.class_prob),
                              bool(req.instance.gauge))
    target = _target(inst.e_gs, req.eps_target)
    n = 0
    while True:
        n += chunk
        r = sg.pt_run(inst, req.width, n, req.beta0, req.beta1, seed=req.seed)
        if r["minE"] <= target:
            return dict(minE=r["minE"], sweeps=n, reached=1, e_gs=inst.e_gs)
        if n >= req.sweep_cap:
            return dict(minE=r["minE"], sweeps=n, reached=0, e_gs=inst.e_gs)


def _expected_sa_whole_restarts(sg, req):
    inst = sg.Instance.create(req.instance.L, req.instance.seed, tuple(req.instance.class_prob),
                              bool(req.instance.gauge))
    target = _target(inst.e_gs, req.eps_target)
    S, best, k, sweeps = req.sweeps_per_restart, None, 0, 0
    while True:
        n = min(S, req.sweep_cap - sweeps)
        assert n == S, "cap must be a whole number of restarts here"
        r = sg.sa_run(inst, req.width, S, req.beta0, req.beta1, schedule=req.schedule,
                      seed=req.seed, instance_id=k)
        m = int(r["E"].min())
        best = m if best is None else min(best, m)
        sweeps += S
        if best <= target:
            return dict(minE=best, sweeps=sweeps, reached=1, e_gs=inst.e_gs)
        if sweeps >= req.sweep_cap:
            return dict(minE=best, sweeps=sweeps, reached=0, e_gs=inst.e_gs)
        k += 1


def _solve(sg, reqs, chunk, max_active=64, budget=8 * GiB):
    with sg.Server(budget, max_active=max_active, chunk_sweeps=chunk) as srv:
        tickets = [srv.submit(r) for r in reqs]
        return [srv.poll(t, timeout_ms=-1) for t in tickets]


def _key(res):
    return (res["status"], res["reached"], res["sweeps"], res["minE"], res["e_gs"])


def test_pt_request_matches_pt_run(sg):
    chunk = 20
    for L, K, eps, cap in [(6, 8, 0.0, 200), (8, 12, 0.05, 160), (10, 16, 0.0, 60)]:
        req = sg.request(sg.SG_REQ_PT, L, seed=1000 + L, width=K, beta0=0.2, beta1=3.0,
                         eps_target=eps, sweep_cap=cap, run_seed=77 + L)
        (res,) = _solve(sg, [req], chunk)
        exp = _expected_pt(sg, req, chunk)
        assert res["status"] == sg.SG_OK
        assert (res["minE"], res["sweeps"], res["reached"], res["e_gs"]) == \
            (exp["minE"], exp["sweeps"], exp["reached"], exp["e_gs"])
        assert res["min_eps"] == pytest.approx((exp["minE"] - exp["e_gs"]) / abs(exp["e_gs"]))


def test_pt_request_on_clusters_matches_row_kernels(sg, monkeypatch):
    """Small PT requests run as one cluster-kernel launch per chunk (sweep index in device
    memory, replayed as a graph); the same requests run through the row kernels give the
    same minimum energies and sweep counts (32 temperatures; L = 8 and 16)."""
    chunk = 25
    reqs = [sg.request(sg.SG_REQ_PT, L, seed=2024 + L, width=32, beta0=0.2, beta1=3.0, eps_target=0.0,
                       sweep_cap=100, run_seed=3 + L) for L in (8, 16)]
    got = _solve(sg, reqs, chunk)
    monkeypatch.setenv("SG_PT_CLUSTER", "0")
    for req, res in zip(reqs, got):
        exp = _expected_pt(sg, req, chunk)
        assert res["status"] == sg.SG_OK
        assert (res["minE"], res["sweeps"], res["reached"]) == (exp["minE"], exp["sweeps"], exp["reached"])


@pytest.mark.parametrize("R", [4, 8, 12, 32])  # plane widths 1, 2, 1 (three planes), 4 words
def test_sa_request_matches_sa_run_restarts(sg, R):
    S = 30
    # L <= 16 run in the shared plane launch, larger lattices as multi-block sweeps
    for L, eps, cap in [(4, 0.0, 3 * S), (8, 0.0, 4 * S), (12, 0.02, 2 * S), (20, 0.0, 2 * S),
                        (24, 0.01, 3 * S)]:
        req = sg.request(sg.SG_REQ_SA, L, seed=500 + L, width=R, beta0=0.1, beta1=3.0,
                         eps_target=eps, sweep_cap=cap, run_seed=9 + R, sweeps_per_restart=S,
                         schedule=sg.SG_SCHEDULE_GEOMETRIC)
        (res,) = _solve(sg, [req], chunk=S)
        exp = _expected_sa_whole_restarts(sg, req)
        assert res["status"] == sg.SG_OK
        assert (res["minE"], res["sweeps"], res["reached"], res["e_gs"]) == \
            (exp["minE"], exp["sweeps"], exp["reached"], exp["e_gs"])


def test_sa_request_restart0_matches_oracle(sg):
    L, R, S = 4, 8, 12
    req = sg.request(sg.SG_REQ_SA, L, seed=4242, width=R, beta0=0.2, beta1=2.5, eps_target=0.0,
                     sweep_cap=S, run_seed=(3 << 32) + 5, sweeps_per_restart=S)
    (res,) = _solve(sg, [req], chunk=S)
    J3, _, egs = o.generate(L, 4242, (1 / 3, 1 / 3, 1 / 3), True)
    _, E = o.sa_run(L, J3, (3 << 32) + 5, 0, S, 0.2, 2.5, False, R=R)
    assert res["minE"] == int(np.min(E)) and res["e_gs"] == egs


def _mix(sg):
    reqs = []
    for k in range(16):
        L = (4, 6, 8, 10, 12, 16, 20, 24)[k % 8]
        if k % 3 == 2:
            reqs.append(sg.request(sg.SG_REQ_PT, L, seed=9000 + k, width=(8, 12)[k % 2],
                                   beta0=0.2, beta1=3.0, eps_target=0.0, sweep_cap=90, run_seed=k))
        else:
            reqs.append(sg.request(sg.SG_REQ_SA, L, seed=9000 + k, width=(4, 8, 16, 32)[k % 4],
                                   beta0=0.1, beta1=3.0, eps_target=(0.0, 0.03)[k % 2],
                                   sweep_cap=100, run_seed=k, sweeps_per_restart=40))
    return reqs


def test_results_identical_alone_and_mixed(sg):
    chunk = 15  # does not divide the restart length: rounds end inside restarts too
    reqs = _mix(sg)
    mixed = _solve(sg, reqs, chunk)
    alone = [_solve(sg, [r], chunk)[0] for r in reqs]
    serial = _solve(sg, reqs, chunk, max_active=1)
    for m, a, s in zip(mixed, alone, serial):
        assert m["status"] == sg.SG_OK
        assert _key(m) == _key(a) == _key(s)


def test_budget_limits_admission(sg):
    """A budget that fits one request at a time still serves all of them, one after the
    other: each is admitted only after the previous one has finished."""
    import time
    reqs = [sg.request(sg.SG_REQ_PT, 16, seed=70 + k, width=16, beta0=0.2, beta1=3.0,
                       eps_target=0.0, sweep_cap=200, run_seed=k) for k in range(4)]
    one = max(sg.request_bytes(r) for r in reqs)
    with sg.Server(one + one // 2, max_active=8, chunk_sweeps=20) as srv:
        tickets, t_sub = [], []
        for r in reqs:
            t_sub.append(time.perf_counter())
            tickets.append(srv.submit(r))
        res = [srv.poll(t, timeout_ms=-1) for t in tickets]
    ref = _solve(sg, reqs, 20)
    for a, b in zip(res, ref):
        assert _key(a) == _key(b)
    for k in range(1, len(res)):
        # admitted (t_sub[k] + queue_s) no earlier than the previous one finished
        assert t_sub[k] + res[k]["queue_s"] >= t_sub[k - 1] + res[k - 1]["total_s"] - 2e-3


def test_cancel_queued_and_running(sg):
    long_req = sg.request(sg.SG_REQ_PT, 16, seed=1, width=16, beta0=0.2, beta1=3.0, eps_target=0.0,
                          sweep_cap=10 ** 9, run_seed=1)
    with sg.Server(8 * GiB, max_active=1, chunk_sweeps=10) as srv:
        t1 = srv.submit(long_req)
        t2 = srv.submit(long_req)
        srv.cancel(t2)  # waiting behind t1 (max_active = 1)
        r2 = srv.poll(t2, timeout_ms=-1)
        assert r2["status"] == sg.SG_ECANCELED and r2["sweeps"] == 0
        assert srv.poll(t1, timeout_ms=0) is None
        srv.cancel(t1)
        r1 = srv.poll(t1, timeout_ms=-1)
        assert r1["status"] == sg.SG_ECANCELED
        with pytest.raises(sg.SGError) as e:
            srv.poll(t1, timeout_ms=0)  # reported once, then forgotten
        assert e.value.code == sg.SG_EINVAL


def test_destroy_with_work_in_flight(sg):
    long_req = sg.request(sg.SG_REQ_SA, 16, seed=3, width=64, beta0=0.1, beta1=3.0, eps_target=0.0,
                          sweep_cap=10 ** 9, run_seed=3, sweeps_per_restart=1000)
    srv = sg.Server(8 * GiB, max_active=2, chunk_sweeps=25)
    for _ in range(4):
        srv.submit(long_req)
    srv.close()  # running ones stop at the next round boundary, waiting ones are dropped


def test_admission_errors(sg):
    req = sg.request(sg.SG_REQ_SA, 8, seed=1, width=8, beta0=0.1, beta1=3.0, eps_target=0.0,
                     sweep_cap=10 ** 9, run_seed=1, sweeps_per_restart=1000)
    with sg.Server(1024, max_active=1, chunk_sweeps=10) as srv:
        with pytest.raises(sg.SGError) as e:
            srv.submit(req)  # alone larger than the budget
        assert e.value.code == sg.SG_ENOMEM
    with sg.Server(8 * GiB, max_active=1, chunk_sweeps=10, queue_capacity=1) as srv:
        codes, tickets = [], []
        for _ in range(3):
            try:
                tickets.append(srv.submit(req))
                codes.append(sg.SG_OK)
            except sg.SGError as err:
                codes.append(err.code)
        assert sg.SG_EBUSY in codes and codes[0] == sg.SG_OK
        for t in tickets:
            srv.cancel(t)
            assert srv.poll(t, timeout_ms=-1)["status"] == sg.SG_ECANCELED
    with sg.Server(8 * GiB) as srv:
        for bad in [dict(L=5), dict(width=0), dict(beta0=0.0), dict(eps_target=-0.1), dict(sweep_cap=0)]:
            args = dict(kind=sg.SG_REQ_SA, L=8, seed=1, width=8, beta0=0.1, beta1=3.0, eps_target=0.0,
                        sweep_cap=10)
            args.update(bad)
            with pytest.raises(sg.SGError) as e:
                srv.submit(sg.request(**args))
            assert e.value.code == sg.SG_EINVAL
        with pytest.raises(sg.SGError):
            srv.submit(sg.request(sg.SG_REQ_PT, 8, 1, width=300, beta0=0.2, beta1=3.0,
                                  eps_target=0.0, sweep_cap=10))
