"""Benchmark: Metropolis spin-flip attempts/s of parallel tempering on tile-planted
L=64 cubic-lattice spin glasses (16 instances x 32 temperatures, geometric beta
0.2 -> 3.0, exchange after every sweep, 10^4 sweeps), through the libsg C ABI.

One step = one full run of the hot path over the batch: initial spins, 10^4
checkerboard Metropolis sweeps of every slot, an exchange attempt after each
sweep, the energy recompute and the optimality gap eps of the minimum energy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is attempts/s with the instances already
resident on the device; `e2e` is the same metric with host couplings uploaded
and results read back inside the timed region; `roofline` covers the dominant sweep kernel;
`cpu_baseline` times the CPU oracle on a bounded sample on the host cores.
For N > 1 each rank runs its own 16 instances (weak scaling, no collective on the
data path); value = all ranks' attempts / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time
from concurrent.futures import ProcessPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2501_17267_gb300 import workloads as wl  # noqa: E402

WORK = wl.PT_L64
METRIC = "Metropolis spin-flip attempts/s"
UNIT = "attempts/s"
# what the bit-packed sweep kernel moves per attempt: a spin bit read and written once per
# sweep (2/8 B), 3 coupling bytes per site shared by R replicas
BYTES_PER_ATTEMPT = 2.0 / 8.0 + 3.0 / WORK.temps


def _peaks():
    """(HBM GB/s, its source, max SM MHz)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured", float(p.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


# Roofs of one attempt.  The sweeps are integer work whose fixed core is the draws: the
# eight leading-byte bit planes of a word of 32 replicas come from two Philox4x32-10
# blocks of 20 32x32->64-bit multiplies each (the low 24 bits are drawn for 1/256 of the
# draws only), so 16 attempts per block.  The binding roof is the rate at which this GPU
# produces Philox blocks when drawing is all it does -- measured by sg_philox_rate -- and
# `frac` is the kernel's multiply rate over that measured rate.  The nominal figure
# (SMs x 32 multiplies per clock) is kept beside it for context.  HBM: the spin bytes
# per attempt as the int8 layout would move them (1 B read + 1 B written + 3/R B of
# couplings) and as the bit-packed kernel moves them (1/8 + 1/8 + 3/R B); the 55 MB
# working set of the PT workload stays in L2 either way.
MULS_PER_BLOCK = 20
WIDE_MULS_PER_SM_CLOCK = 32
ATTEMPTS_PER_BLOCK = 16


def hbm_views(replicas):
    return {"int8_layout": 2.0 + 3.0 / replicas, "bit_packed": 2.0 / 8.0 + 3.0 / replicas}


def _roof(rate, attempts_per_block, views, blocks_per_s, sms, sm_mhz, hbm_peak, hbm_kind, **extra):
    """The roofline object of a sweep kernel running `rate` attempts/s: its multiply rate
    against the measured Philox block rate (blocks_per_s; the nominal peak stands in,
    marked "derived", when the measurement is missing), with the HBM views beside it."""
    muls = MULS_PER_BLOCK / attempts_per_block
    achieved = rate * muls / 1e12
    derived = sms * WIDE_MULS_PER_SM_CLOCK * sm_mhz * 1e6 / 1e12
    if blocks_per_s:
        peak = blocks_per_s * MULS_PER_BLOCK / 1e12
        src = "measured: Philox4x32-10 alone on this GPU (sg_philox_rate), after the timed region"
    else:
        peak = derived
        src = f"derived: {sms} SMs x {WIDE_MULS_PER_SM_CLOCK} multiplies per clock at {sm_mhz:.0f} MHz"
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T 32x32->64-bit multiplies/s",
         "frac": achieved / peak, "peak_source": src, "muls_per_attempt": muls, "attempts_per_s": rate,
         "peak_attempts_per_s": peak * 1e12 / muls,
         "nominal_peak": {"value": derived, "frac": achieved / derived,
                          "source": f"{sms} SMs x {WIDE_MULS_PER_SM_CLOCK} multiplies per clock at {sm_mhz:.0f} MHz"},
         "hbm_views": {name: {"bytes_per_attempt": b, "achieved_gbs": rate * b / 1e9, "peak_gbs": hbm_peak,
                              "frac": rate * b / 1e9 / hbm_peak, "peak_source": hbm_kind}
                       for name, b in views.items()}}
    r.update(extra)
    return r


def _philox_blocks_per_s(sg):
    """The device's Philox4x32-10 block rate when drawing is all it does, or None."""
    try:
        return sg.philox_rate()
    except Exception:  # noqa: BLE001 -- the roofline then falls back to the nominal peak
        return None


L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2


def _l2_flusher(torch):
    """A callable that overwrites a buffer larger than L2 on the current stream; the
    timed loops call it before every step (its time counts in the step)."""
    buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    state = {"k": 0}

    def flush():
        state["k"] = (state["k"] + 1) & 0xFF
        buf.fill_(state["k"])

    return flush


def _traffic_record(name):
    """DRAM bytes per launch of a sweep kernel from the committed ncu capture
    profiles/<name>.traffic.json, if the kernel's sources are unchanged since it was
    taken (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name + ".traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        return rec if h.hexdigest() == rec["sources_sha256"] else None
    except Exception:
        return None


# ---------------------------------------------------------------- CPU oracle leg

def _oracle_job(args):
    k, sweeps = args
    from oracle import oracle as o
    J3, _, _ = o.generate(WORK.L, WORK.instance_seed(k), WORK.class_prob, True)
    t = time.perf_counter()
    o.pt_run(WORK.L, J3, WORK.run_seed, k, WORK.temps, sweeps, WORK.beta_min, WORK.beta_max)
    return time.perf_counter() - t


def oracle_sample(sweeps: int, workers: int):
    """The oracle, as it stands, on all 16 instances for `sweeps` sweeps, one process
    per instance on `workers` host cores.  Wall time includes each run's initial
    state and energy evaluation."""
    t = time.perf_counter()
    # an executor, not a Pool: a worker that dies raises here instead of hanging the run
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_job, [(k, sweeps) for k in range(WORK.instances)]))
    wall = time.perf_counter() - t
    attempts = WORK.instances * WORK.temps * WORK.L ** 3 * sweeps
    return attempts / wall, wall


def cpu_baseline(sweeps: int):
    from oracle import oracle as o
    o.build()
    workers = min(WORK.instances, os.cpu_count() or 1)
    rate, wall = oracle_sample(sweeps, workers)
    return {"value": rate, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"all {WORK.instances} instances, first {sweeps} sweeps of the {WORK.sweeps} "
                      f"(L={WORK.L}, {WORK.temps} temperatures), one spawn process per instance; "
                      f"{wall:.1f} s wall incl. initial state + energy; rate extrapolated linearly in "
                      f"sweeps (cost per sweep is constant).  {sweeps} rather than 10^2 sweeps keeps the "
                      f"default run within minutes; the oracle's 101-sweep runs of all 16 instances are "
                      f"the parity test's",
            "cpu": _cpu_model()}


# CPU part numbers of the Arm cores GPU hosts carry, for hosts whose tools print only the part
_ARM_PARTS = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1", "0xd49": "Neoverse-N2"}


def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo; an Arm part number is named)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    part = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name"):
                    return line.split(":", 1)[1].strip()
                if low.startswith("cpu part") and part is None:
                    part = line.split(":", 1)[1].strip().lower()
    except Exception:
        pass
    if part:
        return _ARM_PARTS.get(part, f"Arm CPU part {part}")
    return "unknown"


def run_reference(args, rank):
    if rank != 0:
        return
    from oracle import oracle as o
    o.build()
    workers = min(WORK.instances, os.cpu_count() or 1)
    for _ in range(args.warmup):
        oracle_sample(args.ref_sweeps, workers)
    rates, walls = [], []
    for _ in range(args.steps):
        r, w = oracle_sample(args.ref_sweeps, workers)
        rates.append(r)
        walls.append(w)
    attempts = WORK.instances * WORK.temps * WORK.L ** 3 * args.ref_sweeps * args.steps
    value = attempts / sum(walls)
    # n_gpus is the launch's N, as for the other arm; the oracle itself uses host cores only
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "gpus_used": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(walls) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": _config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"each step: all {WORK.instances} instances, first "
                                       f"{args.ref_sweeps} sweeps, one spawn process per instance",
                             "cpu": _cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config():
    return {"workload": WORK.name, "L": WORK.L, "instances": WORK.instances, "temps": WORK.temps,
            "sweeps": WORK.sweeps, "beta": f"geometric {WORK.beta_min}->{WORK.beta_max}",
            "exchange": "every sweep", "tiles": "uniform F22/F42/F6, gauged",
            "cache": "L2 flushed (256 MB written) before every timed step; the step's 17 MB of spins and "
                     "38 MB of coupling records then stay in L2 across its sweeps"}


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling every 200 ms.  start() launches it and waits for its first
    sample, so that its start-up (NVML initialisation, which can stall the GPU on a
    freshly booted box) happens before the warm-up; mark() opens the timed window and
    stop() keeps the samples that arrived inside it (plus the one that closes it)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.t0 = None
        self.reader = None

    def start(self):
        import threading
        first = threading.Event()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def read():
            for line in self.proc.stdout:
                self.lines.append((time.time(), line))
                first.set()
            first.set()

        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        first.wait(timeout=30)

    def mark(self):
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t1 = time.time()
        time.sleep(0.25)  # the sample that closes the window
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.reader.join(timeout=10)
        t0 = self.t0 if self.t0 is not None else 0.0
        window = [line for t, line in self.lines if t0 <= t <= t1 + 0.25]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in window:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- serving leg

def _serving_request(sg, w, item, sa_cap, pt_cap):
    if item["kind"] == "SA":
        return sg.request(sg.SG_REQ_SA, item["L"], item["seed"], w.sa_replicas, w.sa_beta0, w.sa_beta1,
                          w.eps_target, sa_cap, run_seed=item["run_seed"],
                          sweeps_per_restart=w.sa_sweeps_per_restart, schedule=sg.SG_SCHEDULE_LINEAR,
                          class_prob=w.class_prob)
    return sg.request(sg.SG_REQ_PT, item["L"], item["seed"], w.pt_temps, w.pt_beta_min, w.pt_beta_max,
                      w.eps_target, pt_cap, run_seed=item["run_seed"], class_prob=w.class_prob)


def _pcts(xs):
    import numpy as np
    if not xs:
        return {"p50": None, "p95": None, "p99": None}
    a = np.asarray(xs, dtype=np.float64)
    return {"p50": float(np.percentile(a, 50)), "p95": float(np.percentile(a, 95)),
            "p99": float(np.percentile(a, 99))}


def _pcts_censored(reached, n_total):
    """Percentiles of the time to target over ALL n_total requests, the ones stopped at
    the sweep cap counted as never reaching it (+infinity): nearest rank on the sorted
    times; a percentile that falls among the censored requests is null, marked in
    `censored`."""
    import math
    xs = sorted(reached)
    out = {"censored_fraction": 1 - len(xs) / max(n_total, 1), "censored": []}
    for name, p in (("p50", 0.50), ("p95", 0.95), ("p99", 0.99)):
        k = max(1, math.ceil(p * n_total)) - 1  # 0-based nearest rank
        if n_total and k < len(xs):
            out[name] = float(xs[k])
        else:
            out[name] = None
            out["censored"].append(name)
    return out


def run_served(sg, w, stream, sa_cap, pt_cap, chunk, max_active, budget):
    """The stream through the continuously batched server: each request is submitted at
    its arrival time; latency = submit lateness + the server's submit-to-done time."""
    reqs = [_serving_request(sg, w, it, sa_cap, pt_cap) for it in stream]
    width = {"SA": w.sa_replicas, "PT": w.pt_temps}
    with sg.Server(budget, max_active=max_active, chunk_sweeps=chunk, queue_capacity=1 << 20) as srv:
        t0 = time.perf_counter()
        tickets, late = [], []
        for it, r in zip(stream, reqs):
            now = time.perf_counter() - t0
            if it["t"] > now:
                time.sleep(it["t"] - now)
            ts = time.perf_counter() - t0
            tickets.append(srv.submit(r))
            late.append(ts - it["t"])
        res = [srv.poll(t, -1) for t in tickets]
    lat = [lt + r["total_s"] for lt, r in zip(late, res)]
    ends = [it["t"] + x for it, x in zip(stream, lat)]
    makespan = max(ends) if ends else 0.0
    reached = [x for x, r in zip(lat, res) if r["status"] == 0 and r["reached"]]
    attempts = sum(r["sweeps"] * it["L"] ** 3 * width[it["kind"]] for it, r in zip(stream, res))
    by_kind = {}
    for kind in ("SA", "PT"):
        ks = [(x, r) for x, r, it in zip(lat, res, stream) if it["kind"] == kind]
        by_kind[kind] = {"requests": len(ks),
                         "tte_s": _pcts_censored([x for x, r in ks if r["status"] == 0 and r["reached"]], len(ks)),
                         "censored": sum(1 for x, r in ks if not r["reached"]) / max(len(ks), 1)}
    return {"requests": len(stream), "errors": sum(1 for r in res if r["status"] != 0),
            "tte_s": _pcts_censored(reached, len(stream)),
            "tte_reached_only_s": _pcts(reached),
            "stop_s": _pcts(lat),
            "censored_fraction": 1 - len(reached) / max(len(stream), 1),
            "throughput_req_s": len(stream) / makespan if makespan else None,
            "attempts_per_s": attempts / makespan if makespan else None,
            "makespan_s": makespan, "max_submit_late_s": max(late) if late else 0.0,
            "queue_s": _pcts([r["queue_s"] for r in res]), "service_s": _pcts([r["run_s"] for r in res]),
            "by_kind": by_kind,
            "definitions": "tte_s: time from arrival to eps <= target over all requests, the ones stopped "
                           "at the sweep cap counted as not reached (a percentile among them is null); "
                           "tte_reached_only_s: the same over the requests that reached it; stop_s: arrival "
                           "to done, reached or capped; queue_s: submit to admitted; service_s: admitted "
                           "to done, in the mix"}


def run_one_at_a_time(sg, w, stream, sa_cap, pt_cap, limit_s):
    """The same stream served the plain way: one request at a time in arrival order, each
    through the one-shot calls with one instance per launch -- SA as successive sg_sa_run
    restarts (instance_id = restart) checked after each, PT as one sg_pt_run of the cap.
    Requests not finished within limit_s count as unfinished, their latency bounded below
    by limit_s - arrival.  service_s is each request's own processing time on the
    otherwise idle GPU; wait_s is how long it waited for the requests before it."""
    import numpy as np
    t0 = time.perf_counter()
    lat, reached, unfinished, service, wait = [], [], 0, [], []
    for it in stream:
        now = time.perf_counter() - t0
        if now > limit_s:
            unfinished += 1
            lat.append(limit_s - it["t"])
            continue
        if it["t"] > now:
            time.sleep(it["t"] - now)
        start = time.perf_counter() - t0
        inst = sg.Instance.create(it["L"], it["seed"], w.class_prob, True)
        target = inst.e_gs + int(np.floor(w.eps_target * abs(inst.e_gs)))
        ok = False
        if it["kind"] == "SA":
            S, done, k = w.sa_sweeps_per_restart, 0, 0
            while done < sa_cap and not ok:
                n = min(S, sa_cap - done)
                r = sg.sa_run(inst, w.sa_replicas, n, w.sa_beta0, w.sa_beta1, "linear",
                              seed=it["run_seed"], instance_id=k)
                ok = int(r["E"].min()) <= target
                done += n
                k += 1
        else:
            r = sg.pt_run(inst, w.pt_temps, pt_cap, w.pt_beta_min, w.pt_beta_max, seed=it["run_seed"])
            ok = r["minE"] <= target
        inst.close()
        end = time.perf_counter() - t0
        x = end - it["t"]
        lat.append(x)
        service.append(end - start)
        wait.append(start - it["t"])
        if ok:
            reached.append(x)
    return {"requests": len(stream), "unfinished_at_limit": unfinished, "limit_s": limit_s,
            "tte_s": _pcts_censored(reached, len(stream)), "tte_reached_only_s": _pcts(reached),
            "stop_s": _pcts(lat), "service_s": _pcts(service), "wait_s": _pcts(wait),
            "censored_fraction": 1 - len(reached) / max(len(stream), 1)}


def serving_leg(sg, args, w):
    stream = w.stream(args.serve_seconds)
    sa_cap = args.sa_cap or w.sa_sweep_cap
    pt_cap = args.pt_cap or w.pt_sweep_cap
    budget = int(args.serve_budget_gb * (1 << 30))
    served = run_served(sg, w, stream, sa_cap, pt_cap, args.serve_chunk, args.serve_max_active, budget)
    out = {"workload": w.name, "rate_per_s": w.rate_per_s, "window_s": args.serve_seconds,
           "eps_target": w.eps_target, "sa_sweep_cap": sa_cap, "pt_sweep_cap": pt_cap,
           "chunk_sweeps": args.serve_chunk, "max_active": args.serve_max_active,
           "hbm_budget_bytes": budget, "served": served}
    if args.serve_baseline_seconds > 0:
        base = [it for it in stream if it["t"] < args.serve_baseline_seconds]
        out["one_at_a_time"] = run_one_at_a_time(sg, w, base, sa_cap, pt_cap, args.serve_baseline_limit)
        out["one_at_a_time"]["window_s"] = args.serve_baseline_seconds
        if args.serve_baseline_seconds < args.serve_seconds:
            sub = run_served(sg, w, base, sa_cap, pt_cap, args.serve_chunk, args.serve_max_active, budget)
            out["served_same_window"] = sub
    return out


# ---------------------------------------------------------------- batched leg

def batched_line(sg, args, torch, clocks_cls, local):
    """Batched uneven SA: 512 instances, L uniform over {8,12,16,24,32,48}, 64 replicas,
    sweeps uniform over {100, 1000, 10000}, all in one sg_sa_run_batch (one persistent
    graph-captured launch, plane width from the autotuner)."""
    w = wl.BATCHED
    shapes = w.draw()
    insts = [sg.Instance.create(L, w.instance_seed(k), w.class_prob, True) for k, (L, S) in enumerate(shapes)]
    params = [dict(replicas=w.replicas, sweeps=S, beta0=w.beta0, beta1=w.beta1, schedule="linear", seed=0,
                   instance_id=k) for k, (L, S) in enumerate(shapes)]
    attempts = sum(L ** 3 * w.replicas * S for L, S in shapes)
    stream = torch.cuda.current_stream()
    clocks = clocks_cls(local)
    clocks.start()
    flush = _l2_flusher(torch)
    for _ in range(args.warmup):
        flush()
        out = sg.sa_run_batch(insts, params)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark()
    ev0.record(stream)
    for _ in range(args.steps):
        flush()
        out = sg.sa_run_batch(insts, params)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    # one more step with launch timing on: the persistent sweep launch alone
    sg.stats_read(reset=True)
    sg.stats_enable(True)
    sg.sa_run_batch(insts, params)
    torch.cuda.synchronize()
    sg.stats_enable(False)
    st = sg.stats_read(reset=True)
    sw = st["sweep_chunk"] if st["sweep_chunk"]["launches"] else st["sweep"]
    peak, peak_kind, sm_mhz = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = None
    if sw["device_ms"] > 0:
        roof = _roof(sw["units"] / (sw["device_ms"] / 1000.0), ATTEMPTS_PER_BLOCK, hbm_views(w.replicas),
                     _philox_blocks_per_s(sg), sms, sm_mhz, peak, peak_kind, traffic=None,
                     kernel="persistent batch kernel (one plane per block, or per thread-block cluster: autotuned)",
                     launch_ms=sw["device_ms"] / max(sw["launches"], 1))
    value = attempts * args.steps / (ms / 1000.0)
    eps = [float(e) for o in out for e in o["eps"][:4]]
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w.name, "instances": w.instances, "L": list(w.L_choices),
                       "replicas": w.replicas, "sweeps": list(w.sweep_choices),
                       "attempts_per_step": attempts, "beta": f"linear {w.beta0}->{w.beta1}",
                       "cache": "L2 flushed (256 MB written) before every timed step"},
            "roofline": roof, "gpu_launches": sum(v["launches"] for v in st.values()),
            "clocks": clk, "eps_mean_sample": sum(eps) / len(eps)}


# ---------------------------------------------------------------- SA throughput leg

def sa_line(sg, args, torch, clocks_cls, local, w=wl.SA_L16):
    """SA throughput: one instance, R replicas, 1000 sweeps, beta linear 0.1 -> 3.0 (by
    default L = 16 with 1024 replicas; wl.SA_L4 is L = 4 with 8); a step is one sg_sa_run:
    each word of 32 replicas annealed by one thread-block cluster for all 1000 sweeps in
    a single launch."""
    inst = sg.Instance.create(w.L, w.instance_seed(0), w.class_prob, True)
    attempts = w.L ** 3 * w.replicas * w.sweeps
    stream = torch.cuda.current_stream()
    steps = max(args.steps, 20)
    clocks = clocks_cls(local)
    clocks.start()
    flush = _l2_flusher(torch)
    for _ in range(max(args.warmup, 3)):
        flush()
        out = sg.sa_run(inst, w.replicas, w.sweeps, w.beta0, w.beta1, "linear", w.run_seed, 0)
    sg.stats_read(reset=True)
    sg.stats_enable(True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark()
    ev0.record(stream)
    for _ in range(steps):
        flush()
        out = sg.sa_run(inst, w.replicas, w.sweeps, w.beta0, w.beta1, "linear", w.run_seed, 0)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sg.stats_enable(False)
    st = sg.stats_read(reset=True)
    ms = ev0.elapsed_time(ev1)
    cluster = st["sweep_chunk"]["launches"] > 0
    sw = st["sweep_chunk"] if cluster else st["sweep"]
    peak, peak_kind, sm_mhz = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = None
    if sw["launches"] and sw["device_ms"] > 0:
        roof = _roof(sw["units"] / (sw["device_ms"] / 1000.0), ATTEMPTS_PER_BLOCK, hbm_views(w.replicas),
                     _philox_blocks_per_s(sg), sms, sm_mhz, peak, peak_kind, traffic=None,
                     kernel="sa_cluster_kernel" if cluster else "sweep_bits_kernel<SA>",
                     launch_ms=sw["device_ms"] / sw["launches"], share_of_step=sw["device_ms"] / ms,
                     note=f"working set {w.L ** 3 * 4 * ((w.replicas + 31) // 32) / 1e6:.3g} MB of spin words: "
                          "L2-resident, so HBM is not what limits it")
    eps = out["eps"]
    return {"metric": METRIC, "value": attempts * steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": w.name, "L": w.L, "replicas": w.replicas, "sweeps": w.sweeps,
                       "beta": f"linear {w.beta0}->{w.beta1}",
                       "cache": "L2 flushed (256 MB written) before every timed step; the spins then stay in L2 "
                                "across the step's sweeps"},
            "roofline": roof, "gpu_launches": sum(v["launches"] for v in st.values()), "clocks": clk,
            "eps": {"min": float(min(eps)), "median": float(sorted(eps)[len(eps) // 2]),
                    "max": float(max(eps))}}


# ---------------------------------------------------------------- fragment meta-heuristic leg

FRAG = dict(L=50, l=5, sweeps=20, beta0=0.5, beta1=6.0, instances=20)
# a fragment site's draws: one Philox4x32-10 block serves 4 reads, at most
FRAG_ATTEMPTS_PER_BLOCK = 4


def fragment_line(sg, args, torch, clocks_cls, local):
    """The fragment meta-heuristic (Sec. II) with SA fragment anneals: 20 F6 instances at
    L = 50, cubes of side 5, 20 sweeps of 32 reads per fragment; a step is one
    sg_fragment_run_batch (125 wave launches).  The oracle is timed beside it on one
    L = 10 instance (same per-attempt work)."""
    f = FRAG
    insts = [sg.Instance.create(f["L"], 9 * 10 ** 6 + 1000 * f["L"] + k, (0, 0, 1), True)
             for k in range(f["instances"])]
    params = [dict(l=f["l"], sweeps=f["sweeps"], beta0=f["beta0"], beta1=f["beta1"], seed=1, instance_id=k)
              for k in range(f["instances"])]
    V = f["l"] ** 3
    attempts = f["instances"] * f["L"] ** 3 * 32 * f["sweeps"] * (V + 1) / 2
    stream = torch.cuda.current_stream()
    steps = max(args.steps, 3)
    clocks = clocks_cls(local)
    clocks.start()
    flush = _l2_flusher(torch)
    for _ in range(max(args.warmup, 3)):
        flush()
        out = sg.fragment_run_batch(insts, params)
    sg.stats_read(reset=True)
    sg.stats_enable(True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark()
    ev0.record(stream)
    for _ in range(steps):
        flush()
        out = sg.fragment_run_batch(insts, params)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sg.stats_enable(False)
    st = sg.stats_read(reset=True)
    ms = ev0.elapsed_time(ev1)
    sw = st["sweep"]
    peak, peak_kind, sm_mhz = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = None
    if sw["launches"] and sw["device_ms"] > 0:
        rate = sw["units"] / (sw["device_ms"] / 1000.0)
        # a fragment site's draws: one Philox block serves four reads, at most
        roof = _roof(rate, FRAG_ATTEMPTS_PER_BLOCK, {}, _philox_blocks_per_s(sg), sms, sm_mhz, peak, peak_kind,
                     kernel="fragment_wave_kernel", traffic=None, launch_ms=sw["device_ms"] / sw["launches"],
                     share_of_step=sw["device_ms"] / ms,
                     note="bond terms of the 32 reads counted bit-sliced, weighted by |J| (fragments may hold "
                          "|J| = 2 or 0 bonds and cube boundaries); reads with x < 0 take their draw one by one; "
                          "muls_per_attempt is the most the draws can cost")
    cpu = None
    if not args.no_cpu:
        from oracle import oracle as o
        J3, _, _ = o.generate(10, 7, (0, 0, 1), True)
        t0 = time.perf_counter()
        o.fragment_run(10, J3, f["l"], f["sweeps"], f["beta0"], f["beta1"], 1, 0)
        dt = time.perf_counter() - t0
        cpu = {"value": 10 ** 3 * 32 * f["sweeps"] * (V + 1) / 2 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one F6 instance at L = 10, same l, sweeps and schedule ({dt:.1f} s, one core)"}
    eps = [r["eps"] for r in out]
    return {"metric": METRIC, "value": attempts * steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "fragment_F6_L50_l5_S20", **f,
                       "cache": "L2 flushed (256 MB written) before every timed step"},
            "roofline": roof, "cpu_baseline": cpu, "gpu_launches": sum(v["launches"] for v in st.values()),
            "clocks": clk, "mean_eps": float(sum(eps) / len(eps))}


# ---------------------------------------------------------------- GPU leg

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps", type=int, default=WORK.sweeps,
                    help="sweeps per run (default: the workload's 10^4)")
    ap.add_argument("--instances", type=int, default=WORK.instances,
                    help="instances per rank (default: the workload's 16; fewer only for profiling)")
    ap.add_argument("--cpu-sweeps", type=int, default=10)
    ap.add_argument("--ref-sweeps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="pt", choices=["pt", "serving", "batched", "sa", "fragment"],
                    help="pt: the PT throughput line (with a short serving leg); serving: the "
                         "serving stream alone; batched: 512 uneven SA instances in one launch; "
                         "sa: SA throughput at L=16 with 1024 replicas")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg of the pt line")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the SA L=16 and batched sub-lines of the pt line")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="arrival window (default: the workload's 60 s)")
    ap.add_argument("--serve-baseline-seconds", type=float, default=None,
                    help="window of the one-request-at-a-time comparison (default 5 s / 10 s)")
    ap.add_argument("--serve-baseline-limit", type=float, default=30.0,
                    help="wall-clock limit of the comparison arm")
    ap.add_argument("--serve-chunk", type=int, default=100)
    ap.add_argument("--serve-max-active", type=int, default=512)
    ap.add_argument("--serve-budget-gb", type=float, default=160.0)
    ap.add_argument("--sa-cap", type=int, default=0)
    ap.add_argument("--pt-cap", type=int, default=0)
    args = ap.parse_args()
    alone = args.workload == "serving"
    if args.serve_seconds is None:
        args.serve_seconds = wl.SERVING.duration_s
    if args.serve_baseline_seconds is None:
        args.serve_baseline_seconds = 10.0 if alone else 5.0

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    # CPU oracle leg first: its spawn pool starts before this process touches the GPU
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_sweeps)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    torch.cuda.init()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_17267_gb300 import build as libbuild
    if rank == 0:
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    libbuild.build()
    from paper_2501_17267_gb300 import sg

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    if args.workload in ("batched", "sa", "fragment"):
        if rank == 0:
            fn = {"batched": batched_line, "sa": sa_line, "fragment": fragment_line}[args.workload]
            print(json.dumps(fn(sg, args, torch, ClockSampler, local)), flush=True)
        barrier()
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if alone:
        if rank == 0:
            res = serving_leg(sg, args, wl.SERVING)
            sv = res["served"]
            # p50 over all requests with the capped ones counted as not reached: null (and
            # named in tte_s.censored) when more than half of the stream was capped
            line = {"metric": "served TTe at eps <= 1% (p50 over all requests, capped = not reached)",
                    "value": sv["tte_s"]["p50"], "unit": "s",
                    "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
                    "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                    "config": {"workload": wl.SERVING.name, "rate_per_s": wl.SERVING.rate_per_s,
                               "window_s": args.serve_seconds},
                    "serving": res}
            print(json.dumps(line), flush=True)
        barrier()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    S = args.sweeps
    from paper_2501_17267_gb300 import ranks
    mine = ranks.rank_units(rank, args.instances)  # this rank's instances (weak scaling)
    insts = [sg.Instance.create(WORK.L, WORK.instance_seed(g), WORK.class_prob, True) for g in mine]
    params = [dict(temps=WORK.temps, sweeps=S, beta_min=WORK.beta_min, beta_max=WORK.beta_max,
                   seed=WORK.run_seed, instance_id=g) for g in mine]
    stream = torch.cuda.current_stream()

    def step():
        return sg.pt_run_batch(insts, params)

    clocks = ClockSampler(local)
    clocks.start()
    flush = _l2_flusher(torch)
    for _ in range(args.warmup):
        flush()
        out = step()
    sg.stats_read(reset=True)
    sg.stats_enable(True)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark()
    ev0.record(stream)
    for _ in range(args.steps):
        flush()
        out = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    sg.stats_enable(False)
    st = sg.stats_read(reset=True)
    ms = ev0.elapsed_time(ev1)
    ms_max = ranks.max_over_ranks(ms, device="cuda")
    attempts_per_step = len(mine) * WORK.temps * WORK.L ** 3 * S
    value = ranks.job_rate(attempts_per_step, world, args.steps, ms_max)
    launches = sum(v["launches"] for v in st.values())

    # roofline of the dominant sweep kernel -- the kind that made most of the attempts: the
    # row kernels (two launches per sweep) or the cluster form (one launch per chunk of up to
    # 2000 sweeps; with 16 instances at L = 64, 15 run on clusters while the row kernels run
    # the 16th beside them) -- from its launches' CUDA-event durations in the timed region:
    # attempts per launch / mean launch duration against the integer roof, with the HBM
    # view (algorithmic bytes per launch / duration) beside it
    chunk_kernel = "pt_coop_kernel" if os.environ.get("SG_PT_COOP") == "1" else "pt_cluster_kernel"
    parts = {}
    for kind, kname in (("sweep", "sweep_bits_kernel<PT>"), ("sweep_chunk", chunk_kernel)):
        p = st[kind]
        if p["launches"] and p["device_ms"] > 0:
            parts[kname] = {"launches": p["launches"], "attempts": p["units"], "device_ms": p["device_ms"],
                            "attempts_per_s": p["units"] / (p["device_ms"] / 1000.0),
                            "share_of_attempts": p["units"] / (attempts_per_step * args.steps)}
    rows = st["sweep"]["units"] >= st["sweep_chunk"]["units"]
    sw = st["sweep"] if rows else st["sweep_chunk"]
    peak, peak_kind, sm_mhz = _peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = None
    if sw["launches"] and sw["device_ms"] > 0:
        per_launch_s = sw["device_ms"] / 1000.0 / sw["launches"]
        attempts_per_launch = sw["units"] / sw["launches"]
        rec = _traffic_record("sweep_bits_pt_L64_I16_K32" if rows else "pt_cluster_L64_I15_K32")
        roof = _roof(attempts_per_launch / per_launch_s, ATTEMPTS_PER_BLOCK, hbm_views(WORK.temps),
                     _philox_blocks_per_s(sg), sms, sm_mhz, peak, peak_kind,
                     traffic=rec["traffic_bytes_per_launch"] if rec else None,
                     traffic_unit="DRAM bytes per launch (ncu)",
                     algorithmic_bytes_per_launch=attempts_per_launch * BYTES_PER_ATTEMPT,
                     kernel="sweep_bits_kernel<PT>" if rows else chunk_kernel,
                     launch_ms=1000 * per_launch_s,
                     attempts_per_launch=attempts_per_launch, share_of_step=sw["device_ms"] / ms,
                     parts=parts)

    # end to end: host couplings in, results out, inside the timed region
    e2e = None
    if not args.no_e2e:
        host = [i.get() for i in insts]

        def e2e_step():
            hi = [sg.Instance.from_couplings(WORK.L, J3, egs) for (J3, _, egs) in host]
            r = sg.pt_run_batch(hi, params)
            for x in hi:
                x.close()
            return r

        e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e_s = time.perf_counter() - t0
        e_max = ranks.max_over_ranks(e_s, device="cuda")
        K = WORK.temps
        e2e = {"value": ranks.job_rate(attempts_per_step, world, args.steps, 1000.0 * e_max), "unit": UNIT,
               "h2d_bytes_per_step": len(mine) * 3 * WORK.L ** 3,
               "d2h_bytes_per_step": len(mine) * (8 * K + 4 * K + 8 * (K - 1) + 8 + 8)}

    serving = None
    if rank == 0 and not args.no_serve:
        serving = serving_leg(sg, args, wl.SERVING)
    # the other throughput workloads, each timed the same way (own warm-up, L2 flush,
    # clocks, launch statistics): SA at L = 16 with 1024 replicas, and the 512 uneven
    # SA instances in one persistent launch
    sub_lines = None
    if rank == 0 and not args.no_sub:
        sub_lines = {"sa_L4": sa_line(sg, args, torch, ClockSampler, local, wl.SA_L4),
                     "sa_L16": sa_line(sg, args, torch, ClockSampler, local),
                     "batched": batched_line(sg, args, torch, ClockSampler, local)}
    barrier()

    if rank == 0:
        mins = [o["min_eps"] for o in out]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic", "config": _config(),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "min_eps_mean": float(np.mean(mins)),
                "kernel_stats": st, "serving": serving, "sub_lines": sub_lines}
        if S != WORK.sweeps or args.instances != WORK.instances:
            line["config"]["sweeps"] = S
            line["config"]["instances"] = args.instances
            line["note"] = (f"reduced work ({args.instances} instances, {S} sweeps) -- not the workload's "
                            f"{WORK.instances} x {WORK.sweeps}")
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
