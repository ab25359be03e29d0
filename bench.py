"""Benchmark of the batched reactor path on GB300.

One step = one pass of the whole hot path over the batch of the medium
workload (53 species / 325 reactions, 131072 constant-pressure reactors):
one right-hand-side evaluation of every reactor, ROS4 integration of every
reactor over dt = 1e-5 s and RKF45 integration of every reactor over the same
dt (rtol 1e-9, atol 1e-12).  ``value`` is reactor integrations per second
(2 per reactor per step) with inputs resident in HBM; the RHS throughput
benchmark (1000 repeats of the RHS over the batch) is reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): each rank integrates its own batch (weak scaling, no
collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reactor integrations/sec and RHS evals/sec @1 GB300 vs roofline; serving p50/p99 ms"
UNIT = "reactor-integrations/s"
WORKLOAD = "medium"
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (2 flops per DFMA) at the maximum SM clock
L2_BYTES = 129 * 2 ** 20


def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def rank_states(workload: str, n: int, rank: int):
    """Weak scaling: every rank integrates its own seeded batch of n reactors
    (reactors are independent, so no data moves between ranks)."""
    from synth.configs import reactor_states
    return reactor_states(workload, n=n, seed_offset=1000 * rank)


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The job's time is the slowest rank's (the only collective of a run)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return units_per_rank * world / seconds


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches the
    current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        info = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = info.get(kernel)
    if not ent:
        return None
    from paper_1608_05794_gb300.build import sources_digest
    if ent.get("sources_digest") != sources_digest():
        return None
    return ent.get("bytes_per_launch")


def cpu_baseline(sample: int, threads: int = 0):
    """The oracle (as it stands) on the host cores over a bounded sample of
    the same workload: ROS4 + RKF45 of `sample` reactors and one RHS each."""
    from oracle import ORA_RKF45, ORA_ROS4, Oracle, OracleMech
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    cfg = CONFIGS[WORKLOAD]
    om = OracleMech(load_mechanism(cfg["mech"]))
    y, p = reactor_states(WORKLOAD, n=sample)
    cores = threads if threads > 0 else Oracle().hardware_threads()
    t0 = time.perf_counter()
    om.rhs(p, y)
    om.integrate(ORA_ROS4, p, y, cfg["dt"], nthreads=cores)
    om.integrate(ORA_RKF45, p, y, cfg["dt"], nthreads=cores)
    el = time.perf_counter() - t0
    return {"value": 2 * sample / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {sample} of the {cfg['n_reactors']} medium-workload reactors: one RHS, "
                      f"ROS4 and RKF45 over dt={cfg['dt']:g} s each, C++ oracle threaded over reactors",
            "seconds": el}


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    sample = args.cpu_sample
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(sample)
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
    v = float(np.mean(vals))
    from synth.configs import CONFIGS
    cfg = CONFIGS[WORKLOAD]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_dict(cfg),
            "cpu_baseline": {"kind": "oracle", "cores": r["cores"], "sample": r["sample"], "value": v,
                             "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config_dict(cfg):
    return {"workload": f"{WORKLOAD}: {cfg['n_species']} species / {cfg['n_reactions']} reactions "
                        f"({cfg['n_thirdbody']} third-body, {cfg['n_falloff']} Lindemann), "
                        f"{cfg['n_reactors']} constant-pressure reactors, RHS + ROS4 + RKF45 over "
                        f"dt={cfg['dt']:g} s, rtol 1e-9, atol 1e-12",
            "reactors": cfg["n_reactors"], "species": cfg["n_species"], "reactions": cfg["n_reactions"],
            "dt": cfg["dt"], "rtol": 1e-9, "atol": 1e-12,
            "l2": "inputs (57 MB) fit in L2: a 256 MiB buffer is written between steps"}


def run_ours(args):
    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism, reactor_states

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    cfg = CONFIGS[WORKLOAD]
    m = load_mechanism(cfg["mech"])
    gm = ck.load_mechanism(m)
    work = ck.count_work(gm)
    N = cfg["n_reactors"]
    y_np, p_np = rank_states(WORKLOAD, N, rank)
    dev = torch.device("cuda", torch.cuda.current_device())
    y0 = torch.as_tensor(y_np, device=dev)
    p = torch.as_tensor(p_np, device=dev)
    dt = torch.full((N,), cfg["dt"], dtype=torch.float64, device=dev)
    y_ros = torch.empty_like(y0)
    y_rk = torch.empty_like(y0)
    f = torch.empty_like(y0)
    st_ros = torch.empty(N, dtype=torch.int32, device=dev)
    st_rk = torch.empty(N, dtype=torch.int32, device=dev)
    steps_ros = torch.empty((N, 2), dtype=torch.int32, device=dev)
    steps_rk = torch.empty((N, 2), dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for k in ("rhs", "ros4", "rkf45")}
    dur = {k: [] for k in ev}

    def step(record: bool):
        flush.fill_(1.0)
        y_ros.copy_(y0)
        y_rk.copy_(y0)
        ev["rhs"][0].record(stream)
        ck.rhs(gm, p, y0, f, stream=stream)
        ev["rhs"][1].record(stream)
        ev["ros4"][0].record(stream)
        ck.integrate_ros4(gm, p, y_ros, dt, st_ros, steps=steps_ros, stream=stream)
        ev["ros4"][1].record(stream)
        ev["rkf45"][0].record(stream)
        ck.integrate_rkf45(gm, p, y_rk, dt, st_rk, steps=steps_rk, stream=stream)
        ev["rkf45"][1].record(stream)
        if record:
            torch.cuda.synchronize()
            for k, (a, b) in ev.items():
                dur[k].append(a.elapsed_time(b) / 1e3)

    for _ in range(args.warmup):
        step(False)
    barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    barrier()
    elapsed = t0.elapsed_time(t1) / 1e3
    clocks = sampler.stop() if sampler else None
    elapsed = max_over_ranks(elapsed, world, dev)
    value = aggregate_rate(2.0 * N * args.steps, world, elapsed)

    # correctness guard: every reactor finished
    st_ok = int((st_ros == 0).sum().item()) == N and int((st_rk == 0).sum().item()) == N

    # RHS throughput benchmark: repeats of the RHS over the batch
    rhs_rate = None
    if args.rhs_repeats > 0:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a.record(stream)
        for _ in range(args.rhs_repeats):
            ck.rhs(gm, p, y0, f, stream=stream)
        b.record(stream)
        barrier()
        rhs_rate = N * args.rhs_repeats / (a.elapsed_time(b) / 1e3)

    # algorithmic FP64 work per launch (instructions; DFMA-equivalent flops = 2x)
    sr = steps_ros.sum(dim=1).double()
    sk = steps_rk.sum(dim=1).double()
    ros_instr = float(sr.sum().item()) * work["ros4_step_fp64"] + 2 * N * work["rhs_fp64"]
    rk_instr = float(sk.sum().item()) * work["rkf45_step_fp64"] + 2 * N * work["rhs_fp64"]
    rhs_instr = N * work["rhs_fp64"]
    mean = {k: float(np.mean(v)) for k, v in dur.items()}
    instr = {"ros4": ros_instr, "rkf45": rk_instr, "rhs": rhs_instr}
    kernel_names = {"ros4": "k_ros4", "rkf45": "k_rkf45", "rhs": "k_rhs"}
    top = max(mean, key=mean.get)
    achieved = 2.0 * instr[top] / mean[top] / 1e12
    traffic = _traffic_for(kernel_names[top])
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": kernel_names[top],
                "note": "FP64 pipe bound; flops = 2 x FP64 instructions of the algorithm "
                        "(DFMA-equivalent); peak = nominal FP64 of the recipe (1.25 TFLOP/s); a DFMA "
                        "probe measured 1.20 TFLOP/s"}
    breakdown = {k: {"ms": 1e3 * mean[k], "tflops_dfma_eq": 2.0 * instr[k] / mean[k] / 1e12,
                     "frac_of_fp64_peak": 2.0 * instr[k] / mean[k] / 1e12 / FP64_PEAK_TFLOPS}
                 for k in mean}
    breakdown["ros4"]["integrations_per_s"] = N / mean["ros4"]
    breakdown["rkf45"]["integrations_per_s"] = N / mean["rkf45"]
    breakdown["ros4"]["steps_mean"] = float(sr.mean().item())
    breakdown["ros4"]["steps_max"] = int(sr.max().item())
    breakdown["rkf45"]["steps_mean"] = float(sk.mean().item())
    breakdown["rkf45"]["steps_max"] = int(sk.max().item())

    # end to end through the C ABI with host buffers (the library stages)
    e2e = None
    if args.e2e_steps > 0:
        yh = np.ascontiguousarray(y_np)
        ph = np.ascontiguousarray(p_np)
        dth = np.full(N, cfg["dt"])
        fh = np.empty_like(yh)
        sth = np.empty(N, np.int32)
        h2d = d2h = 0
        barrier()
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            ck.rhs(gm, ph, yh, fh)
            h2d += ph.nbytes + yh.nbytes
            d2h += fh.nbytes
            for fn in (ck.integrate_ros4, ck.integrate_rkf45):
                yw = yh.copy()
                fn(gm, ph, yw, dth, sth)
                h2d += ph.nbytes + yw.nbytes + dth.nbytes
                d2h += yw.nbytes + sth.nbytes
        barrier()
        te = max_over_ranks(time.perf_counter() - te, world, dev)
        e2e = {"value": aggregate_rate(2.0 * N * args.e2e_steps, world, te), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.e2e_steps, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "steps": args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        cpu = cpu_baseline(args.cpu_sample)
        cpu.pop("seconds", None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded stand-ins for the paper's GRI-Mech 3.0-sized mechanism and "
                        "reactor states)",
                "config": _config_dict(cfg), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 3 * args.steps, "clocks": clocks,
                "rhs_evals_per_s": rhs_rate, "rhs_repeats": args.rhs_repeats, "breakdown": breakdown,
                "all_reactors_ok": st_ok}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serve(args):
    """Serving trace: Poisson arrivals of reactor batches (log-uniform
    1k-256k cells, one of the three mechanisms, dt log-uniform 1e-6..1e-4 s,
    ROS4 in the precision form or RKF45 50/50), state resident on the device.
    Latency = completion - arrival.  The continuous-batching server is
    compared with the plain form: one synchronous integration per request,
    first come first served."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    names = ["small", "medium", "large"]
    mechs = {nm: ck.load_mechanism(load_mechanism(CONFIGS[nm]["mech"])) for nm in names}
    rng = np.random.default_rng(2004)
    K = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, K))
    reqs = []
    for i in range(K):
        nm = names[int(rng.integers(3))]
        cells = int(round(10 ** rng.uniform(3, np.log10(256e3))))
        dt = 10 ** rng.uniform(-6, -4)
        method = int(rng.integers(2))
        y, p = reactor_states(nm, n=cells, seed_offset=500 + i)
        reqs.append(dict(name=nm, n=cells, dt=dt, method=method, y=torch.as_tensor(y, device="cuda"),
                         p=torch.as_tensor(p, device="cuda")))
    def opts_for(r):
        return ck.SolverOpts.make(precision=1 if r["method"] == 0 else 0)

    def fresh(r):
        return (r["y"].clone(), torch.full((r["n"],), r["dt"], dtype=torch.float64, device="cuda"),
                torch.empty(r["n"], dtype=torch.int32, device="cuda"))

    out = {}
    for form in ("server", "plain"):
        bufs = [fresh(r) for r in reqs]
        torch.cuda.synchronize()
        lat = [0.0] * K
        t0 = time.perf_counter()
        if form == "server":
            srv = ck.Server(hbm_budget_bytes=args.budget_gb << 30, streams=args.streams, chunk_reactors=args.chunk)
            tickets = {}
            pending = set()
            i = 0
            while i < K or pending:
                now = time.perf_counter() - t0
                while i < K and arrivals[i] <= now:
                    y, dt, st = bufs[i]
                    tickets[i] = srv.submit(mechs[reqs[i]["name"]], reqs[i]["method"], reqs[i]["p"], y, dt, st,
                                            opts=opts_for(reqs[i]))
                    pending.add(i)
                    i += 1
                for j in list(pending):
                    if srv.poll(tickets[j]) != 0:
                        lat[j] = time.perf_counter() - t0 - arrivals[j]
                        pending.discard(j)
                time.sleep(0.0005)
            srv.close()
        else:
            for i in range(K):
                now = time.perf_counter() - t0
                if arrivals[i] > now:
                    time.sleep(arrivals[i] - now)
                y, dt, st = bufs[i]
                fn = ck.integrate_ros4 if reqs[i]["method"] == 0 else ck.integrate_rkf45
                fn(mechs[reqs[i]["name"]], reqs[i]["p"], y, dt, st, opts=opts_for(reqs[i]))
                torch.cuda.synchronize()
                lat[i] = time.perf_counter() - t0 - arrivals[i]
        makespan = time.perf_counter() - t0
        ok = all(bool((b[2] == 0).all().item()) for b in bufs)
        cells = sum(r["n"] for r in reqs)
        out[form] = {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                     "reactors_per_s": cells / makespan, "makespan_s": makespan, "all_ok": ok}
    line = {"mode": "serve", "metric": METRIC, "requests": K, "rate_per_s": args.rate,
            "cells_total": int(sum(r["n"] for r in reqs)),
            "trace": "seed 2004: Poisson arrivals; cells log-uniform 1e3-2.56e5; mechanism uniform over the "
                     "10/53/111-species stand-ins; dt log-uniform 1e-6-1e-4 s; ROS4 (precision 1) or RKF45 "
                     "50/50; state resident on the device",
            "server": out["server"], "plain": out["plain"],
            "server_config": {"budget_gb": args.budget_gb, "streams": args.streams, "chunk_reactors": args.chunk}}
    print(json.dumps(line), flush=True)


def waste(steps: np.ndarray, P: int = 32) -> dict:
    """Eq. waste of the paper over consecutive work units of P reactors:
    W_j = 1 - sum_i N_i / (P max_i N_i), N_i = attempted steps of reactor i."""
    n = (len(steps) // P) * P
    if n == 0:
        return {"P": P, "mean": None, "frac_below_1pct": None}
    N = steps[:n].reshape(-1, P).astype(np.float64)
    mx = N.max(axis=1)
    W = 1.0 - N.sum(axis=1) / (P * np.where(mx > 0, mx, 1.0))
    return {"P": P, "mean": float(W.mean()), "frac_below_1pct": float((W < 0.01).mean())}


def run_batch(args):
    """Mixed workload: the three mechanisms 50/35/15 over 200000 reactors,
    half near ignition, dt log-uniform 1e-6..1e-4 s.  For RKF45 and ROS4:
    (a) the plain form, one launch per mechanism in sequence (RKF45 also in
    the paper's one-thread-per-reactor SIMT mapping), and (b) the batching
    form: the three groups as persistent work-queue kernels on forked
    branches, heaviest first, captured in a CUDA graph and replayed, with the
    default launch shapes and with autotuned ones."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from paper_1608_05794_gb300 import autotune
    from synth.configs import CONFIGS, load_mechanism, mixed_batch
    groups = mixed_batch(n=args.batch_reactors)
    mdicts = {nm: load_mechanism(CONFIGS[nm]["mech"]) for nm, *_ in groups}
    mechs = {nm: ck.load_mechanism(mdicts[nm]) for nm in mdicts}
    dev = [dict(name=nm, y=torch.as_tensor(y, device="cuda"), p=torch.as_tensor(p, device="cuda"),
                dt=torch.as_tensor(dt, device="cuda")) for nm, y, p, dt in groups]
    total = sum(g["y"].shape[0] for g in dev)

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    res = {}
    for method, mname in ((1, "rkf45"), (0, "ros4")):
        fn = ck.integrate_ros4 if method == 0 else ck.integrate_rkf45
        forms = {"plain_team": dict(form=2)} if method == 0 else {"simt_thread": dict(form=1),
                                                                  "plain_team": dict(form=2)}
        out = {}
        base_y = None
        for fname, kw in forms.items():
            ys = [g["y"].clone() for g in dev]
            sts = [torch.empty(g["y"].shape[0], dtype=torch.int32, device="cuda") for g in dev]
            stp = [torch.empty((g["y"].shape[0], 2), dtype=torch.int32, device="cuda") for g in dev]

            def run_seq():
                for g, yy, st, sp in zip(dev, ys, sts, stp):
                    fn(mechs[g["name"]], g["p"], yy, g["dt"], st, steps=sp, opts=ck.SolverOpts.make(**kw))
            t = timed(run_seq)
            steps_all = np.concatenate([sp.cpu().numpy().sum(1) for sp in stp])
            out[fname] = {"s": t, "reactors_per_s": total / t,
                          "all_ok": all(bool((st == 0).all().item()) for st in sts), "waste": waste(steps_all)}
            if fname == "plain_team":
                base_y = [yy.cpu().numpy() for yy in ys]
        tuned = {}
        for g in dev:
            k = min(args.tune_sample, g["y"].shape[0])
            tuned[g["name"]] = autotune.tune(mechs[g["name"]], mdicts[g["name"]], method, g["p"][:k], g["y"][:k],
                                             g["dt"][:k], sample=k)
        for gname, use_tuned in (("graph_groups", False), ("graph_tuned_groups", True)):
            ys = [g["y"].clone() for g in dev]
            sts = [torch.empty(g["y"].shape[0], dtype=torch.int32, device="cuda") for g in dev]
            specs = [dict(mech=mechs[g["name"]], p=g["p"], y=yy, dt=g["dt"], status=st,
                          opts=ck.SolverOpts.make(**(tuned[g["name"]] if use_tuned else {"form": 2})))
                     for g, yy, st in zip(dev, ys, sts)]
            ck.integrate_groups(method, specs, use_graph=True)  # capture
            torch.cuda.synchronize()
            for yy, g in zip(ys, dev):
                yy.copy_(g["y"])
            t = timed(lambda: ck.integrate_groups(method, specs, use_graph=True))
            same = all(np.array_equal(yy.cpu().numpy(), b) for yy, b in zip(ys, base_y))
            out[gname] = {"s": t, "reactors_per_s": total / t,
                          "all_ok": all(bool((st == 0).all().item()) for st in sts),
                          "results_equal_plain_bitwise": same}
            if use_tuned:
                out[gname]["tuned"] = {nm: tuned[nm] for nm in tuned}
        res[mname] = out
    ck.graph_cache_clear()
    line = {"mode": "batch", "metric": METRIC, "reactors": total,
            "workload": "small/medium/large stand-ins 50/35/15, half near ignition, T U[900,2800] K, dt "
                        "log-uniform 1e-6-1e-4 s, rtol 1e-9 atol 1e-12",
            "groups": {g["name"]: int(g["y"].shape[0]) for g in dev}, "results": res}
    print(json.dumps(line), flush=True)


def run_fdjac(args):
    """ROS4 with the forward-difference Jacobian the paper used (Sec. 5)
    against the analytic Jacobian (Sec. 6) on the same medium-workload
    reactors: integrations/s, attempted steps, RHS evaluations per step and
    the FP64 rate of each form (DFMA-equivalent, from ck_count_work)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    cfg = CONFIGS[WORKLOAD]
    m = load_mechanism(cfg["mech"])
    gm = ck.load_mechanism(m)
    work = ck.count_work(gm)
    N = args.fd_reactors
    y_np, p_np = reactor_states(WORKLOAD, n=N)
    y0 = torch.as_tensor(y_np, device="cuda")
    p = torch.as_tensor(p_np, device="cuda")
    dt = torch.full((N,), cfg["dt"], dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    n = len(m["mw"]) + 1
    out = {}
    finals = {}
    for name, jac in (("analytic", 0), ("forward_difference", 1)):
        y = torch.empty_like(y0)
        st = torch.empty(N, dtype=torch.int32, device="cuda")
        steps = torch.empty((N, 2), dtype=torch.int32, device="cuda")
        opts = ck.SolverOpts.make(jac=jac)
        times = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            y.copy_(y0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ck.integrate_ros4(gm, p, y, dt, st, steps=steps, opts=opts)
            b.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                times.append(a.elapsed_time(b) / 1e3)
        t = float(np.mean(times))
        attempted = float(steps.sum().item())
        per_step = work["ros4_fd_step_fp64"] if jac else work["ros4_step_fp64"]
        tflops = 2.0 * per_step * attempted / t / 1e12
        out[name] = {"s": t, "integrations_per_s": N / t, "steps_mean": attempted / N,
                     "rhs_per_step": (n + 3) if jac else 3, "jacobians_per_step": 0 if jac else 1,
                     "tflops_dfma_eq": tflops, "frac_of_fp64_peak": tflops / FP64_PEAK_TFLOPS,
                     "all_ok": bool((st == 0).all().item())}
        finals[name] = y.cpu().numpy()
    dY = np.abs(finals["analytic"][:, 1:] - finals["forward_difference"][:, 1:]).max()
    dT = (np.abs(finals["analytic"][:, 0] - finals["forward_difference"][:, 0]) / finals["analytic"][:, 0]).max()
    line = {"mode": "fdjac", "metric": "ROS4 reactor integrations/s, analytic vs forward-difference Jacobian",
            "workload": f"medium: {len(m['mw'])} species / {len(m['rtype'])} reactions, first {N} reactors, "
                        f"dt={cfg['dt']:g} s, rtol 1e-9, atol 1e-12",
            "results": out, "analytic_speedup": out["forward_difference"]["s"] / out["analytic"]["s"],
            "max_abs_dY_between_forms": float(dY), "max_rel_dT_between_forms": float(dT),
            "paper_context": "Sec. 5-6: forward differences cost S+1 RHS per Jacobian; an analytic Jacobian "
                             "gave 2.9x for ROS4 on GRI-Mech 3.0 (other hardware)"}
    print(json.dumps(line), flush=True)


def run_variants(args):
    """The reactor and rate-form variants of Sec. 3 on the medium mechanism,
    each timed like the default step (RHS x repeats, ROS4, RKF45 over
    dt = 1e-5 s): constant pressure with K_c reverse rates (the default),
    constant volume (densities log-uniform 0.1-3 kg/m^3), and constant
    pressure with a quarter of the reversible reactions on explicit reverse
    Arrhenius coefficients."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from oracle.mechgen import with_explicit_reverse
    from synth.configs import CONFIGS, cv_states, load_mechanism, reactor_states
    cfg = CONFIGS[WORKLOAD]
    base = load_mechanism(cfg["mech"])
    N = args.variant_reactors
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    res = {}
    for name, mech, reactor in (("constant_pressure", base, 0), ("constant_volume", base, 1),
                                ("explicit_reverse", with_explicit_reverse(base), 0)):
        gm = ck.load_mechanism(mech, reactor=reactor)
        work = ck.count_work(gm)
        y_np, par_np = (cv_states(WORKLOAD, N) if reactor else reactor_states(WORKLOAD, n=N))
        y0 = torch.as_tensor(y_np, device="cuda")
        par = torch.as_tensor(par_np, device="cuda")
        dt = torch.full((N,), cfg["dt"], dtype=torch.float64, device="cuda")
        out = {}
        f = torch.empty_like(y0)
        t = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(args.rhs_repeats_variant):
                ck.rhs(gm, par, y0, f)
            b.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                t.append(a.elapsed_time(b) / 1e3 / args.rhs_repeats_variant)
        trhs = float(np.mean(t))
        out["rhs"] = {"evals_per_s": N / trhs,
                      "tflops_dfma_eq": 2.0 * work["rhs_fp64"] * N / trhs / 1e12}
        for mname, fn, per_key in (("ros4", ck.integrate_ros4, "ros4_step_fp64"),
                                   ("rkf45", ck.integrate_rkf45, "rkf45_step_fp64")):
            y = torch.empty_like(y0)
            st = torch.empty(N, dtype=torch.int32, device="cuda")
            steps = torch.empty((N, 2), dtype=torch.int32, device="cuda")
            t = []
            for i in range(args.warmup + args.steps):
                flush.fill_(1.0)
                y.copy_(y0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn(gm, par, y, dt, st, steps=steps)
                b.record()
                torch.cuda.synchronize()
                if i >= args.warmup:
                    t.append(a.elapsed_time(b) / 1e3)
            tm = float(np.mean(t))
            att = float(steps.sum().item())
            tf = 2.0 * work[per_key] * att / tm / 1e12
            out[mname] = {"integrations_per_s": N / tm, "steps_mean": att / N, "tflops_dfma_eq": tf,
                          "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS, "all_ok": bool((st == 0).all().item())}
        res[name] = out
    line = {"mode": "variants", "metric": "reactor integrations/s and RHS evals/s per reactor / rate-form variant",
            "workload": f"medium: {len(base['mw'])} species / {len(base['rtype'])} reactions, {N} reactors, "
                        f"dt={cfg['dt']:g} s, rtol 1e-9, atol 1e-12",
            "results": res}
    print(json.dumps(line), flush=True)


def run_precision(args):
    """ROS4 in the FP64 form and the precision forms (FP32 LU and solves with
    one or two FP64 refinement steps) on the medium and large workloads;
    reports integrations/s and the largest final-state difference from the
    FP64 form (the parity tests compare every form with the oracle)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    res = {}
    for name, N in (("medium", args.precision_reactors), ("large", args.precision_reactors // 2)):
        cfg = CONFIGS[name]
        gm = ck.load_mechanism(load_mechanism(cfg["mech"]))
        y_np, p_np = reactor_states(name, n=N)
        y0 = torch.as_tensor(y_np, device="cuda")
        p = torch.as_tensor(p_np, device="cuda")
        dt = torch.full((N,), cfg["dt"], dtype=torch.float64, device="cuda")
        st = torch.empty(N, dtype=torch.int32, device="cuda")
        out, finals = {}, {}
        for prec in (0, 1, 2):
            y = torch.empty_like(y0)
            ts = []
            for i in range(args.warmup + args.steps):
                y.copy_(y0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ck.integrate_ros4(gm, p, y, dt, st, opts=ck.SolverOpts.make(precision=prec))
                b.record()
                torch.cuda.synchronize()
                if i >= args.warmup:
                    ts.append(a.elapsed_time(b) / 1e3)
            finals[prec] = y.cpu().numpy()
            out[f"precision_{prec}"] = {"integrations_per_s": N / float(np.mean(ts)),
                                        "all_ok": bool((st == 0).all().item())}
        for prec in (1, 2):
            d = finals[prec] - finals[0]
            out[f"precision_{prec}"]["max_rel_dT_vs_fp64"] = float(np.max(np.abs(d[:, 0]) / finals[0][:, 0]))
            out[f"precision_{prec}"]["max_abs_dY_vs_fp64"] = float(np.max(np.abs(d[:, 1:])))
        res[f"{name} ({N} reactors)"] = out
    print(json.dumps({"mode": "precision", "metric": "ROS4 reactor integrations/s, FP64 vs FP32 LU + FP64 refinement",
                      "dt": "each workload's", "results": res}), flush=True)


def run_profile_case(args):
    """A small case of one kernel for ncu (warm-up launches, then 3 launches)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    cfg = CONFIGS[WORKLOAD]
    gm = ck.load_mechanism(load_mechanism(cfg["mech"]))
    N = args.reactors
    y_np, p_np = reactor_states(WORKLOAD, n=N)
    y0 = torch.as_tensor(y_np, device="cuda")
    p = torch.as_tensor(p_np, device="cuda")
    dt = torch.full((N,), args.dt or cfg["dt"], dtype=torch.float64, device="cuda")
    y = torch.empty_like(y0)
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup + args.steps):
        y.copy_(y0)
        if args.profile_case == "ros4":
            ck.integrate_ros4(gm, p, y, dt, st)
        elif args.profile_case == "rkf45":
            ck.integrate_rkf45(gm, p, y, dt, st)
        else:
            ck.rhs(gm, p, y0, y)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "reactors": N, "launches": args.warmup + args.steps,
                      "ok": bool((st == 0).all().item()) if args.profile_case != "rhs" else True}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rhs-repeats", type=int, default=1000)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=128)
    ap.add_argument("--profile-case", choices=["ros4", "rkf45", "rhs"], default=None,
                    help="profiling only: launch one kernel a few times on a small batch, print no bench line")
    ap.add_argument("--reactors", type=int, default=2048, help="batch size of --profile-case")
    ap.add_argument("--dt", type=float, default=None, help="dt of --profile-case (default: the workload's)")
    ap.add_argument("--mode", choices=["bench", "serve", "batch", "fdjac", "variants", "precision"], default="bench")
    ap.add_argument("--precision-reactors", type=int, default=32768, help="precision: medium reactors (large: half)")
    ap.add_argument("--variant-reactors", type=int, default=32768, help="variants: medium-workload reactors")
    ap.add_argument("--rhs-repeats-variant", type=int, default=20, help="variants: RHS passes per timing")
    ap.add_argument("--fd-reactors", type=int, default=8192, help="fdjac: medium-workload reactors")
    ap.add_argument("--batch-reactors", type=int, default=200000, help="batch: reactors of the mixed workload")
    ap.add_argument("--tune-sample", type=int, default=4096, help="batch: reactors timed per autotuner candidate")
    ap.add_argument("--requests", type=int, default=12, help="serve: requests in the trace")
    ap.add_argument("--rate", type=float, default=500.0, help="serve: Poisson arrival rate, requests/s")
    ap.add_argument("--budget-gb", type=int, default=64, help="serve: HBM budget of the server")
    ap.add_argument("--streams", type=int, default=4, help="serve: server streams")
    ap.add_argument("--chunk", type=int, default=8192, help="serve: reactors per launched chunk")
    args = ap.parse_args()
    if args.mode == "serve":
        run_serve(args)
    elif args.mode == "fdjac":
        run_fdjac(args)
    elif args.mode == "variants":
        run_variants(args)
    elif args.mode == "precision":
        run_precision(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
