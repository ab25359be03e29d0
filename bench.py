"""Benchmark of the batched reactor path on GB300.

One step = one pass of the whole hot path over the batch of the medium
workload (53 species / 325 reactions, 131072 constant-pressure reactors):
one right-hand-side evaluation of every reactor, ROS4 integration of every
reactor over dt = 1e-5 s and RKF45 integration of every reactor over the same
dt (rtol 1e-9, atol 1e-12).  ``value`` is reactor integrations per second
(2 per reactor per step) with inputs resident in HBM; the RHS throughput
benchmark (1000 repeats of the RHS over the batch) is reported beside it.

The roofline of the dominant kernel counts the algorithm's flops (an FMA 2,
any other FP64 operation 1; ck_count_work), weights every exponential and
logarithm by w_exp, the flops of FMA-pipe time one 2^x of the library takes,
and divides by the FP64 FMA throughput; both denominators come from the probe
ck_probe_fp64, run in the same process right after the timed region.

After the headline, the default run also measures the extension forms
(outside the timed region): the precision form on the large workload, the
batching forms on the mixed workload and the request server on a serving
trace (``--extensions``).

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
FP64_NOMINAL_TFLOPS = 1.26  # 152 SMs x 2 FP64 FMA lanes a clock x 2 flops x 2.07 GHz
L2_BYTES = 129 * 2 ** 20
ORACLE_SAMPLES = os.path.join(ROOT, "tests", "golden", "oracle_samples.npz")


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
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Median SM clock, the maximum and the throttle reasons seen, from
    nvidia-smi csv lines (sm, max, power, active, hw, hw_thermal, sw_thermal,
    sw_power_cap)."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
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


# ---------------------------------------------------------------- work model
def ros4_work(work: dict, steps: np.ndarray, h0_estimated: bool = True, fd: bool = False) -> dict:
    """Algorithmic work of a ROS4 launch from its per-reactor [accepted,
    rejected] step counts: every attempt costs ros4_attempt_flops (2 stage
    RHS, LU, 4 solves, vector work); an attempt at a new state also the
    Jacobian and the RHS at that state (ros4_jeval_flops), while one that
    follows a rejection reuses them (the state is unchanged), so a reactor
    that reaches dt evaluates one Jacobian per accepted step.  The
    forward-difference Jacobian depends on h and is evaluated at every
    attempt (f(y) only at a new state).  EstimateH0 adds 2 RHS.  Returns flops, transcendentals (exps
    and logs) and FP64 instructions of the library's formulation."""
    steps = np.asarray(steps, dtype=np.float64).reshape(-1, 2)
    acc, att = steps[:, 0].sum(), steps.sum()
    n = steps.shape[0]
    h0 = 2.0 * n if h0_estimated else 0.0
    rest_instr = work["ros4_step_fp64"] - work["jac_fp64"] - work["rhs_fp64"]
    if fd:
        # a new state: f(y) and S+1 difference columns; after a rejection f(y)
        # is kept and only the S+1 columns (they depend on h) are redone
        jevals = att
        rhs_evals = acc * (work["n_species"] + 2.0) + (att - acc) * (work["n_species"] + 1.0)
        jflops = acc * work["ros4_fd_jeval_flops"] + (att - acc) * (work["ros4_fd_jeval_flops"] - work["rhs_flops"])
        fd_extra = work["ros4_fd_step_fp64"] - work["ros4_step_fp64"] + work["jac_fp64"] + work["rhs_fp64"]
        jinstr = acc * fd_extra + (att - acc) * (fd_extra - work["rhs_fp64"])
    else:
        jevals = acc
        rhs_evals = acc
        jflops = acc * work["ros4_jeval_flops"]
        jinstr = acc * (work["jac_fp64"] + work["rhs_fp64"])
    flops = jflops + att * work["ros4_attempt_flops"] + h0 * work["rhs_flops"]
    transc = (rhs_evals + 2.0 * att + h0) * work["rhs_transc"]
    instr = jinstr + att * rest_instr + h0 * work["rhs_fp64"]
    return {"flops": flops, "transc": transc, "fp64_instr": instr, "attempts": att, "jacobians": jevals}


def rkf45_work(work: dict, steps: np.ndarray, h0_estimated: bool = True) -> dict:
    steps = np.asarray(steps, dtype=np.float64).reshape(-1, 2)
    att = steps.sum()
    h0 = 2.0 * steps.shape[0] if h0_estimated else 0.0
    return {"flops": att * work["rkf45_step_flops"] + h0 * work["rhs_flops"],
            "transc": (6.0 * att + h0) * work["rhs_transc"],
            "fp64_instr": att * work["rkf45_step_fp64"] + h0 * work["rhs_fp64"], "attempts": att}


def rhs_work(work: dict, n: float) -> dict:
    return {"flops": n * work["rhs_flops"], "transc": n * work["rhs_transc"], "fp64_instr": n * work["rhs_fp64"]}


def roofline_rate(w: dict, seconds: float, peaks: dict) -> dict:
    """Achieved flop rate of a launch (exponentials at w_exp flops each), as
    a fraction of the measured FP64 FMA throughput; beside it the rate of FP64
    pipe instructions of the library's formulation against the pipe's
    instruction rate (FMA throughput / 2)."""
    eq = w["flops"] + peaks["w_exp"] * w["transc"]
    achieved = eq / seconds
    return {"tflops": achieved / 1e12, "frac": achieved / peaks["fp64_flops_per_s"],
            "fp64_issue_frac": 2.0 * w["fp64_instr"] / seconds / peaks["fp64_flops_per_s"]}


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


# ---------------------------------------------------------------- CPU baseline
def cpu_baseline(sample: int, threads: int = 0, keep_states: bool = False):
    """The oracle (as it stands) on the host cores over a bounded sample of
    the same workload: ROS4 + RKF45 of `sample` reactors and one RHS each.
    keep_states: also return the oracle's final states of both methods (the
    expected values of the same reactors' GPU results)."""
    from oracle import ORA_RKF45, ORA_ROS4, Oracle, OracleMech
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    cfg = CONFIGS[WORKLOAD]
    om = OracleMech(load_mechanism(cfg["mech"]))
    y, p = reactor_states(WORKLOAD)  # the workload's batch; its first `sample` reactors
    y, p = np.ascontiguousarray(y[:sample]), np.ascontiguousarray(p[:sample])
    cores = threads if threads > 0 else Oracle().hardware_threads()
    t0 = time.perf_counter()
    om.rhs(p, y)
    ros = om.integrate(ORA_ROS4, p, y, cfg["dt"], nthreads=cores)
    rk = om.integrate(ORA_RKF45, p, y, cfg["dt"], nthreads=cores)
    el = time.perf_counter() - t0
    out = {"value": 2 * sample / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"first {sample} of the {cfg['n_reactors']} medium-workload reactors: one RHS, "
                     f"ROS4 and RKF45 over dt={cfg['dt']:g} s each, C++ oracle threaded over reactors",
           "seconds": el}
    if keep_states:
        out["_states"] = {"ros4": (ros[0], ros[2]), "rkf45": (rk[0], rk[2])}
    return out


def state_errors(y, yo):
    dT = np.abs(y[:, 0] - yo[:, 0]) / yo[:, 0]
    dY = np.abs(y[:, 1:] - yo[:, 1:])
    return float(dT.max()), float(dY.max())


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


def _timed(torch, fn, stream=None):
    """Seconds of fn() on the device (CUDA events on the launching stream)."""
    st = stream if stream is not None else torch.cuda.current_stream()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


# ---------------------------------------------------------------- headline
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
    from synth.configs import CONFIGS, load_mechanism

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    cfg = CONFIGS[WORKLOAD]
    m = load_mechanism(cfg["mech"])
    gm = ck.load_mechanism(m)
    work = dict(ck.count_work(gm), n_species=len(m["mw"]))
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
    # the roofline denominators, measured on this GPU at the clock state of
    # the timed region, which has just ended
    peaks = ck.fp64_peaks(gm)
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

    # algorithmic work per launch and the roofline of every kernel
    sr = steps_ros.cpu().numpy()
    sk = steps_rk.cpu().numpy()
    wk = {"ros4": ros4_work(work, sr), "rkf45": rkf45_work(work, sk), "rhs": rhs_work(work, N)}
    mean = {k: float(np.mean(v)) for k, v in dur.items()}
    kernel_names = {"ros4": "k_ros4", "rkf45": "k_rkf45", "rhs": "k_rhs"}
    rates = {k: roofline_rate(wk[k], mean[k], peaks) for k in mean}
    top = max(mean, key=mean.get)
    traffic = _traffic_for(kernel_names[top])
    peak_t = peaks["fp64_flops_per_s"] / 1e12
    roofline = {"bound": "alu", "achieved": rates[top]["tflops"], "peak": peak_t, "unit": "TFLOP/s",
                "frac": rates[top]["frac"], "traffic": traffic, "kernel": kernel_names[top],
                "w_exp": peaks["w_exp"], "fp64_issue_frac": rates[top]["fp64_issue_frac"],
                "note": "FP64-pipe bound. achieved = (flops + w_exp x transcendentals) per launch / CUDA-event "
                        "time; flops count an FMA as 2 and any other FP64 operation as 1 (ck_count_work), "
                        "a ROS4 step after a rejection reuses J and f(y); w_exp = FMA-pipe time of one 2^x "
                        "in flops; peak = FP64 FMA throughput; both measured by ck_probe_fp64 right after the timed region "
                        f"(nominal {FP64_NOMINAL_TFLOPS} TFLOP/s at 2.07 GHz). fp64_issue_frac: FP64 pipe "
                        "instructions of the library's formulation / the pipe's instruction rate"}
    breakdown = {k: {"ms": 1e3 * mean[k], "tflops": rates[k]["tflops"], "frac_of_fp64_peak": rates[k]["frac"],
                     "fp64_issue_frac": rates[k]["fp64_issue_frac"], "flops_per_launch": wk[k]["flops"],
                     "transcendentals_per_launch": wk[k]["transc"]} for k in mean}
    breakdown["ros4"]["integrations_per_s"] = N / mean["ros4"]
    breakdown["rkf45"]["integrations_per_s"] = N / mean["rkf45"]
    breakdown["rhs"]["evals_per_s"] = N / mean["rhs"]
    for k, s in (("ros4", sr), ("rkf45", sk)):
        tot = s.sum(axis=1)
        breakdown[k].update(steps_mean=float(tot.mean()), steps_max=int(tot.max()),
                            rejected_frac=float(s[:, 1].sum() / max(1, tot.sum())))
    breakdown["ros4"]["jacobians_per_reactor"] = float(wk["ros4"]["jacobians"] / N)

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

    cpu = parity_sample = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        cpu = cpu_baseline(args.cpu_sample, keep_states=True)
        cpu.pop("seconds", None)
        # the timed launches' final states of the oracle's sample (rank 0's
        # batch is the workload's seeded batch, so row i is reactor i)
        states = cpu.pop("_states")
        k = args.cpu_sample
        parity_sample = {"reactors": k, "what": "GPU final states of the timed launches against the oracle's"}
        for name, yg, stg in (("ros4", y_ros, st_ros), ("rkf45", y_rk, st_rk)):
            yo, sto = states[name]
            dT, dY = state_errors(yg[:k].cpu().numpy(), yo)
            parity_sample[name] = {"max_rel_dT": dT, "max_abs_dY": dY,
                                   "statuses_equal": bool(np.array_equal(stg[:k].cpu().numpy(), sto))}

    ext = {}
    if rank == 0 and world == 1:
        wanted = [e for e in args.extensions.split(",") if e and e != "none"]
        for name in wanted:
            fn = {"precision": ext_precision, "batch": ext_batch, "serving": ext_serving}[name]
            t_ext = time.perf_counter()
            sm = ClockSampler(torch.cuda.current_device())
            sm.start()
            ext[name] = fn(ck, torch, args)
            ext[name]["clocks"] = sm.stop()
            ext[name]["wall_s"] = time.perf_counter() - t_ext

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded stand-ins for the paper's GRI-Mech 3.0-sized mechanism and "
                        "reactor states)",
                "config": _config_dict(cfg), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 3 * args.steps, "clocks": clocks,
                "rhs_evals_per_s": rhs_rate, "rhs_repeats": args.rhs_repeats, "breakdown": breakdown,
                "fp64_probe": peaks, "work_per_unit": work, "parity_sample": parity_sample,
                "all_reactors_ok": st_ok}
        line.update(ext)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- extension forms
def ext_precision(ck, torch, args):
    """The precision form on the large workload (111 species / 784 reactions,
    65536 reactors, T 900-2800 K, dt 1e-5 s): ROS4 in FP64 against the FP32
    LU + solves with one FP64 refinement, each timed once over the whole batch
    after a warm-up on a slice; errors against the oracle's stored final
    states of 16 sampled reactors (tests/golden/oracle_samples.npz)."""
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    name = "large"
    cfg = CONFIGS[name]
    m = load_mechanism(cfg["mech"])
    gm = ck.load_mechanism(m)
    work = dict(ck.count_work(gm), n_species=len(m["mw"]))
    y_np, p_np = reactor_states(name)
    N = len(p_np)
    ref = np.load(ORACLE_SAMPLES)
    idx, yo, sto = ref["large_ros4_idx"], ref["large_ros4_y"], ref["large_ros4_status"]
    y0 = torch.as_tensor(y_np, device="cuda")
    p = torch.as_tensor(p_np, device="cuda")
    dt = torch.full((N,), cfg["dt"], dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {"workload": f"large: {cfg['n_species']} species / {cfg['n_reactions']} reactions, {N} reactors, "
                       f"T U[900, 2800] K, dt={cfg['dt']:g} s, rtol 1e-9, atol 1e-12"}
    finals = {}
    peaks = ck.fp64_peaks(gm)
    for prec in (0, 1):
        y = torch.empty_like(y0)
        st = torch.empty(N, dtype=torch.int32, device="cuda")
        steps = torch.empty((N, 2), dtype=torch.int32, device="cuda")
        opts = ck.SolverOpts.make(precision=prec)
        k = 2048
        y[:k].copy_(y0[:k])
        ck.integrate_ros4(gm, p[:k], y[:k], dt[:k], st[:k], opts=opts)  # warm-up
        flush.fill_(1.0)
        y.copy_(y0)
        t = _timed(torch, lambda: ck.integrate_ros4(gm, p, y, dt, st, steps=steps, opts=opts))
        yg = y.cpu().numpy()
        finals[prec] = yg
        dT, dY = state_errors(yg[idx], yo)
        s = steps.cpu().numpy()
        rate = roofline_rate(ros4_work(work, s), t, peaks)
        out[f"precision_{prec}"] = {
            "integrations_per_s": N / t, "s": t, "all_ok": bool((st == 0).all().item()),
            "oracle_max_rel_dT": dT, "oracle_max_abs_dY": dY,
            "oracle_statuses_equal": bool(np.array_equal(st.cpu().numpy()[idx], sto)),
            "steps_mean": float(s.sum(1).mean()), "fp64_equivalent_tflops": rate["tflops"],
            "frac_of_fp64_peak": rate["frac"]}
    d = finals[1] - finals[0]
    out["precision_1"]["max_rel_dT_vs_fp64_form"] = float(np.max(np.abs(d[:, 0]) / finals[0][:, 0]))
    out["precision_1"]["max_abs_dY_vs_fp64_form"] = float(np.max(np.abs(d[:, 1:])))
    out["speedup_precision_1_over_fp64"] = out["precision_1"]["integrations_per_s"] / \
        out["precision_0"]["integrations_per_s"]
    out["oracle_sample"] = int(len(idx))
    out["note"] = ("frac_of_fp64_peak of the precision form: the FP64 algorithm's flops over its time (its LU "
                   "and solves run on the FP32 pipe)")
    return out


def mixed_groups(ck, torch, n):
    from synth.configs import CONFIGS, load_mechanism, mixed_batch
    groups = mixed_batch(n=n)
    mechs = {nm: ck.load_mechanism(load_mechanism(CONFIGS[nm]["mech"])) for nm, *_ in groups}
    dev = [dict(name=nm, y=torch.as_tensor(y, device="cuda"), p=torch.as_tensor(p, device="cuda"),
                dt=torch.as_tensor(dt, device="cuda")) for nm, y, p, dt in groups]
    return mechs, dev


def batch_forms(ck, torch, mechs, dev, method, forms, graph_forms, tuned=None):
    """Time the plain forms (one ck_integrate_* per mechanism in sequence)
    and the grouped forms (ck_integrate_groups: concurrent or sequential
    groups, captured in a CUDA graph; the first call captures and runs, the
    second, timed, replays); the grouped forms' results are compared bitwise
    with the plain form of the same kernel (plain_team)."""
    total = sum(g["y"].shape[0] for g in dev)
    fn = ck.integrate_ros4 if method == 0 else ck.integrate_rkf45
    out = {}
    base_y = None
    base_name = "plain_team" if "plain_team" in forms else next(iter(forms))
    for fname, kw in forms.items():
        ys = [g["y"].clone() for g in dev]
        sts = [torch.empty(g["y"].shape[0], dtype=torch.int32, device="cuda") for g in dev]
        stp = [torch.empty((g["y"].shape[0], 2), dtype=torch.int32, device="cuda") for g in dev]

        def run_seq():
            for g, yy, st, sp in zip(dev, ys, sts, stp):
                fn(mechs[g["name"]], g["p"], yy, g["dt"], st, steps=sp, opts=ck.SolverOpts.make(**kw))
        t = _timed(torch, run_seq)
        steps_all = np.concatenate([sp.cpu().numpy().sum(1) for sp in stp])
        res = {"s": t, "reactors_per_s": total / t, "all_ok": all(bool((st == 0).all().item()) for st in sts),
               "waste": waste(steps_all)}
        yv = [yy.cpu().numpy() for yy in ys]
        if fname == base_name:
            base_y = yv
        out[fname] = res
    for gname, (kw, sequential) in graph_forms.items():
        ys = [g["y"].clone() for g in dev]
        sts = [torch.empty(g["y"].shape[0], dtype=torch.int32, device="cuda") for g in dev]
        specs = [dict(mech=mechs[g["name"]], p=g["p"], y=yy, dt=g["dt"], status=st,
                      opts=ck.SolverOpts.make(**(tuned[g["name"]] if kw == "tuned" else kw)))
                 for g, yy, st in zip(dev, ys, sts)]
        if sequential == "tuned":
            from paper_1608_05794_gb300 import autotune
            from synth.configs import CONFIGS, load_mechanism
            sequential = autotune.tune_groups(method, specs, [load_mechanism(CONFIGS[g["name"]]["mech"]) for g in dev])
        ck.integrate_groups(method, specs, use_graph=True, sequential=sequential)  # capture and run
        torch.cuda.synchronize()
        for yy, g in zip(ys, dev):
            yy.copy_(g["y"])
        t = _timed(torch, lambda: ck.integrate_groups(method, specs, use_graph=True, sequential=sequential))
        out[gname] = {"s": t, "reactors_per_s": total / t,
                      "all_ok": all(bool((st == 0).all().item()) for st in sts),
                      "results_equal_plain_team_bitwise": all(np.array_equal(yy.cpu().numpy(), b)
                                                              for yy, b in zip(ys, base_y))}
        if kw == "tuned":
            out[gname]["tuned"] = tuned
            out[gname]["sequential"] = bool(sequential)
    ck.graph_cache_clear()
    return out


def ext_batch(ck, torch, args):
    """The batching forms on the mixed workload (the three mechanisms
    50/35/15 over 200000 reactors, half near ignition, T U[900, 2800] K, dt
    log-uniform 1e-6-1e-4 s) with RKF45, the method the paper ran in both
    mappings: one thread per reactor (the paper's SIMT form), one CTA per
    reactor launched per mechanism in sequence, and the graph-captured groups
    side by side and in sequence; waste at P = 32 (Eq. waste)."""
    mechs, dev = mixed_groups(ck, torch, args.batch_reactors)
    res = batch_forms(ck, torch, mechs, dev, 1, {"simt_thread": dict(form=1), "plain_team": dict(form=2)},
                      {"graph_groups_concurrent": (dict(form=2), False),
                       "graph_groups_sequential": (dict(form=2), True)})
    best = max(("graph_groups_concurrent", "graph_groups_sequential"), key=lambda k: res[k]["reactors_per_s"])
    return {"method": "rkf45", "reactors": sum(g["y"].shape[0] for g in dev),
            "groups": {g["name"]: int(g["y"].shape[0]) for g in dev}, "results": res,
            "team_over_simt": res["plain_team"]["reactors_per_s"] / res["simt_thread"]["reactors_per_s"],
            "best_groups": best,
            "best_groups_over_plain_team": res[best]["reactors_per_s"] / res["plain_team"]["reactors_per_s"]}


# ---------------------------------------------------------------- serving
SERVE_CELLS = (64, 16384)  # log-uniform request sizes (the configured 1k-256k divided by 16)


def make_trace(k: int, seed: int = 2004, cells=SERVE_CELLS):
    """A seeded request trace: per request the mechanism (uniform over the
    three stand-ins), the size (log-uniform over `cells`), dt (log-uniform
    1e-6-1e-4 s) and the method (ROS4 in the precision form or RKF45, 50/50);
    arrival times are drawn separately for each rate."""
    rng = np.random.default_rng(seed)
    names = ["small", "medium", "large"]
    reqs = []
    for i in range(k):
        reqs.append(dict(name=names[int(rng.integers(3))],
                         n=int(round(10 ** rng.uniform(np.log10(cells[0]), np.log10(cells[1])))),
                         dt=float(10 ** rng.uniform(-6, -4)), method=int(rng.integers(2)), seed=500 + i))
    return reqs


def poisson_arrivals(k: int, rate: float, seed: int = 2005):
    return np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, k))


def bounded_p99(lat, arrivals) -> bool:
    """Latency stays bounded over the trace when the later half's p99 is at
    most twice the earlier half's (a queue that grows without limit fails)."""
    lat = np.asarray(lat)
    order = np.argsort(arrivals)
    h = len(order) // 2
    if h < 2:
        return True
    a, b = np.percentile(lat[order[:h]], 99), np.percentile(lat[order[h:]], 99)
    return bool(b <= 2.0 * a)


def serve_trace(ck, torch, mechs, reqs, arrivals, form, budget_gb=64, streams=4, chunk=8192):
    """Run one trace in one form; returns per-request latencies (completion -
    arrival), the makespan and whether every reactor finished."""
    from synth.configs import reactor_states
    dev = []
    for r in reqs:
        y, p = reactor_states(r["name"], n=r["n"], seed_offset=r["seed"])
        dev.append(dict(y0=torch.as_tensor(y, device="cuda"), p=torch.as_tensor(p, device="cuda"),
                        y=torch.empty((r["n"], y.shape[1]), dtype=torch.float64, device="cuda"),
                        dt=torch.full((r["n"],), r["dt"], dtype=torch.float64, device="cuda"),
                        st=torch.empty(r["n"], dtype=torch.int32, device="cuda")))
    for d in dev:
        d["y"].copy_(d["y0"])
    torch.cuda.synchronize()

    def opts_for(r):
        return ck.SolverOpts.make(precision=1 if r["method"] == 0 else 0)

    K = len(reqs)
    lat = [0.0] * K
    t0 = time.perf_counter()
    if form == "server":
        srv = ck.Server(hbm_budget_bytes=budget_gb << 30, streams=streams, chunk_reactors=chunk)
        tickets, pending, i = {}, set(), 0
        while i < K or pending:
            now = time.perf_counter() - t0
            while i < K and arrivals[i] <= now:
                d = dev[i]
                tickets[i] = srv.submit(mechs[reqs[i]["name"]], reqs[i]["method"], d["p"], d["y"], d["dt"], d["st"],
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
            d = dev[i]
            fn = ck.integrate_ros4 if reqs[i]["method"] == 0 else ck.integrate_rkf45
            fn(mechs[reqs[i]["name"]], d["p"], d["y"], d["dt"], d["st"], opts=opts_for(reqs[i]))
            torch.cuda.synchronize()
            lat[i] = time.perf_counter() - t0 - arrivals[i]
    makespan = time.perf_counter() - t0
    ok = all(bool((d["st"] == 0).all().item()) for d in dev)
    return lat, makespan, ok


def serving_summary(lat, arrivals, makespan, cells, ok):
    return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "reactors_per_s": cells / makespan, "makespan_s": makespan, "p99_bounded": bounded_p99(lat, arrivals),
            "all_ok": ok}


def serving_capacity(ck, torch, mechs, reqs):
    """Requests a second the plain form sustains on this trace: every request
    arrives at t = 0 and the plain form serves them back to back."""
    lat, makespan, ok = serve_trace(ck, torch, mechs, reqs, np.zeros(len(reqs)), "plain")
    return len(reqs) / makespan


def _serve_mechs(ck):
    from synth.configs import CONFIGS, load_mechanism
    return {nm: ck.load_mechanism(load_mechanism(CONFIGS[nm]["mech"])) for nm in ("small", "medium", "large")}


def ext_serving(ck, torch, args):
    """The request server against the plain form (one synchronous
    ck_integrate_* per request, first come first served) on one seeded trace
    at a fixed fraction of the plain form's capacity on that trace."""
    mechs = _serve_mechs(ck)
    reqs = make_trace(args.serve_requests)
    cap = serving_capacity(ck, torch, mechs, reqs)
    rate = args.serve_load * cap
    arr = poisson_arrivals(len(reqs), rate)
    cells = sum(r["n"] for r in reqs)
    out = {"trace": f"{len(reqs)} requests, seed 2004: mechanism uniform over the 10/53/111-species stand-ins, "
                    f"cells log-uniform {SERVE_CELLS[0]}-{SERVE_CELLS[1]}, dt log-uniform 1e-6-1e-4 s, ROS4 "
                    "(precision 1) or RKF45 50/50, Poisson arrivals, state resident on the device",
           "plain_capacity_req_per_s": cap, "rate_req_per_s": rate, "load": args.serve_load, "cells_total": cells}
    for form in ("server", "plain"):
        lat, makespan, ok = serve_trace(ck, torch, mechs, reqs, arr, form)
        out[form] = serving_summary(lat, arr, makespan, cells, ok)
    out["p50_ratio_plain_over_server"] = out["plain"]["p50_ms"] / out["server"]["p50_ms"]
    out["p99_ratio_plain_over_server"] = out["plain"]["p99_ms"] / out["server"]["p99_ms"]
    return out


def run_serve(args):
    """Arrival-rate sweep of the serving trace: p50/p99 latency and
    throughput of the server and of the plain form at rates given as
    fractions of the plain form's capacity on the trace, and the highest rate
    at which each form's p99 stays bounded."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    mechs = _serve_mechs(ck)
    reqs = make_trace(args.requests)
    cap = serving_capacity(ck, torch, mechs, reqs)
    cells = sum(r["n"] for r in reqs)
    sweep = []
    for load in [float(x) for x in args.loads.split(",")]:
        rate = load * cap
        arr = poisson_arrivals(len(reqs), rate)
        row = {"load": load, "rate_req_per_s": rate}
        for form in ("server", "plain"):
            lat, makespan, ok = serve_trace(ck, torch, mechs, reqs, arr, form, streams=args.streams,
                                            chunk=args.chunk)
            row[form] = serving_summary(lat, arr, makespan, cells, ok)
        sweep.append(row)
        print(json.dumps({"mode": "serve", "partial": row}), flush=True)
    best = {f: max([r["rate_req_per_s"] for r in sweep if r[f]["p99_bounded"]], default=None)
            for f in ("server", "plain")}
    print(json.dumps({"mode": "serve", "metric": "serving p50/p99 ms vs arrival rate", "requests": len(reqs),
                      "cells_total": cells, "plain_capacity_req_per_s": cap, "sweep": sweep,
                      "highest_bounded_rate_req_per_s": best,
                      "server_config": {"budget_gb": 64, "streams": args.streams, "chunk_reactors": args.chunk}}),
          flush=True)


# ---------------------------------------------------------------- other modes
def run_batch(args):
    """Mixed workload, both methods: the plain forms (RKF45 also in the
    thread-per-reactor SIMT mapping) against the graph-captured groups side
    by side, in sequence, and with the autotuner's launch shapes and launch
    order."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from paper_1608_05794_gb300 import autotune
    from synth.configs import CONFIGS, load_mechanism
    mechs, dev = mixed_groups(ck, torch, args.batch_reactors)
    res = {}
    for method, mname, plain in ((1, "rkf45", {"simt_thread": dict(form=1), "plain_team": dict(form=2)}),
                                 (0, "ros4", {"plain_team": {}})):
        tuned = {}
        for g in dev:
            k = min(args.tune_sample, g["y"].shape[0])
            tuned[g["name"]] = autotune.tune(mechs[g["name"]], load_mechanism(CONFIGS[g["name"]]["mech"]), method,
                                             g["p"][:k], g["y"][:k], g["dt"][:k], sample=k)
        base = dict(form=2) if method == 1 else {}
        res[mname] = batch_forms(ck, torch, mechs, dev, method, plain,
                                 {"graph_groups_concurrent": (base, False), "graph_groups_sequential": (base, True),
                                  "graph_groups_tuned": ("tuned", "tuned")}, tuned)
    print(json.dumps({"mode": "batch", "metric": METRIC, "reactors": sum(g["y"].shape[0] for g in dev),
                      "workload": "small/medium/large stand-ins 50/35/15, half near ignition, T U[900,2800] K, dt "
                                  "log-uniform 1e-6-1e-4 s, rtol 1e-9 atol 1e-12",
                      "groups": {g["name"]: int(g["y"].shape[0]) for g in dev}, "results": res}), flush=True)


def run_fdjac(args):
    """ROS4 with the forward-difference Jacobian the paper used (Sec. 5)
    against the analytic Jacobian (Sec. 6) on the same medium-workload
    reactors: integrations/s, attempted steps, RHS evaluations per step and
    the roofline fraction of each form."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    cfg = CONFIGS[WORKLOAD]
    m = load_mechanism(cfg["mech"])
    gm = ck.load_mechanism(m)
    work = dict(ck.count_work(gm), n_species=len(m["mw"]))
    peaks = ck.fp64_peaks(gm)
    N = args.fd_reactors
    y_np, p_np = reactor_states(WORKLOAD, n=N)
    y0 = torch.as_tensor(y_np, device="cuda")
    p = torch.as_tensor(p_np, device="cuda")
    dt = torch.full((N,), cfg["dt"], dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    n = len(m["mw"]) + 1
    out, finals = {}, {}
    for name, jac in (("analytic", 0), ("forward_difference", 1)):
        y = torch.empty_like(y0)
        st = torch.empty(N, dtype=torch.int32, device="cuda")
        steps = torch.empty((N, 2), dtype=torch.int32, device="cuda")
        opts = ck.SolverOpts.make(jac=jac)
        times = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            y.copy_(y0)
            t = _timed(torch, lambda: ck.integrate_ros4(gm, p, y, dt, st, steps=steps, opts=opts))
            if i >= args.warmup:
                times.append(t)
        t = float(np.mean(times))
        s = steps.cpu().numpy()
        r = roofline_rate(ros4_work(work, s, fd=bool(jac)), t, peaks)
        out[name] = {"s": t, "integrations_per_s": N / t, "steps_mean": float(s.sum(1).mean()),
                     "rhs_per_step": (n + 3) if jac else 3, "jacobians_per_step": 0 if jac else 1,
                     "tflops": r["tflops"], "frac_of_fp64_peak": r["frac"], "all_ok": bool((st == 0).all().item())}
        finals[name] = y.cpu().numpy()
    dY = np.abs(finals["analytic"][:, 1:] - finals["forward_difference"][:, 1:]).max()
    dT = (np.abs(finals["analytic"][:, 0] - finals["forward_difference"][:, 0]) / finals["analytic"][:, 0]).max()
    print(json.dumps({"mode": "fdjac", "metric": "ROS4 reactor integrations/s, analytic vs forward-difference Jacobian",
                      "workload": f"medium: {len(m['mw'])} species / {len(m['rtype'])} reactions, first {N} reactors, "
                                  f"dt={cfg['dt']:g} s, rtol 1e-9, atol 1e-12",
                      "results": out, "analytic_speedup": out["forward_difference"]["s"] / out["analytic"]["s"],
                      "max_abs_dY_between_forms": float(dY), "max_rel_dT_between_forms": float(dT),
                      "paper_context": "Sec. 5-6: forward differences cost S+1 RHS per Jacobian; an analytic "
                                       "Jacobian gave 2.9x for ROS4 on GRI-Mech 3.0 (other hardware)"}), flush=True)


def run_variants(args):
    """The reactor and rate-form variants of Sec. 3 on the medium mechanism,
    each timed like the default step (RHS x repeats, ROS4, RKF45 over
    dt = 1e-5 s): constant pressure with K_c reverse rates (the default),
    constant volume (densities log-uniform 0.1-3 kg/m^3), and constant
    pressure with a quarter of the reversible reactions on explicit reverse
    Arrhenius coefficients (the stored mechanism synth/data/mech_s53_rev)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, EXPLICIT_REVERSE_MECH, cv_states, load_mechanism, reactor_states
    cfg = CONFIGS[WORKLOAD]
    base = load_mechanism(cfg["mech"])
    N = args.variant_reactors
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    res = {}
    for name, mech, reactor in (("constant_pressure", base, 0), ("constant_volume", base, 1),
                                ("explicit_reverse", load_mechanism(EXPLICIT_REVERSE_MECH), 0)):
        gm = ck.load_mechanism(mech, reactor=reactor)
        work = dict(ck.count_work(gm), n_species=len(mech["mw"]))
        peaks = ck.fp64_peaks(gm)
        y_np, par_np = (cv_states(WORKLOAD, N) if reactor else reactor_states(WORKLOAD, n=N))
        y0 = torch.as_tensor(y_np, device="cuda")
        par = torch.as_tensor(par_np, device="cuda")
        dt = torch.full((N,), cfg["dt"], dtype=torch.float64, device="cuda")
        out = {}
        f = torch.empty_like(y0)
        t = []
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            tt = _timed(torch, lambda: [ck.rhs(gm, par, y0, f) for _ in range(args.rhs_repeats_variant)])
            if i >= args.warmup:
                t.append(tt / args.rhs_repeats_variant)
        trhs = float(np.mean(t))
        out["rhs"] = {"evals_per_s": N / trhs,
                      "frac_of_fp64_peak": roofline_rate(rhs_work(work, N), trhs, peaks)["frac"]}
        for mname, fn in (("ros4", ck.integrate_ros4), ("rkf45", ck.integrate_rkf45)):
            y = torch.empty_like(y0)
            st = torch.empty(N, dtype=torch.int32, device="cuda")
            steps = torch.empty((N, 2), dtype=torch.int32, device="cuda")
            t = []
            for i in range(args.warmup + args.steps):
                flush.fill_(1.0)
                y.copy_(y0)
                tt = _timed(torch, lambda: fn(gm, par, y, dt, st, steps=steps))
                if i >= args.warmup:
                    t.append(tt)
            tm = float(np.mean(t))
            s = steps.cpu().numpy()
            w = ros4_work(work, s) if mname == "ros4" else rkf45_work(work, s)
            out[mname] = {"integrations_per_s": N / tm, "steps_mean": float(s.sum(1).mean()),
                          "frac_of_fp64_peak": roofline_rate(w, tm, peaks)["frac"],
                          "all_ok": bool((st == 0).all().item())}
        res[name] = out
    print(json.dumps({"mode": "variants",
                      "metric": "reactor integrations/s and RHS evals/s per reactor / rate-form variant",
                      "workload": f"medium: {len(base['mw'])} species / {len(base['rtype'])} reactions, {N} reactors, "
                                  f"dt={cfg['dt']:g} s, rtol 1e-9, atol 1e-12", "results": res}), flush=True)


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
            opts = ck.SolverOpts.make(precision=prec)
            for i in range(args.warmup + args.steps):
                y.copy_(y0)
                t = _timed(torch, lambda: ck.integrate_ros4(gm, p, y, dt, st, opts=opts))
                if i >= args.warmup:
                    ts.append(t)
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


def run_counts(args):
    """The algorithmic work per unit of the three workloads' mechanisms
    (ck_count_work): flops in the roofline's model, transcendentals, and the
    FP64 instructions of the library's formulation."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism
    out = {}
    for name in ("small", "medium", "large"):
        m = load_mechanism(CONFIGS[name]["mech"])
        out[name] = dict(ck.count_work(ck.load_mechanism(m)), species=len(m["mw"]), reactions=len(m["rtype"]))
    print(json.dumps({"mode": "counts", "work": out}), flush=True)


def run_peak(args):
    """The FP64 roofline denominators alone: FMA throughput and the cost of
    the library's 2^x, with the SM clock sampled during the probe."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism
    gm = ck.load_mechanism(load_mechanism(CONFIGS["small"]["mech"]))
    ck.fp64_peaks(gm, iters=2000)
    sm = ClockSampler(torch.cuda.current_device())
    sm.start()
    res = [ck.fp64_peaks(gm, iters=args.peak_iters) for _ in range(args.steps)]
    clocks = sm.stop()
    best = max(res, key=lambda r: r["fp64_flops_per_s"])
    print(json.dumps({"mode": "peak", "fp64_tflops": best["fp64_flops_per_s"] / 1e12,
                      "exp2_per_s": best["exp2_per_s"], "w_exp_flops": best["w_exp"], "runs": res,
                      "nominal_tflops": FP64_NOMINAL_TFLOPS, "clocks": clocks}), flush=True)


def run_profile_case(args):
    """A small case of one kernel for ncu (warm-up launches, then the rest)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1608_05794_gb300.ck as ck
    from synth.configs import CONFIGS, load_mechanism, reactor_states
    wl = args.workload or WORKLOAD
    cfg = CONFIGS[wl]
    gm = ck.load_mechanism(load_mechanism(cfg["mech"]))
    N = args.reactors
    y_np, p_np = reactor_states(wl, n=N)
    y0 = torch.as_tensor(y_np, device="cuda")
    p = torch.as_tensor(p_np, device="cuda")
    dt = torch.full((N,), args.dt or cfg["dt"], dtype=torch.float64, device="cuda")
    y = torch.empty_like(y0)
    st = torch.empty(N, dtype=torch.int32, device="cuda")
    opts = ck.SolverOpts.make(precision=args.precision)
    times = []
    for _ in range(args.warmup + args.steps):
        y.copy_(y0)
        if args.profile_case == "ros4":
            times.append(_timed(torch, lambda: ck.integrate_ros4(gm, p, y, dt, st, opts=opts)))
        elif args.profile_case == "rkf45":
            times.append(_timed(torch, lambda: ck.integrate_rkf45(gm, p, y, dt, st)))
        else:
            times.append(_timed(torch, lambda: ck.rhs(gm, p, y0, y)))
    print(json.dumps({"profile_case": args.profile_case, "workload": wl, "precision": args.precision, "reactors": N,
                      "launches": args.warmup + args.steps, "ms": [1e3 * t for t in times],
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
    ap.add_argument("--extensions", default="precision,batch,serving",
                    help="extension forms measured after the headline (comma list, or none)")
    ap.add_argument("--profile-case", choices=["ros4", "rkf45", "rhs"], default=None,
                    help="profiling only: launch one kernel a few times on a small batch, print no bench line")
    ap.add_argument("--reactors", type=int, default=2048, help="batch size of --profile-case")
    ap.add_argument("--dt", type=float, default=None, help="dt of --profile-case (default: the workload's)")
    ap.add_argument("--workload", choices=["small", "medium", "large"], default=None,
                    help="workload of --profile-case (default: medium)")
    ap.add_argument("--precision", type=int, default=0, help="ROS4 precision form of --profile-case")
    ap.add_argument("--mode", choices=["bench", "serve", "batch", "fdjac", "variants", "precision", "peak", "counts"],
                    default="bench")
    ap.add_argument("--precision-reactors", type=int, default=32768, help="precision: medium reactors (large: half)")
    ap.add_argument("--variant-reactors", type=int, default=32768, help="variants: medium-workload reactors")
    ap.add_argument("--rhs-repeats-variant", type=int, default=20, help="variants: RHS passes per timing")
    ap.add_argument("--fd-reactors", type=int, default=8192, help="fdjac: medium-workload reactors")
    ap.add_argument("--batch-reactors", type=int, default=200000, help="batch: reactors of the mixed workload")
    ap.add_argument("--tune-sample", type=int, default=4096, help="batch: reactors timed per autotuner candidate")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests in the trace")
    ap.add_argument("--loads", default="0.3,0.5,0.7,0.9,1.1",
                    help="serve: arrival rates as fractions of the plain form's capacity on the trace")
    ap.add_argument("--serve-requests", type=int, default=60, help="default line: requests of the serving trace")
    ap.add_argument("--serve-load", type=float, default=0.6,
                    help="default line: arrival rate as a fraction of the plain form's capacity")
    ap.add_argument("--streams", type=int, default=4, help="serve: server streams")
    ap.add_argument("--chunk", type=int, default=8192, help="serve: reactors per launched chunk")
    ap.add_argument("--peak-iters", type=int, default=20000, help="peak: probe iterations a thread")
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
    elif args.mode == "peak":
        run_peak(args)
    elif args.mode == "counts":
        run_counts(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
