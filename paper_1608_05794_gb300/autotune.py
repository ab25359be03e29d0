"""Launch-shape autotuner for the integrators.

For one (mechanism, method, precision) it times every candidate launch shape
on a sample of the caller's reactors and keeps the fastest; for a mixed
batch (ck_integrate_groups) it also times the groups side by side against
one after another and keeps the faster.  The shapes only
change how reactors are mapped to the GPU (thread per reactor or CTA per
reactor, the thread grid of a ROS4 team, resident CTAs per SM); every shape
computes every reactor with the same arithmetic in the same order, so the
choice never changes a result.  Choices are cached in a JSON file keyed by
the mechanism's content digest, the method, the precision and the GPU name.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import ck

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def mech_digest(m: dict, reactor: int = 0) -> str:
    h = hashlib.sha256()
    for k in ("mw", "nasa", "tmid", "reac", "prod", "arrh", "rtype", "rev", "arrh0", "eff_ptr", "eff_sp", "eff_val",
              "arrh_rev"):
        if k in m:
            h.update(k.encode())
            h.update(np.ascontiguousarray(m[k]).tobytes())
    h.update(str(int(reactor)).encode())
    return h.hexdigest()[:16]


def candidates(method: int, n_species: int):
    if method == 0:
        out = [dict(team=0, variant=v) for v in (0, 5, 4, 3)]
        if n_species + 1 <= 56:
            out.append(dict(team=16, variant=0))
        return out
    return [dict(form=1, variant=0), dict(form=1, variant=2), dict(form=2, variant=0), dict(form=2, variant=16),
            dict(form=2, variant=8)]


def _time(fn, torch):
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def tune(mech, mdict, method, p, y, dt, precision=0, cache=DEFAULT_CACHE, sample=4096, refresh=False):
    """Best launch shape (a dict of SolverOpts fields) for this mechanism and
    method, timed on up to `sample` of the given device reactors."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = f"{mech_digest(mdict, getattr(mech, 'reactor', 0))}:{method}:{precision}:{gpu}"
    db = {}
    if os.path.exists(cache):
        try:
            db = json.load(open(cache))
        except (OSError, ValueError):
            db = {}
    if key in db and not refresh:
        return db[key]["opts"]
    k = min(sample, y.shape[0])
    fn = ck.integrate_ros4 if method == 0 else ck.integrate_rkf45
    timings = []
    for cand in candidates(method, mech.S):
        opts = ck.SolverOpts.make(precision=precision, **cand)
        yy = y[:k].clone()
        st = torch.empty(k, dtype=torch.int32, device=y.device)
        fn(mech, p[:k], yy, dt[:k], st, opts=opts)  # warm-up (and resource setup)
        yy = y[:k].clone()
        t = _time(lambda: fn(mech, p[:k], yy, dt[:k], st, opts=opts), torch)
        timings.append((t, cand))
    best = min(timings, key=lambda x: x[0])[1]
    db[key] = {"opts": best, "timings_s": [[t, c] for t, c in timings], "sample": k}
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tmp = cache + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1)
    os.replace(tmp, cache)
    return best


def tune_groups(method, groups, mdicts, cache=DEFAULT_CACHE, refresh=False):
    """True when the groups of a ck_integrate_groups call run faster one
    after another than side by side.  Both launch orders are captured in a
    CUDA graph, run once and replayed once under timing on the caller's
    groups (device tensors; every group's y is restored between runs); the
    two give bitwise the same results.  Cached under the mechanisms' content
    digests, the group sizes (to the next power of two), the method and the
    GPU name.  mdicts: the mechanism dict of each group."""
    import torch
    gpu = torch.cuda.get_device_name()
    parts = [f"{mech_digest(md, getattr(g['mech'], 'reactor', 0))}x{1 << max(0, int(g['y'].shape[0] - 1).bit_length())}"
             for g, md in zip(groups, mdicts)]
    key = "groups:" + ":".join(parts) + f":{method}:{gpu}"
    db = {}
    if os.path.exists(cache):
        try:
            db = json.load(open(cache))
        except (OSError, ValueError):
            db = {}
    if key in db and not refresh:
        return db[key]["sequential"]
    y0 = [g["y"].clone() for g in groups]
    times = {}
    for seq in (False, True):
        ck.integrate_groups(method, groups, use_graph=True, sequential=seq)  # capture and run
        for g, y in zip(groups, y0):
            g["y"].copy_(y)
        times[seq] = _time(lambda: ck.integrate_groups(method, groups, use_graph=True, sequential=seq), torch)
        for g, y in zip(groups, y0):
            g["y"].copy_(y)
    best = times[True] < times[False]
    db[key] = {"sequential": best, "timings_s": {"concurrent": times[False], "sequential": times[True]}}
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tmp = cache + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1)
    os.replace(tmp, cache)
    return best
