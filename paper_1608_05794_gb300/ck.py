"""Python binding of ``libck.so`` (argument marshalling only).

Every computation runs in the CUDA library declared in ``include/ck.h``;
this module converts torch tensors / numpy arrays into pointers and checks
return codes.  Device tensors are passed through (the call is asynchronous
on the given or current torch stream); numpy arrays are host memory, which
the library stages through the device and synchronizes.  There is no CPU
fallback: if the library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build

__all__ = [
    "Mechanism", "load_mechanism", "rhs", "jacobian", "lu_factor", "lu_solve", "integrate_ros4",
    "integrate_rkf45", "integrate_ros4_noalloc", "count_work", "Server", "integrate_groups", "Group",
    "graph_cache_clear", "device_errors", "SolverOpts", "CKError", "STATUS", "library_path", "probe_fp64",
    "fp64_peaks",
]

STATUS = {0: "OK", 1: "MAXSTEPS", 2: "HMIN", 3: "NONFINITE", 4: "SINGULAR", 5: "BADINPUT"}


class CKError(RuntimeError):
    pass


def _load():
    path = LIB
    if not os.path.exists(path):
        path = build()
    return C.CDLL(path)


_lib = _load()
_DP = C.c_void_p


class MechDesc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32), ("mw", _DP), ("nasa", _DP),
                ("t_mid", _DP), ("reac", _DP), ("prod", _DP), ("arrh", _DP), ("rtype", _DP),
                ("reversible", _DP), ("arrh0", _DP), ("eff_ptr", _DP), ("eff_sp", _DP), ("eff_val", _DP),
                ("n_elements", C.c_int32), ("elem_count", _DP), ("elem_mass", _DP), ("arrh_rev", _DP),
                ("reactor", C.c_int32)]


class SolverOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double), ("fixed_h", C.c_double),
                ("max_steps", C.c_int32), ("precision", C.c_int32), ("variant", C.c_int32),
                ("form", C.c_int32), ("team", C.c_int32), ("jac", C.c_int32)]

    @classmethod
    def make(cls, rtol=1e-9, atol=1e-12, h0=0.0, fixed_h=0.0, max_steps=100000, precision=0, variant=0,
             form=0, team=0, jac=0):
        return cls(rtol, atol, h0, fixed_h, max_steps, precision, variant, form, team, jac)

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Group(C.Structure):
    _fields_ = [("mech", C.c_void_p), ("n", C.c_int64), ("p", _DP), ("y", _DP), ("dt", _DP), ("h_inout", _DP),
                ("steps", _DP), ("status", _DP), ("opts", SolverOpts), ("work_weight", C.c_double)]


class WorkCounts(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("rhs_fp64", "rhs_exps", "jac_fp64", "lu_fp64", "solve_fp64",
                                           "ros4_step_fp64", "rkf45_step_fp64", "rhs_bytes",
                                           "integrate_bytes", "ros4_fd_step_fp64",
                                           "rhs_flops", "rhs_transc", "jac_flops", "lu_flops", "solve_flops",
                                           "ros4_jeval_flops", "ros4_attempt_flops", "ros4_step_flops",
                                           "rkf45_step_flops", "ros4_fd_jeval_flops")]


class ServerInfo(C.Structure):
    _fields_ = [("queued", C.c_int64), ("active", C.c_int64), ("completed", C.c_int64),
                ("bytes_in_use", C.c_uint64), ("budget", C.c_uint64), ("reserved", C.c_uint64)]


def _bind():
    L = _lib
    L.ck_load_mechanism.argtypes = [C.POINTER(MechDesc), C.POINTER(C.c_void_p)]
    L.ck_free_mechanism.argtypes = [C.c_void_p]
    L.ck_mech_info.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.ck_rhs.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP, _DP]
    L.ck_jacobian.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP, _DP]
    L.ck_jacobian_fd.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP, C.c_double, C.c_double, _DP, _DP]
    L.ck_lu_factor.argtypes = [C.c_int64, C.c_int32, _DP, _DP, _DP, _DP]
    L.ck_lu_solve.argtypes = [C.c_int64, C.c_int32, _DP, _DP, _DP, _DP]
    for f in (L.ck_integrate_ros4, L.ck_integrate_rkf45):
        f.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP, _DP, C.POINTER(SolverOpts), _DP, _DP, _DP]
    L.ck_integrate_ros4_noalloc.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP, _DP, C.POINTER(SolverOpts), _DP,
                                            _DP, _DP]
    L.ck_count_work.argtypes = [C.c_void_p, C.POINTER(WorkCounts)]
    L.ck_integrate_groups.argtypes = [C.c_int32, C.c_int32, C.POINTER(Group), C.c_int32, _DP]
    L.ck_server_create.argtypes = [C.c_size_t, C.c_int32, C.c_int64, C.POINTER(C.c_void_p)]
    L.ck_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, _DP, _DP, _DP, C.POINTER(SolverOpts),
                            _DP, _DP, C.POINTER(C.c_uint64)]
    L.ck_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(C.c_int32)]
    L.ck_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_double]
    L.ck_cancel.argtypes = [C.c_void_p, C.c_uint64]
    L.ck_release.argtypes = [C.c_void_p, C.c_uint64]
    L.ck_server_stats.argtypes = [C.c_void_p, C.POINTER(ServerInfo)]
    L.ck_server_destroy.argtypes = [C.c_void_p]
    L.ck_device_errors.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]
    L.ck_probe_fp64.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.ck_status_str.restype = C.c_char_p
    L.ck_last_error.restype = C.c_char_p
    L.ck_version.restype = C.c_char_p


_bind()


def library_path() -> str:
    return _lib._name


def _check(rc: int, what: str):
    if rc != 0:
        msg = _lib.ck_last_error().decode()
        raise CKError(f"{what}: {_lib.ck_status_str(rc).decode()} ({rc}): {msg}")


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream, *arrays):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for a in arrays:
        if a is not None and hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _check_dtype(a, kind, name):
    if a is None:
        return
    dt = a.dtype
    ok = (str(dt) in ("torch.float64", "float64")) if kind == "f8" else (str(dt) in ("torch.int32", "int32"))
    if not ok:
        raise TypeError(f"{name} must be {'float64' if kind == 'f8' else 'int32'}, got {dt}")


class Mechanism:
    """A mechanism loaded on the current CUDA device (see ck_load_mechanism).

    reactor 0: constant pressure (the per-reactor parameter p of every call is
    the pressure, Pa); 1: constant volume (p is the fixed density, kg/m^3).
    Reactions with rev == 2 take explicit reverse Arrhenius coefficients from
    m["arrh_rev"] [R, 3]."""

    def __init__(self, m: dict, check_atoms: bool = True, reactor: int = 0):
        S = int(np.asarray(m["mw"]).shape[0])
        R = int(np.asarray(m["reac"]).shape[0])
        keep = dict(
            mw=np.ascontiguousarray(m["mw"], np.float64),
            nasa=np.ascontiguousarray(m["nasa"], np.float64),
            tmid=np.ascontiguousarray(m["tmid"], np.float64),
            reac=np.ascontiguousarray(m["reac"], np.int32),
            prod=np.ascontiguousarray(m["prod"], np.int32),
            arrh=np.ascontiguousarray(m["arrh"], np.float64),
            rtype=np.ascontiguousarray(m["rtype"], np.int32),
            rev=np.ascontiguousarray(m["rev"], np.int32),
            arrh0=np.ascontiguousarray(m["arrh0"], np.float64),
            eff_ptr=np.ascontiguousarray(m["eff_ptr"], np.int32),
            eff_sp=np.ascontiguousarray(m["eff_sp"], np.int32),
            eff_val=np.ascontiguousarray(m["eff_val"], np.float64),
        )
        if "arrh_rev" in m:
            keep["arrh_rev"] = np.ascontiguousarray(m["arrh_rev"], np.float64)
        n_el = 0
        if check_atoms and "elem" in m:
            keep["elem"] = np.ascontiguousarray(m["elem"], np.int32)
            n_el = keep["elem"].shape[1]
        self._keep = keep
        d = MechDesc()
        d.n_species, d.n_reactions = S, R
        for f, k in (("mw", "mw"), ("nasa", "nasa"), ("t_mid", "tmid"), ("reac", "reac"), ("prod", "prod"),
                     ("arrh", "arrh"), ("rtype", "rtype"), ("reversible", "rev"), ("arrh0", "arrh0"),
                     ("eff_ptr", "eff_ptr"), ("eff_sp", "eff_sp"), ("eff_val", "eff_val")):
            setattr(d, f, keep[k].ctypes.data if keep[k].size else None)
        d.n_elements = n_el
        d.elem_count = keep["elem"].ctypes.data if n_el else None
        d.elem_mass = None
        d.arrh_rev = keep["arrh_rev"].ctypes.data if "arrh_rev" in keep and keep["arrh_rev"].size else None
        d.reactor = int(reactor)
        h = C.c_void_p()
        _check(_lib.ck_load_mechanism(C.byref(d), C.byref(h)), "ck_load_mechanism")
        self.h = h
        self.S, self.R, self.n = S, R, S + 1
        self.reactor = int(reactor)

    def close(self):
        if getattr(self, "h", None):
            _lib.ck_free_mechanism(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_mechanism(m: dict, check_atoms: bool = True, reactor: int = 0) -> Mechanism:
    return Mechanism(m, check_atoms, reactor)


def rhs(mech: Mechanism, p, y, out, stream=None):
    """dydt = f(y) for every reactor (ck_rhs)."""
    for a, nm in ((p, "p"), (y, "y"), (out, "out")):
        _check_dtype(a, "f8", nm)
    n = y.shape[0]
    _check(_lib.ck_rhs(mech.h, n, _ptr(p), _ptr(y), _ptr(out), _stream(stream, y)), "ck_rhs")
    return out


def jacobian(mech: Mechanism, p, y, out, stream=None):
    """Analytic Jacobians [n, S+1, S+1] (ck_jacobian)."""
    n = y.shape[0]
    _check(_lib.ck_jacobian(mech.h, n, _ptr(p), _ptr(y), _ptr(out), _stream(stream, y)), "ck_jacobian")
    return out


def jacobian_fd(mech: Mechanism, p, y, h, out, rtol=1e-9, atol=1e-12, stream=None):
    """Forward-difference Jacobians [n, S+1, S+1] at step sizes h[n] (ck_jacobian_fd)."""
    n = y.shape[0]
    _check(_lib.ck_jacobian_fd(mech.h, n, _ptr(p), _ptr(y), _ptr(h), float(rtol), float(atol), _ptr(out),
                               _stream(stream, y)), "ck_jacobian_fd")
    return out


def lu_factor(a, piv, info, stream=None):
    batch, dim = a.shape[0], a.shape[1]
    _check(_lib.ck_lu_factor(batch, dim, _ptr(a), _ptr(piv), _ptr(info), _stream(stream, a)), "ck_lu_factor")


def lu_solve(lu, piv, b, stream=None):
    batch, dim = lu.shape[0], lu.shape[1]
    _check(_lib.ck_lu_solve(batch, dim, _ptr(lu), _ptr(piv), _ptr(b), _stream(stream, lu)), "ck_lu_solve")


def _integrate(fn, name, mech, p, y, dt, status, h_inout=None, steps=None, opts=None, stream=None):
    _check_dtype(y, "f8", "y")
    _check_dtype(status, "i4", "status")
    n = y.shape[0]
    o = opts if opts is not None else SolverOpts.make()
    _check(fn(mech.h, n, _ptr(p), _ptr(y), _ptr(dt), _ptr(h_inout), C.byref(o), _ptr(steps), _ptr(status),
              _stream(stream, y)), name)


def integrate_ros4(mech, p, y, dt, status, h_inout=None, steps=None, opts=None, stream=None):
    """ROS4 over [0, dt] for every reactor, in place on y (ck_integrate_ros4)."""
    _integrate(_lib.ck_integrate_ros4, "ck_integrate_ros4", mech, p, y, dt, status, h_inout, steps, opts, stream)


def integrate_rkf45(mech, p, y, dt, status, h_inout=None, steps=None, opts=None, stream=None):
    """RKF45 over [0, dt] for every reactor, in place on y (ck_integrate_rkf45)."""
    _integrate(_lib.ck_integrate_rkf45, "ck_integrate_rkf45", mech, p, y, dt, status, h_inout, steps, opts,
               stream)


def integrate_ros4_noalloc(mech, p, y, dt, status, h_inout=None, steps=None, opts=None, stream=None):
    """ROS4 without any device allocation (ck_integrate_ros4_noalloc): device
    tensors only; calls on one device must not overlap on the GPU."""
    _integrate(_lib.ck_integrate_ros4_noalloc, "ck_integrate_ros4_noalloc", mech, p, y, dt, status, h_inout,
               steps, opts, stream)


GROUPS_GRAPH, GROUPS_SEQUENTIAL = 1, 2


def integrate_groups(method, groups, use_graph=True, stream=None, sequential=False):
    """Integrate several (mech, p, y, dt, status, steps, opts, weight) groups in
    one call (ck_integrate_groups); device tensors only.  sequential: one
    group after another on the stream instead of side by side."""
    arr = (Group * len(groups))()
    keep = []
    first = None
    for g, spec in zip(arr, groups):
        mech, p, y, dt, status = spec["mech"], spec["p"], spec["y"], spec["dt"], spec["status"]
        first = first if first is not None else y
        g.mech = mech.h
        g.n = y.shape[0]
        g.p, g.y, g.dt, g.status = _ptr(p), _ptr(y), _ptr(dt), _ptr(status)
        g.h_inout = _ptr(spec.get("h_inout"))
        g.steps = _ptr(spec.get("steps"))
        g.opts = spec.get("opts") or SolverOpts.make()
        g.work_weight = float(spec.get("weight", 0.0))
        keep.append(spec)
    flags = (GROUPS_GRAPH if use_graph else 0) | (GROUPS_SEQUENTIAL if sequential else 0)
    _check(_lib.ck_integrate_groups(int(method), len(groups), arr, flags, _stream(stream, first)),
           "ck_integrate_groups")


def graph_cache_clear():
    _check(_lib.ck_graph_cache_clear(), "ck_graph_cache_clear")


class Server:
    """Request server with continuous batching (ck_server_*).  Arrays passed
    to submit() must stay alive until the request is done."""

    ROS4, RKF45 = 0, 1

    def __init__(self, hbm_budget_bytes: int, streams: int = 4, chunk_reactors: int = 0):
        h = C.c_void_p()
        _check(_lib.ck_server_create(int(hbm_budget_bytes), int(streams), int(chunk_reactors), C.byref(h)),
               "ck_server_create")
        self.h = h
        self._keep = {}

    def submit(self, mech, method, p, y, dt, status, steps=None, opts=None) -> int:
        t = C.c_uint64()
        o = opts if opts is not None else SolverOpts.make()
        _check(_lib.ck_submit(self.h, mech.h, int(method), y.shape[0], _ptr(p), _ptr(y), _ptr(dt), C.byref(o),
                              _ptr(status), _ptr(steps), C.byref(t)), "ck_submit")
        self._keep[t.value] = (p, y, dt, status, steps, o)
        return t.value

    def poll(self, ticket) -> int:
        st = C.c_int32()
        _check(_lib.ck_poll(self.h, int(ticket), C.byref(st)), "ck_poll")
        return st.value

    def wait(self, ticket, timeout_s=600.0):
        _check(_lib.ck_wait(self.h, int(ticket), float(timeout_s)), "ck_wait")

    def cancel(self, ticket):
        _check(_lib.ck_cancel(self.h, int(ticket)), "ck_cancel")

    def release(self, ticket):
        _check(_lib.ck_release(self.h, int(ticket)), "ck_release")
        self._keep.pop(int(ticket), None)

    def stats(self) -> dict:
        i = ServerInfo()
        _check(_lib.ck_server_stats(self.h, C.byref(i)), "ck_server_stats")
        return {k: getattr(i, k) for k, _ in ServerInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib.ck_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count_work(mech: Mechanism) -> dict:
    w = WorkCounts()
    _check(_lib.ck_count_work(mech.h, C.byref(w)), "ck_count_work")
    return {k: getattr(w, k) for k, _ in WorkCounts._fields_}


def probe_fp64(mech: Mechanism, kind: int, iters: int) -> tuple[float, float]:
    """(seconds, ops) of an FP64 throughput probe (ck_probe_fp64): kind 0
    FMA flops, kind 1 the library's 2^x evaluations."""
    sec, ops = C.c_double(), C.c_double()
    _check(_lib.ck_probe_fp64(mech.h, int(kind), int(iters), C.byref(sec), C.byref(ops)), "ck_probe_fp64")
    return sec.value, ops.value


def fp64_peaks(mech: Mechanism, iters: int = 10000) -> dict:
    """Measured FP64 FMA throughput (flop/s) and the cost of one 2^x in
    flops of FMA-pipe time (w_exp): the roofline denominators."""
    t_f, f = probe_fp64(mech, 0, iters)
    t_e, e = probe_fp64(mech, 1, iters // 2)
    peak = f / t_f
    w_exp = peak * t_e / e - 2.0  # the probe loop's 2 adds per exponential are not the exponential's
    return {"fp64_flops_per_s": peak, "exp2_per_s": e / t_e, "w_exp": w_exp, "dfma_s": t_f, "exp2_s": t_e}


def device_errors(mech: Mechanism, reset: bool = False) -> int:
    bits = C.c_int32()
    _check(_lib.ck_device_errors(mech.h, C.byref(bits), int(reset)), "ck_device_errors")
    return bits.value


def version() -> str:
    return _lib.ck_version().decode()
