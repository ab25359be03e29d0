"""ctypes wrapper of the C++ oracle (TEST INFRASTRUCTURE).

Builds ``oracle/_build/libck_oracle.so`` with g++ (FP64, no fast-math, no FMA
contraction so that the oracle rounds the same way on every host) and exposes
numpy-level calls.  See ``oracle_api.h`` for what each entry point computes and
which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libck_oracle.so")
_SRC = [os.path.join(_HERE, "ck_oracle.cpp")]
_HDR = os.path.join(_HERE, "oracle_api.h")

ORA_ROS4 = 0
ORA_RKF45 = 1
STATUS = {0: "OK", 1: "MAXSTEPS", 2: "HMIN", 3: "NONFINITE", 4: "SINGULAR", 5: "BADINPUT"}

_lock = threading.Lock()


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    with _lock:
        newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp] + _SRC + ["-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class _Opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double),
                ("fixed_h", C.c_double), ("max_steps", C.c_int32), ("jac", C.c_int32)]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)


class Oracle:
    """Loaded oracle library (one per process)."""

    _inst = None

    def __new__(cls):
        if cls._inst is None:
            inst = super().__new__(cls)
            inst.lib = C.CDLL(build_oracle())
            inst._bind()
            cls._inst = inst
        return cls._inst

    def _bind(self):
        L = self.lib
        L.ora_mech_create.restype = C.c_void_p
        L.ora_mech_create.argtypes = [C.c_int32, C.c_int32, _DP, _DP, _DP, _IP, _IP, _DP, _IP, _IP,
                                      _DP, _IP, _IP, _DP, _DP, C.c_int32]
        L.ora_mech_free.argtypes = [C.c_void_p]
        L.ora_thermo.argtypes = [C.c_void_p, C.c_double, _DP, _DP, _DP]
        L.ora_rate_coeffs.argtypes = [C.c_void_p, C.c_double, _DP, _DP, _DP, _DP]
        L.ora_rhs.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP]
        L.ora_rhs_detail.argtypes = [C.c_void_p, C.c_double, _DP, _DP, _DP, _DP]
        L.ora_rhs_complex.argtypes = [C.c_void_p, C.c_double, _DP, _DP, _DP, _DP]
        L.ora_jacobian.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP, _DP]
        L.ora_lu_factor.restype = C.c_int32
        L.ora_lu_factor.argtypes = [C.c_int32, _DP, _IP]
        L.ora_lu_solve.argtypes = [C.c_int32, _DP, _IP, _DP]
        L.ora_integrate.argtypes = [C.c_void_p, C.c_int32, C.c_int64, _DP, _DP, _DP, _DP,
                                    C.POINTER(_Opts), _IP, _IP, C.c_int32]
        L.ora_test_integrate.argtypes = [C.c_int32, C.c_int32, C.c_int32, _DP, _DP, C.c_double,
                                         C.POINTER(_Opts), _IP, _IP]
        L.ora_test_onestep.argtypes = [C.c_int32, C.c_int32, C.c_int32, _DP, _DP, C.c_double, _DP, _DP]
        L.ora_hardware_threads.restype = C.c_int32
        L.ora_jacobian_fd.argtypes = [C.c_void_p, C.c_int64, _DP, _DP, _DP, C.c_double, C.c_double, _DP]
        L.ora_test_jacobian_fd.argtypes = [C.c_int32, C.c_int32, _DP, _DP, C.c_double, C.c_double, C.c_double,
                                           _DP]
        L.ora_rhs_evals.restype = C.c_int64
        L.ora_rhs_evals.argtypes = [C.c_int32]

    @staticmethod
    def opts(rtol=1e-9, atol=1e-12, h0=0.0, fixed_h=0.0, max_steps=100000, jac=0):
        """jac: ROS4 Jacobian, 0 analytic (Sec. 6), 1 forward differences (Sec. 5)."""
        return _Opts(rtol, atol, h0, fixed_h, max_steps, jac)

    def rhs_evals(self, reset: bool = False) -> int:
        """Right-hand-side evaluations made by integrate() since the last reset."""
        return int(self.lib.ora_rhs_evals(1 if reset else 0))

    def hardware_threads(self) -> int:
        return int(self.lib.ora_hardware_threads())

    def lu_factor(self, a):
        a = np.array(a, dtype=np.float64, order="C", copy=True)
        n = a.shape[0]
        piv = np.zeros(n, np.int32)
        info = self.lib.ora_lu_factor(n, _p(a, C.c_double), _p(piv, C.c_int32))
        return a, piv, int(info)

    def lu_solve(self, lu, piv, b):
        b = np.array(b, dtype=np.float64, copy=True)
        lu = np.ascontiguousarray(lu, dtype=np.float64)
        piv = np.ascontiguousarray(piv, dtype=np.int32)
        self.lib.ora_lu_solve(lu.shape[0], _p(lu, C.c_double), _p(piv, C.c_int32), _p(b, C.c_double))
        return b

    def test_integrate(self, problem, method, params, y0, dt, **kw):
        params = np.ascontiguousarray(params, dtype=np.float64).ravel()
        y = np.array(y0, dtype=np.float64, copy=True).ravel()
        dim = y.size
        o = self.opts(**kw)
        steps = np.zeros(2, np.int32)
        st = np.zeros(1, np.int32)
        self.lib.ora_test_integrate(problem, method, dim, _p(params, C.c_double), _p(y, C.c_double),
                                    float(dt), C.byref(o), _p(steps, C.c_int32), _p(st, C.c_int32))
        return y, steps, int(st[0])

    def test_jacobian_fd(self, problem, params, y, h, rtol=1e-9, atol=1e-12):
        """Forward-difference Jacobian (Sec. 5) of a test problem at y, step size h."""
        params = np.ascontiguousarray(params, dtype=np.float64).ravel()
        y = np.ascontiguousarray(y, dtype=np.float64).ravel()
        J = np.zeros((y.size, y.size))
        self.lib.ora_test_jacobian_fd(problem, y.size, _p(params, C.c_double), _p(y, C.c_double), float(h),
                                      float(rtol), float(atol), _p(J, C.c_double))
        return J

    def test_onestep(self, problem, method, params, y0, h):
        params = np.ascontiguousarray(params, dtype=np.float64).ravel()
        y = np.ascontiguousarray(y0, dtype=np.float64).ravel()
        ynew = np.zeros_like(y)
        err = np.zeros_like(y)
        self.lib.ora_test_onestep(problem, method, y.size, _p(params, C.c_double), _p(y, C.c_double),
                                  float(h), _p(ynew, C.c_double), _p(err, C.c_double))
        return ynew, err


class OracleMech:
    """A mechanism (dict of numpy arrays as from ``synth.load_mechanism``)
    loaded into the oracle."""

    def __init__(self, mech: dict, reactor: int = 0):
        """reactor 0: constant pressure (the per-reactor parameter p is the
        pressure, Pa); 1: constant volume (p is the fixed density, kg/m^3).
        Reactions with rev == 2 take explicit reverse Arrhenius coefficients
        from mech["arrh_rev"] [R, 3]."""
        self.o = Oracle()
        m = mech
        self.reactor = int(reactor)
        self.S = int(m["mw"].shape[0])
        self.R = int(m["reac"].shape[0])
        self.n = self.S + 1
        self._keep = dict(
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
            arrh_rev=np.ascontiguousarray(m["arrh_rev"] if "arrh_rev" in m else np.zeros((len(m["reac"]), 3)),
                                          np.float64),
        )
        k = self._keep
        if k["eff_sp"].size == 0:
            k["eff_sp"] = np.zeros(1, np.int32)
            k["eff_val"] = np.zeros(1, np.float64)
        d, i = C.c_double, C.c_int32
        self.h = self.o.lib.ora_mech_create(
            self.S, self.R, _p(k["mw"], d), _p(k["nasa"], d), _p(k["tmid"], d), _p(k["reac"], i),
            _p(k["prod"], i), _p(k["arrh"], d), _p(k["rtype"], i), _p(k["rev"], i), _p(k["arrh0"], d),
            _p(k["eff_ptr"], i), _p(k["eff_sp"], i), _p(k["eff_val"], d),
            _p(k["arrh_rev"], d) if k["arrh_rev"].size else None, self.reactor)
        if not self.h:
            raise ValueError("oracle rejected the mechanism")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.o.lib.ora_mech_free(h)
            self.h = None

    def thermo(self, T):
        cp = np.zeros(self.S); hr = np.zeros(self.S); sr = np.zeros(self.S)
        self.o.lib.ora_thermo(self.h, float(T), _p(cp, C.c_double), _p(hr, C.c_double), _p(sr, C.c_double))
        return cp, hr, sr

    def rate_coeffs(self, T):
        kf = np.zeros(self.R); kc = np.zeros(self.R); kr = np.zeros(self.R); k0 = np.zeros(self.R)
        self.o.lib.ora_rate_coeffs(self.h, float(T), _p(kf, C.c_double), _p(kc, C.c_double),
                                   _p(kr, C.c_double), _p(k0, C.c_double))
        return kf, kc, kr, k0

    def rhs(self, p, y):
        y = np.ascontiguousarray(y, np.float64).reshape(-1, self.n)
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(p, np.float64), (y.shape[0],)))
        out = np.zeros_like(y)
        self.o.lib.ora_rhs(self.h, y.shape[0], _p(p, C.c_double), _p(y, C.c_double), _p(out, C.c_double))
        return out

    def rhs_detail(self, p, y):
        y = np.ascontiguousarray(y, np.float64).ravel()
        wdot = np.zeros(self.S); q = np.zeros(self.R); g = np.zeros(self.n)
        self.o.lib.ora_rhs_detail(self.h, float(p), _p(y, C.c_double), _p(wdot, C.c_double),
                                  _p(q, C.c_double), _p(g, C.c_double))
        return wdot, q, g

    def rhs_gross(self, p, y):
        y = np.ascontiguousarray(y, np.float64).reshape(-1, self.n)
        p = np.broadcast_to(np.asarray(p, np.float64), (y.shape[0],))
        return np.stack([self.rhs_detail(p[i], y[i])[2] for i in range(y.shape[0])])

    def rhs_complex(self, p, y):
        y = np.asarray(y, np.complex128).ravel()
        yr = np.ascontiguousarray(y.real); yi = np.ascontiguousarray(y.imag)
        fr = np.zeros(self.n); fi = np.zeros(self.n)
        self.o.lib.ora_rhs_complex(self.h, float(p), _p(yr, C.c_double), _p(yi, C.c_double),
                                   _p(fr, C.c_double), _p(fi, C.c_double))
        return fr + 1j * fi

    def jacobian(self, p, y, gross=False):
        y = np.ascontiguousarray(y, np.float64).reshape(-1, self.n)
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(p, np.float64), (y.shape[0],)))
        J = np.zeros((y.shape[0], self.n, self.n))
        G = np.zeros_like(J) if gross else None
        self.o.lib.ora_jacobian(self.h, y.shape[0], _p(p, C.c_double), _p(y, C.c_double),
                                _p(J, C.c_double), _p(G, C.c_double) if gross else None)
        return (J, G) if gross else J

    def jacobian_fd(self, p, y, h, rtol=1e-9, atol=1e-12):
        """Forward-difference Jacobians (Sec. 5) at step sizes h, as ROS4 with jac=1 builds them."""
        y = np.ascontiguousarray(y, np.float64).reshape(-1, self.n)
        nr = y.shape[0]
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(p, np.float64), (nr,)))
        h = np.ascontiguousarray(np.broadcast_to(np.asarray(h, np.float64), (nr,)))
        J = np.zeros((nr, self.n, self.n))
        self.o.lib.ora_jacobian_fd(self.h, nr, _p(p, C.c_double), _p(y, C.c_double), _p(h, C.c_double),
                                   float(rtol), float(atol), _p(J, C.c_double))
        return J

    def integrate(self, method, p, y, dt, h_inout=None, nthreads=0, **kw):
        """Integrate every reactor over [0, dt].  Returns (y, steps[n,2], status[n], h)."""
        y = np.array(y, np.float64, copy=True).reshape(-1, self.n)
        nr = y.shape[0]
        p = np.ascontiguousarray(np.broadcast_to(np.asarray(p, np.float64), (nr,)))
        dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (nr,)))
        h = None if h_inout is None else np.array(np.broadcast_to(h_inout, (nr,)), np.float64)
        steps = np.zeros((nr, 2), np.int32)
        status = np.zeros(nr, np.int32)
        o = Oracle.opts(**kw)
        self.o.lib.ora_integrate(self.h, int(method), nr, _p(p, C.c_double), _p(y, C.c_double),
                                 _p(dt, C.c_double), _p(h, C.c_double) if h is not None else None,
                                 C.byref(o), _p(steps, C.c_int32), _p(status, C.c_int32), int(nthreads))
        return y, steps, status, h
