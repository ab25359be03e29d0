"""Pins of the oracle's integrators against facts the mathematics fixes.

* RKF45 (App. B): one step on y' = lam y equals the exact stability
  polynomial of the printed tableau, R(z) = 1 + sum_k z^(k+1) b^T A^k 1, whose
  coefficients are 1, 1, 1/2, 1/6, 1/24, 1/104 (order 4 for the propagated b)
  and whose fifth-order twin has 1/120 (order 5 for bh); the fixed-step global
  error has slope 4.
* ROS4 (Sec. 2 transformed form, App. C): one step on y' = lam y differs from
  e^z by O(z^5) (order 4), the embedded solution ynew + err by O(z^4)
  (order 3), |R(-inf)| is tiny (L-stability), and the fixed-step global error
  on the nonlinear y' = -y^2 has slope 4.
"""
from fractions import Fraction
import math
import os

import numpy as np
import pytest

from oracle import ORA_RKF45, ORA_ROS4

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rkf45_table():
    A = [[Fraction(0)] * 6 for _ in range(6)]
    b = bh = None
    for line in open(os.path.join(GOLD, "rkf45_tableau.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        head, vals = line.split(":")
        vals = [Fraction(v) for v in vals.split()]
        if head.startswith("a "):
            i = int(head.split()[1]) - 1
            for j, v in enumerate(vals):
                A[i][j] = v
        elif head == "b":
            b = vals
        elif head == "bh":
            bh = vals
    return A, b, bh


def _stability_coeffs(A, w):
    """Coefficients of R(z) = 1 + sum_k z^(k+1) w^T A^k 1 (A strictly lower)."""
    n = len(w)
    v = [Fraction(1)] * n
    out = [Fraction(1)]
    for _ in range(n):
        out.append(sum(w[i] * v[i] for i in range(n)))
        v = [sum(A[i][j] * v[j] for j in range(n)) for i in range(n)]
    return out


def test_rkf45_stability_polynomial_exact(oracle_lib):
    A, b, bh = _rkf45_table()
    cb = _stability_coeffs(A, b)
    cbh = _stability_coeffs(A, bh)
    # order conditions for y' = lam y: 1/k! up to the order
    assert cb[:5] == [Fraction(1, math.factorial(k)) for k in range(5)]
    assert cb[5] == Fraction(1, 104)  # not 1/120: b is fourth order
    assert cbh[:6] == [Fraction(1, math.factorial(k)) for k in range(6)]
    for z in (-0.9, -0.3, 0.2, -2.5, -3.0):
        ynew, err = oracle_lib.test_onestep(0, ORA_RKF45, [z], [1.0], 1.0)
        R = sum(float(c) * z ** k for k, c in enumerate(cb))
        Rh = sum(float(c) * z ** k for k, c in enumerate(cbh))
        scale = sum(abs(float(c)) * abs(z) ** k for k, c in enumerate(cbh))
        assert abs(ynew[0] - R) <= 2e-15 * scale
        D = sum(float(ch - c) * z ** k for k, (c, ch) in enumerate(zip(cb + [0], cbh)))
        assert abs(err[0] - D) <= 2e-15 * scale


def _slope(hs, errs):
    return np.polyfit(np.log(hs), np.log(errs), 1)[0]


@pytest.mark.parametrize("method", [ORA_RKF45, ORA_ROS4])
def test_global_order_four_nonlinear(oracle_lib, method):
    # y' = -y^2, y(0) = 1, exact y(1) = 1/2
    errs, hs = [], []
    for N in (8, 16, 32, 64):
        y, steps, st = oracle_lib.test_integrate(1, method, [], [1.0], 1.0, fixed_h=1.0 / N)
        assert st == 0 and steps[0] == N
        errs.append(abs(y[0] - 0.5))
        hs.append(1.0 / N)
    assert abs(_slope(hs, errs) - 4.0) < 0.15


@pytest.mark.parametrize("method", [ORA_RKF45, ORA_ROS4])
def test_global_order_four_linear(oracle_lib, method):
    errs, hs = [], []
    for N in (16, 32, 64, 128):
        y, steps, st = oracle_lib.test_integrate(0, method, [-2.0], [1.0], 1.0, fixed_h=1.0 / N)
        errs.append(abs(y[0] - math.exp(-2.0)))
        hs.append(1.0 / N)
    assert abs(_slope(hs, errs) - 4.0) < 0.15


def test_ros4_local_orders(oracle_lib):
    zs = np.array([-0.02, -0.04, -0.08, -0.16])
    e_main, e_emb = [], []
    for z in zs:
        ynew, err = oracle_lib.test_onestep(0, ORA_ROS4, [z], [1.0], 1.0)
        e_main.append(abs(ynew[0] - math.exp(z)))
        e_emb.append(abs(ynew[0] + err[0] - math.exp(z)))
    # local error of an order-p method is O(z^(p+1))
    assert abs(_slope(-zs, e_main) - 5.0) < 0.2
    assert abs(_slope(-zs, e_emb) - 4.0) < 0.2


def test_ros4_gamma_table_value_satisfies_order_conditions():
    # With the table's gamma = 0.57282 the printed a, c, m reproduce e^z to
    # O(z^5); with the text's 0.572816 already the first-order term is off.
    vals = {}
    for line in open(os.path.join(GOLD, "ros4_coefficients.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)

    def R_series(g):
        # Taylor coefficients of R(z) from (1/g - z) u_i = z(1 + sum a u) + sum c u
        import sympy as sp
        z = sp.symbols("z")
        a = {(2, 1): vals["a21"], (3, 1): vals["a31"], (3, 2): vals["a32"], (4, 1): vals["a41"],
             (4, 2): vals["a42"], (4, 3): vals["a43"]}
        c = {(2, 1): vals["c21"], (3, 1): vals["c31"], (3, 2): vals["c32"], (4, 1): vals["c41"],
             (4, 2): vals["c42"], (4, 3): vals["c43"]}
        u = {}
        for i in range(1, 5):
            num = z * (1 + sum(a.get((i, j), 0) * u[j] for j in range(1, i))) + \
                sum(c.get((i, j), 0) * u[j] for j in range(1, i))
            u[i] = num / (1 / sp.Float(g, 20) - z)
        R = 1 + sum(vals[f"m{i}"] * u[i] for i in range(1, 5))
        ser = sp.series(R, z, 0, 5).removeO()
        return [float(ser.coeff(z, k)) for k in range(5)]

    good = R_series(0.57282)
    for k in range(5):
        assert abs(good[k] - 1.0 / math.factorial(k)) < 1e-12
    bad = R_series(0.572816)
    assert abs(bad[1] - 1.0) > 1e-7


def test_ros4_l_stable(oracle_lib):
    ynew, err = oracle_lib.test_onestep(0, ORA_ROS4, [-1e12], [1.0], 1.0)
    assert abs(ynew[0]) < 1e-4
    y, steps, st = oracle_lib.test_integrate(0, ORA_ROS4, [-1e6, -1.0], [1.0, 1.0], 1.0, fixed_h=0.05)
    assert st == 0 and abs(y[0]) < 1e-6 and abs(y[1] - math.exp(-1.0)) < 1e-5


def test_rkf45_unstable_beyond_limit(oracle_lib):
    # real-axis stability limit of the fourth-order polynomial is near -3.02
    ok, _ = oracle_lib.test_onestep(0, ORA_RKF45, [-2.9], [1.0], 1.0)
    bad, _ = oracle_lib.test_onestep(0, ORA_RKF45, [-3.2], [1.0], 1.0)
    assert abs(ok[0]) < 1.0 < abs(bad[0])


@pytest.mark.parametrize("method", [ORA_RKF45, ORA_ROS4])
def test_adaptive_driver_meets_tolerance(oracle_lib, method):
    # dense linear system with eigenvalues -1, -10, -100
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    A = Q @ np.diag([-1.0, -10.0, -100.0]) @ Q.T
    y0 = np.array([1.0, -0.5, 0.25])
    y, steps, st = oracle_lib.test_integrate(2, method, A, y0, 0.7, rtol=1e-9, atol=1e-12)
    w, V = np.linalg.eigh(A)
    exact = V @ (np.exp(w * 0.7) * (V.T @ y0))
    assert st == 0
    assert np.max(np.abs(y - exact)) < 1e-7
    assert steps[0] > 5


def test_driver_status_codes(oracle_lib):
    y, steps, st = oracle_lib.test_integrate(0, ORA_ROS4, [-1.0], [np.nan], 1.0)
    assert st == 5  # BADINPUT
    y, steps, st = oracle_lib.test_integrate(0, ORA_RKF45, [-1.0], [1.0], 1.0, max_steps=3,
                                             rtol=1e-12, atol=1e-14)
    assert st == 1 and steps.sum() == 3  # MAXSTEPS
    # y' = y^2 blows up at t = 1: the step size collapses
    y, steps, st = oracle_lib.test_integrate(1, ORA_RKF45, [], [-1.0], 2.0)
    assert st in (2, 3)  # HMIN or NONFINITE
    y, steps, st = oracle_lib.test_integrate(0, ORA_ROS4, [-1.0], [1.0], 0.0)
    assert st == 0 and steps.sum() == 0 and y[0] == 1.0
