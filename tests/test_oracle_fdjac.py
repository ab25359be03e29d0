"""Pins of the oracle's forward-difference ROS4 variant (Sec. 5: first-order
forward differences following CVODE, S+1 right-hand sides per Jacobian).

* Increments.  On the scalar y' = -y^2 a forward difference with increment s
  gives -(2y + s) exactly up to rounding, so s can be read back from the
  oracle's result.  CVODE's dense difference quotient fixes three cases:
  - s = 2^-26 |y| (the relative branch) at y = 1;
  - s = atol at y = 0, where f = 0 and the floor is 1/w;
  - s = 1000 h 2^-52 |f| for a long step (the floor branch; with n = 1 the
    weight cancels), and n times that for n equal uncoupled copies.
* Structure.  On a dense linear system f = A y the differences are exact, so
  J_fd = A to rounding.  This catches transposed or misplaced columns and a
  wrong sign.
* Accuracy.  On the three mechanisms J_fd differs from the analytic
  Jacobian (pinned by complex steps) by no more than the forward-difference
  error bound s_j/2 |d2 f_i/dy_j2| + 2 eps_f_i / s_j.
* Cost.  A ROS4 step with differences costs S+1 more right-hand sides than
  with the analytic Jacobian: n + 4 a step against 4 (stage 4 is evaluated
  literally here).
* Result.  ROS4 with either Jacobian reaches the same state within the
  tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import ORA_ROS4, OracleMech
from synth.configs import CONFIGS, load_mechanism

U = 2.0 ** -52


def test_increment_relative_branch(oracle_lib):
    J = oracle_lib.test_jacobian_fd(1, [], [1.0], h=1e-3, rtol=1e-6, atol=1e-10)
    s = -(J[0, 0] + 2.0)
    assert abs(s - 2.0 ** -26) <= 1e-6 * 2.0 ** -26


def test_increment_zero_rhs_branch(oracle_lib):
    for atol in (1e-10, 1e-6):
        J = oracle_lib.test_jacobian_fd(1, [], [0.0], h=1e-3, rtol=1e-6, atol=atol)
        assert -J[0, 0] == pytest.approx(atol, rel=1e-12)


def test_increment_floor_branch(oracle_lib):
    y, h = 1e-3, 1e9          # |f| = 1e-6; floor 1000 h U |f| = 2.2e-10 > 2^-26 y = 1.5e-11
    J = oracle_lib.test_jacobian_fd(1, [], [y], h=h, rtol=1e-6, atol=1e-10)
    s = -(J[0, 0] + 2.0 * y)
    assert s == pytest.approx(1000.0 * h * U * y * y, rel=1e-5)


def test_increment_floor_scales_with_dimension(oracle_lib):
    # n uncoupled copies of y' = -y^2 at equal y: fnorm = |f| w, so the floor
    # is 1000 h U n |f| on every diagonal and the off-diagonals are exactly 0
    y, h = 1e-3, 1e9
    for n in (2, 5):
        J = oracle_lib.test_jacobian_fd(3, [], [y] * n, h=h, rtol=1e-6, atol=1e-10)
        s = -(np.diag(J) + 2.0 * y)
        assert np.allclose(s, 1000.0 * h * U * n * y * y, rtol=1e-5)
        assert np.all(J[~np.eye(n, dtype=bool)] == 0.0)


def test_linear_system_exact(oracle_lib):
    rng = np.random.default_rng(5)
    for n in (1, 3, 8):
        A = rng.normal(size=(n, n)) * 10.0 ** rng.uniform(-2, 2, size=(n, n))
        y = rng.normal(size=n)
        J = oracle_lib.test_jacobian_fd(2, A, y, h=1e-4, rtol=1e-8, atol=1e-12)
        # rounding of f(y + s e_j) - f(y) over s: a few eps |A||y| / s
        s = np.maximum(2.0 ** -26 * np.abs(y), 1e-12)
        bound = 8 * U * (np.abs(A) @ np.abs(y))[:, None] / s[None, :] + 1e-12 * np.abs(A)
        assert np.all(np.abs(J - A) <= bound), np.abs(J - A).max()


def _second_derivatives(om, p, y):
    """d2 f_i / dy_j2 by central differences of the analytic Jacobian."""
    n = len(y)
    D = np.zeros((n, n))
    for j in range(n):
        d = 1e-5 * max(abs(y[j]), 1e-6)
        yp = y.copy(); yp[j] += d
        ym = y.copy(); ym[j] -= d
        D[:, j] = (om.jacobian(p, yp)[0][:, j] - om.jacobian(p, ym)[0][:, j]) / (2 * d)
    return D


@pytest.mark.parametrize("name", ["small", "medium", "large"])
def test_fd_matches_analytic_within_difference_bound(name):
    cfg = CONFIGS[name]
    m = load_mechanism(cfg["mech"])
    om = OracleMech(m)
    rng = np.random.default_rng(17)
    y, p = synth.draw_states(rng, m["names"], m["elem"], m["mw"], m["elements"], 2, cfg["t_range"],
                             cfg["p_range_atm"])
    rtol, atol, h = 1e-9, 1e-12, 1e-7
    for i in range(len(p)):
        J, G = om.jacobian(p[i], y[i], gross=True)
        Jf = om.jacobian_fd(p[i], y[i], h, rtol=rtol, atol=atol)[0]
        f0 = om.rhs(p[i], y[i])[0]
        n = len(f0)
        w = 1.0 / (atol + rtol * np.abs(y[i]))
        fn = np.sqrt(np.mean((f0 * w) ** 2))
        s = np.maximum(2.0 ** -26 * np.abs(y[i]), 1000.0 * h * U * n * fn / w)
        gross_f = om.rhs_gross(p[i], y[i])[0]
        D2 = _second_derivatives(om, p[i], y[i])
        bound = 0.5 * s[None, :] * np.abs(D2) + 64 * U * gross_f[:, None] / s[None, :]
        err = np.abs(Jf - J[0])
        ok = err <= 4 * bound + 1e-10 * G[0] + 1e-30
        assert ok.all(), (name, np.argwhere(~ok)[:5], (err / (bound + 1e-300)).max())


@pytest.mark.parametrize("name", ["small", "medium"])
def test_rhs_evaluations_per_step(name):
    cfg = CONFIGS[name]
    m = load_mechanism(cfg["mech"])
    om = OracleMech(m)
    y, p = synth.configs.reactor_states(name, n=3)
    per = {}
    for jac in (0, 1):
        om.o.rhs_evals(reset=True)
        _, steps, st, _ = om.integrate(ORA_ROS4, p, y, cfg["dt"], h0=cfg["dt"] / 50, jac=jac)
        ev = om.o.rhs_evals(reset=True)
        assert (st == 0).all()
        per[jac] = ev / steps.sum()
    n = om.n
    assert per[0] == 4.0
    assert per[1] == n + 4.0
    assert per[1] - per[0] == m["nasa"].shape[0] + 1  # S+1 (Sec. 5)


@pytest.mark.parametrize("name", ["small", "medium"])
def test_fd_and_analytic_ros4_agree(name):
    cfg = CONFIGS[name]
    m = load_mechanism(cfg["mech"])
    om = OracleMech(m)
    y, p = synth.configs.reactor_states(name, n=4)
    rtol, atol = 1e-9, 1e-12
    ya, _, sa, _ = om.integrate(ORA_ROS4, p, y, cfg["dt"], rtol=rtol, atol=atol)
    yf, _, sf, _ = om.integrate(ORA_ROS4, p, y, cfg["dt"], rtol=rtol, atol=atol, jac=1)
    assert (sa == 0).all() and (sf == 0).all()
    # both are within the tolerance of the exact solution: a few hundred rtol apart at most
    assert np.all(np.abs(ya - yf) <= 1e3 * (rtol * np.abs(ya) + atol))
