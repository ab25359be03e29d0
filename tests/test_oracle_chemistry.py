"""Pins of the oracle's source terms, Jacobian and linear algebra.

Each check is something the physics or the mathematics fixes independently
of the oracle's code:
* mass, element and (constant-pressure) energy conservation of Eqs. ydot,
  tdot, wdot for atom-balanced reactions;
* the closed-form special case of the NASA-7 fits (Eq. tfits) for a
  constant heat capacity, and continuity of the shaped fits at T_mid;
* the Lindemann limits of c_i (k_inf at high [M], k0 [M] at low [M]);
* detailed balance: a state integrated to equilibrium has every reversible
  rate of progress vanish relative to its forward rate, which only holds if
  every K_c (Eqs. kc, krev) is consistent with one set of species potentials;
* the analytic Jacobian against complex-step and central-difference
  derivatives of the right-hand side;
* LU with partial pivoting against LAPACK;
* the closed-form A -> B -> C solution through both integrators;
* the rate coefficients themselves (Eqs. kfor, kc, krev and the Lindemann
  k0) on a hand-built mechanism whose parameters make them round numbers at
  two temperatures.
"""
import numpy as np
import pytest

import synth
from synth.configs import CONFIGS, load_mechanism
from synth.handmade import T_PIN, const_cp_species, cyclic_network, linear_chain, rate_pins
from oracle import ORA_RKF45, ORA_ROS4, OracleMech

R_GAS = 8.314462618
MECHS = ["small", "medium", "large"]


@pytest.fixture(scope="module", params=MECHS)
def mech_case(request):
    cfg = CONFIGS[request.param]
    m = load_mechanism(cfg["mech"])
    om = OracleMech(m)
    rng = np.random.default_rng(11)
    y, p = synth.draw_states(rng, m["names"], m["elem"], m["mw"], m["elements"], 6,
                             cfg["t_range"], cfg["p_range_atm"])
    return request.param, m, om, y, p


def test_mass_and_element_conservation(mech_case):
    name, m, om, y, p = mech_case
    for i in range(len(p)):
        wdot, q, gross = om.rhs_detail(p[i], y[i])
        gw = gross[1:] / m["mw"]  # gross molar rates (times 1/rho)
        # sum_k wdot_k W_k = 0 and sum_k a_ek wdot_k = 0
        scale = np.sum(np.abs(wdot) * m["mw"]) + 1e-300
        assert abs(np.sum(wdot * m["mw"])) <= 1e-13 * scale
        for e in range(m["elem"].shape[1]):
            sc = np.sum(np.abs(wdot) * m["elem"][:, e]) + 1e-300
            assert abs(np.sum(wdot * m["elem"][:, e])) <= 1e-13 * sc
        f = om.rhs(p[i], y[i])[0]
        assert abs(np.sum(f[1:])) <= 1e-13 * np.sum(np.abs(f[1:]))
        assert np.all(gw >= 0)


def test_constant_pressure_energy(mech_case):
    # dh/dt = sum_k Ydot_k H_k / W_k + cp Tdot = 0 at constant p
    name, m, om, y, p = mech_case
    for i in range(len(p)):
        T = y[i, 0]
        f = om.rhs(p[i], y[i])[0]
        cp_R, h_RT, _ = om.thermo(T)
        H = R_GAS * T * h_RT
        cp = np.sum(y[i, 1:] * R_GAS * cp_R / m["mw"])
        terms = np.concatenate([f[1:] * H / m["mw"], [cp * f[0]]])
        assert abs(terms.sum()) <= 1e-12 * np.abs(terms).sum()


def test_thermo_constant_cp_closed_form():
    om = OracleMech(const_cp_species(a1=4.0, a6=-2500.0, a7=12.0))
    for T in (300.0, 999.0, 1000.0, 2500.0):
        cp_R, h_RT, s_R = om.thermo(T)
        assert cp_R[0] == pytest.approx(4.0, rel=1e-15)
        assert h_RT[0] * T == pytest.approx(4.0 * T - 2500.0, rel=1e-14)
        assert s_R[0] == pytest.approx(4.0 * np.log(T) + 12.0, rel=1e-14)


def test_thermo_continuous_at_tmid(mech_case):
    name, m, om, y, p = mech_case
    T = float(m["tmid"][0])
    a = om.thermo(T * (1 - 1e-12))
    b = om.thermo(T)
    for u, v in zip(a, b):
        assert np.allclose(u, v, rtol=1e-9, atol=1e-9)


def test_cp_bounds(mech_case):
    name, m, om, y, p = mech_case
    atoms = m["elem"].sum(axis=1)
    for T in np.linspace(300, 3500, 17):
        cp_R = om.thermo(T)[0]
        assert np.all(cp_R >= 2.5 - 1e-9) and np.all(cp_R <= 3 * atoms + 3 + 1e-9)


def test_lindemann_limits():
    m = load_mechanism(CONFIGS["medium"]["mech"])
    om = OracleMech(m)
    i = int(np.flatnonzero(m["rtype"] == 2)[0])
    T = 1500.0
    kf, kc, kr, k0 = om.rate_coeffs(T)
    S = len(m["mw"])
    y = np.concatenate([[T], np.full(S, 1.0 / S)])
    eff = np.ones(S)
    for e in range(m["eff_ptr"][i], m["eff_ptr"][i + 1]):
        eff[m["eff_sp"][e]] = m["eff_val"][e]

    def parts(p):
        wdot, q, g = om.rhs_detail(p, y)
        rho = p * (1.0 / np.sum(y[1:] / m["mw"])) / (R_GAS * T)
        X = rho * y[1:] / m["mw"]
        fwd = np.prod([X[s] for s in m["reac"][i] if s >= 0])
        rev = np.prod([X[s] for s in m["prod"][i] if s >= 0])
        return q[i], fwd, rev, np.sum(eff * X)

    # high pressure: c -> 1, q -> k_inf (fwd - rev / Kc)
    q, fwd, rev, M = parts(1e13)
    qinf = kf[i] * fwd - kr[i] * rev
    assert q == pytest.approx(qinf, rel=1e-6 + 10 * kf[i] / (k0[i] * M))
    # low pressure: c -> P_r = k0 [M] / k_inf
    q, fwd, rev, M = parts(1e-6)
    q0 = (k0[i] * M / kf[i]) * (kf[i] * fwd - kr[i] * rev)
    assert q == pytest.approx(q0, rel=1e-6 + 10 * k0[i] * M / kf[i])


def test_detailed_balance_at_equilibrium():
    m = cyclic_network()
    om = OracleMech(m)
    y = np.array([[1500.0, 0.7, 0.1, 0.2, 0.0], [1200.0, 0.0, 0.0, 0.0, 1.0],
                  [1800.0, 0.25, 0.25, 0.25, 0.25]])
    p = np.array([101325.0, 3 * 101325.0, 0.5 * 101325.0])
    ye, steps, st, _ = om.integrate(ORA_ROS4, p, y, 1.0, rtol=1e-11, atol=1e-16, max_steps=1000000)
    assert np.all(st == 0)
    worst = 0.0
    for i in range(len(p)):
        T = ye[i, 0]
        rho = p[i] * (1.0 / np.sum(ye[i, 1:] / m["mw"])) / (R_GAS * T)
        X = rho * ye[i, 1:] / m["mw"]
        kf, kc, kr, k0 = om.rate_coeffs(T)
        for r in range(len(kf)):
            fwd = kf[r] * np.prod([X[s] for s in m["reac"][r] if s >= 0])
            rev = kr[r] * np.prod([X[s] for s in m["prod"][r] if s >= 0])
            worst = max(worst, abs(fwd - rev) / (fwd + rev))
    # every reaction balances on its own (the cycle A->B->C->A carries no flux)
    assert worst < 1e-6
    # and the equilibrium constants of the cycle are mutually consistent
    kf, kc, kr, k0 = om.rate_coeffs(1500.0)
    assert kc[0] * kc[1] == pytest.approx(kc[2], rel=1e-13)


def _complex_step_jac(om, p, y):
    n = len(y)
    J = np.zeros((n, n))
    for j in range(n):
        h = 1e-30 * max(abs(y[j]), 1.0)
        yc = y.astype(np.complex128)
        yc[j] += 1j * h
        J[:, j] = om.rhs_complex(p, yc).imag / h
    return J


def test_jacobian_complex_step(mech_case):
    name, m, om, y, p = mech_case
    for i in range(3):
        J, G = om.jacobian(p[i], y[i], gross=True)
        Jc = _complex_step_jac(om, p[i], y[i])
        err = np.abs(J[0] - Jc)
        assert np.all(err <= 1e-10 * G[0] + 1e-20), (name, err.max(), np.unravel_index(np.argmax(err / (G[0] + 1e-300)), err.shape))


def test_jacobian_central_difference():
    cfg = CONFIGS["small"]
    m = load_mechanism(cfg["mech"])
    om = OracleMech(m)
    y, p = synth.configs.reactor_states("small", n=2)
    for i in range(2):
        J, G = om.jacobian(p[i], y[i], gross=True)
        n = len(y[i])
        Jfd = np.zeros((n, n))
        for j in range(n):
            h = 1e-6 * max(abs(y[i, j]), 1e-3)
            yp = y[i].copy(); yp[j] += h
            ym = y[i].copy(); ym[j] -= h
            Jfd[:, j] = (om.rhs(p[i], yp)[0] - om.rhs(p[i], ym)[0]) / (2 * h)
        assert np.all(np.abs(J[0] - Jfd) <= 1e-5 * G[0] + 1e-10)


def test_lu_matches_lapack(oracle_lib):
    rng = np.random.default_rng(2)
    for n in (1, 2, 5, 11, 54):
        for kind in ("random", "diagdom"):
            A = rng.standard_normal((n, n))
            if kind == "diagdom":
                A += np.diag(np.abs(A).sum(axis=1) + 1.0)
            b = rng.standard_normal(n)
            lu, piv, info = oracle_lib.lu_factor(A)
            assert info == 0
            x = oracle_lib.lu_solve(lu, piv, b)
            xr = np.linalg.solve(A, b)
            assert np.allclose(x, xr, rtol=1e-11, atol=1e-11 * np.abs(xr).max())
    # pivoting is required: zero leading entry
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    lu, piv, info = oracle_lib.lu_factor(A)
    assert info == 0 and piv[0] == 2
    x = oracle_lib.lu_solve(lu, piv, [1.0, 2.0, 3.0])
    assert np.allclose(A @ x, [1.0, 2.0, 3.0], atol=1e-14)
    # exactly singular
    lu, piv, info = oracle_lib.lu_factor(np.array([[1.0, 2.0], [2.0, 4.0]]))
    assert info == 2


@pytest.mark.parametrize("method", [ORA_ROS4, ORA_RKF45])
@pytest.mark.parametrize("k1,k2", [(1e2, 1e4), (3e3, 3e3 * (1 + 1e-9)), (1e4, 1e2)])
def test_linear_chain_closed_form(method, k1, k2):
    om = OracleMech(linear_chain(k1, k2))
    t = 1e-3
    y0 = np.array([[1000.0, 1.0, 0.0, 0.0]])
    y, steps, st, _ = om.integrate(method, 101325.0, y0, t, rtol=1e-9, atol=1e-12)
    assert st[0] == 0
    ya = np.exp(-k1 * t)
    if abs(k2 - k1) < 1e-6 * k1:
        yb = k1 * t * np.exp(-k1 * t)
    else:
        yb = k1 / (k2 - k1) * (np.exp(-k1 * t) - np.exp(-k2 * t))
    exact = np.array([1000.0, ya, yb, 1.0 - ya - yb])
    assert abs(y[0, 0] - 1000.0) <= 1e-9
    assert np.max(np.abs(y[0, 1:] - exact[1:])) <= 1e-8
    assert abs(np.sum(y[0, 1:]) - 1.0) <= 1e-12


def test_integrated_enthalpy_and_mass(mech_case):
    name, m, om, y, p = mech_case
    cfg = CONFIGS[name]
    ye, steps, st, _ = om.integrate(ORA_RKF45, p[:2], y[:2], cfg["dt"])
    assert np.all(st == 0)
    for i in range(2):
        def hmix(v):
            cp_R, h_RT, _ = om.thermo(v[0])
            return np.sum(v[1:] * R_GAS * v[0] * h_RT / m["mw"]), np.sum(np.abs(v[1:] * R_GAS * v[0] * h_RT / m["mw"]))
        h0, s0 = hmix(y[i])
        h1, s1 = hmix(ye[i])
        assert abs(h1 - h0) <= 1e-7 * max(s0, s1)
        assert abs(ye[i, 1:].sum() - 1.0) <= 1e-10


def test_rate_coefficients_closed_forms():
    # rate_pins() places round values at T0 and 2 T0 (derived by hand from the
    # parameters): a wrong sign of E or of the Gibbs terms, a dropped beta,
    # p0/RT inverted or the wrong dnu would each move one of them
    om = OracleMech(rate_pins())
    T0 = T_PIN
    p0 = 101325.0
    for T, kf0, kc0, k0 in ((T0, T0, 6.0, 10.0 / (4.0 * T0)),
                             (2 * T0, 2.0 * np.sqrt(2.0) * T0, 3.0 * np.sqrt(2.0), 10.0 / (4.0 * T0))):
        kf, kc, kr, k0s = om.rate_coeffs(T)
        r = R_GAS * T / p0
        expect_kf = [kf0, 50.0, 1000.0]
        expect_kc = [kc0, 5.0 * r, (5.0 / 3.0) * 2.0 ** (-T0 / T) * r]
        assert kf == pytest.approx(expect_kf, rel=1e-14)
        assert kc == pytest.approx(expect_kc, rel=1e-13)
        assert kr == pytest.approx(np.array(expect_kf) / np.array(expect_kc), rel=1e-13)
        assert k0s[2] == pytest.approx(k0, rel=1e-14) and k0s[0] == 0.0 and k0s[1] == 0.0
