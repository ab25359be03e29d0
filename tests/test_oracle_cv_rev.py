"""Pins of the oracle's constant-volume reactor and explicit reverse
Arrhenius coefficients (Sec. 3).

Constant volume (rho fixed; c_v for c_p and u_k for h_k in Eq. tdot):
* Energy.  A closed rigid adiabatic vessel keeps its internal energy:
  sum_k (U_k/W_k) dY_k/dt + c_v dT/dt = 0 at every state, with U_k from the
  (separately pinned) NASA-7 fits.
* Species.  The species rates equal the constant-pressure ones at the
  pressure that gives the same density, because [X] and T then coincide.
* Closed form.  In A -> B -> C with constant cp/R = a1, T-independent rates
  and heat release through the offsets a6_k, energy conservation fixes
  T(t) = T0 + sum_k (Y_k(0) - Y_k(t)) a6_k / (a1 - 1).  At constant
  pressure the same holds with a1 in place of a1 - 1.
* Jacobian.  It matches complex-step derivatives of the right-hand side.
* Integration.  Over a time step the mixture internal energy is conserved to
  the tolerance.

Explicit reverse Arrhenius (Sec. 3):
* Closed form.  For constant-cp species, K_c(T) is itself of Arrhenius form:
  - A_r = A (R/p0)^dnu e^(da1 - da7);
  - beta_r = beta + dnu - da1;
  - Ea_r = Ea - R da6.
  A mechanism given those coefficients explicitly must reproduce the K_c
  path's rates, right-hand side and Jacobian.
* Jacobian.  It matches complex-step derivatives, including on a large
  mechanism with a quarter of its reactions explicit.
"""
import numpy as np
import pytest

import synth
from oracle import ORA_ROS4, ORA_RKF45, OracleMech
from oracle.mechgen import with_explicit_reverse
from synth.configs import CONFIGS, cv_states, load_mechanism
from synth.handmade import cyclic_network, linear_chain

R_GAS = 8.314462618
P0 = 101325.0
MECHS = ["small", "medium", "large"]


def _complex_step_jac(om, p, y, step=1e-30):
    n = len(y)
    J = np.zeros((n, n))
    for j in range(n):
        h = step * max(abs(y[j]), 1.0)
        yc = y.astype(np.complex128)
        yc[j] += 1j * h
        J[:, j] = om.rhs_complex(p, yc).imag / h
    return J


def _assert_matches_complex_step(om, p, y, J, G):
    """The analytic Jacobian agrees with complex-step derivatives within the
    bar of the constant-pressure pin: 1e-10 of the gross sums."""
    Jc = _complex_step_jac(om, p, y)
    err = np.abs(J - Jc)
    ok = err <= 1e-10 * G + 1e-20
    assert ok.all(), (np.argwhere(~ok)[:5], (err / (G + 1e-300)).max())


def _u_mass(om, m, y):
    """Mixture internal energy per unit mass, and its gross magnitude."""
    cp_R, h_RT, _ = om.thermo(y[0])
    u = R_GAS * y[0] * (h_RT - 1.0) / m["mw"]
    return np.sum(y[1:] * u), np.sum(np.abs(y[1:] * u))


@pytest.mark.parametrize("name", MECHS)
def test_cv_internal_energy_balance(name):
    m = load_mechanism(CONFIGS[name]["mech"])
    om = OracleMech(m, reactor=1)
    y, rho = cv_states(name, 8)
    f = om.rhs(rho, y)
    for i in range(len(rho)):
        cp_R, h_RT, _ = om.thermo(y[i, 0])
        u = R_GAS * y[i, 0] * (h_RT - 1.0) / m["mw"]
        cv = np.sum(y[i, 1:] * R_GAS * (cp_R - 1.0) / m["mw"])
        res = np.sum(u * f[i, 1:]) + cv * f[i, 0]
        scale = np.sum(np.abs(u * f[i, 1:])) + abs(cv * f[i, 0])
        assert abs(res) <= 1e-12 * scale, (name, i, res, scale)
        assert abs(np.sum(f[i, 1:])) <= 1e-12 * np.sum(np.abs(f[i, 1:]))


@pytest.mark.parametrize("name", MECHS)
def test_cv_species_rates_equal_cp_at_same_density(name):
    m = load_mechanism(CONFIGS[name]["mech"])
    cv = OracleMech(m, reactor=1)
    cp = OracleMech(m, reactor=0)
    y, rho = cv_states(name, 8, seed_offset=1)
    Wbar = 1.0 / (y[:, 1:] / m["mw"]).sum(axis=1)
    p = rho * R_GAS * y[:, 0] / Wbar
    fv = cv.rhs(rho, y)
    fp = cp.rhs(p, y)
    g = cp.rhs_gross(p, y)
    assert np.all(np.abs(fv[:, 1:] - fp[:, 1:]) <= 1e-12 * g[:, 1:] + 1e-30)
    # the temperature rates differ: heat release goes into u at constant volume
    assert not np.allclose(fv[:, 0], fp[:, 0], rtol=1e-3)


@pytest.mark.parametrize("method", [ORA_ROS4, ORA_RKF45])
@pytest.mark.parametrize("reactor", [0, 1])
def test_linear_chain_with_heat_release_closed_form(method, reactor):
    k1, k2 = 1e3, 3e2
    a6 = np.array([-500.0, -2500.0, -7000.0])
    om = OracleMech(linear_chain(k1, k2, a6=a6), reactor=reactor)
    t = 2e-3
    T0 = 1200.0
    y0 = np.array([[T0, 1.0, 0.0, 0.0]])
    param = 0.8 if reactor == 1 else 101325.0
    y, _, st, _ = om.integrate(method, param, y0, t, rtol=1e-10, atol=1e-14)
    assert st[0] == 0
    ya = np.exp(-k1 * t)
    yb = k1 / (k2 - k1) * (np.exp(-k1 * t) - np.exp(-k2 * t))
    Y = np.array([ya, yb, 1.0 - ya - yb])
    c = 3.5 - 1.0 if reactor == 1 else 3.5
    T = T0 + np.sum((np.array([1.0, 0.0, 0.0]) - Y) * a6) / c
    assert np.max(np.abs(y[0, 1:] - Y)) <= 1e-8
    assert abs(y[0, 0] - T) <= 1e-6 * T


@pytest.mark.parametrize("name", MECHS)
def test_cv_jacobian_complex_step(name):
    m = load_mechanism(CONFIGS[name]["mech"])
    om = OracleMech(m, reactor=1)
    y, rho = cv_states(name, 2, seed_offset=2)
    for i in range(2):
        J, G = om.jacobian(rho[i], y[i], gross=True)
        _assert_matches_complex_step(om, rho[i], y[i], J[0], G[0])


@pytest.mark.parametrize("name", ["small", "medium"])
def test_cv_integrated_internal_energy(name):
    m = load_mechanism(CONFIGS[name]["mech"])
    om = OracleMech(m, reactor=1)
    y, rho = cv_states(name, 3, seed_offset=3)
    ye, _, st, _ = om.integrate(ORA_ROS4, rho, y, CONFIGS[name]["dt"])
    assert np.all(st == 0)
    for i in range(3):
        u0, s0 = _u_mass(om, m, y[i])
        u1, s1 = _u_mass(om, m, ye[i])
        assert abs(u1 - u0) <= 1e-7 * max(s0, s1)
        assert abs(ye[i, 1:].sum() - 1.0) <= 1e-10


def _explicit_from_kc(m):
    """Closed-form explicit reverse coefficients of a constant-cp mechanism."""
    nasa = m["nasa"]
    assert np.allclose(nasa[:, :, 1:5], 0.0) and np.allclose(nasa[:, 0], nasa[:, 1])
    a1, a6, a7 = nasa[:, 0, 0], nasa[:, 0, 5], nasa[:, 0, 6]
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    R = len(m["rev"])
    arr = np.zeros((R, 3))
    for i in range(R):
        nu = np.zeros(len(a1))
        for s in m["prod"][i]:
            if s >= 0:
                nu[s] += 1
        for s in m["reac"][i]:
            if s >= 0:
                nu[s] -= 1
        dnu, da1, da6, da7 = nu.sum(), nu @ a1, nu @ a6, nu @ a7
        A, beta, Ea = m["arrh"][i]
        arr[i] = [A * (R_GAS / P0) ** dnu * np.exp(da1 - da7), beta + dnu - da1, Ea - R_GAS * da6]
    out["rev"] = np.full(R, 2, np.uint8)
    out["arrh_rev"] = arr
    return out


@pytest.mark.parametrize("reactor", [0, 1])
def test_explicit_reverse_closed_form_equivalence(reactor):
    m = cyclic_network()
    me = _explicit_from_kc(m)
    a, b = OracleMech(m, reactor=reactor), OracleMech(me, reactor=reactor)
    for T in (700.0, 1200.0, 2600.0):
        kf_a, kc_a, kr_a, _ = a.rate_coeffs(T)
        kf_b, kc_b, kr_b, _ = b.rate_coeffs(T)
        assert np.allclose(kr_b, kr_a, rtol=1e-12, atol=0)
        assert np.allclose(kc_b, kc_a, rtol=1e-12, atol=0)
    rng = np.random.default_rng(4)
    for _ in range(4):
        Y = rng.dirichlet(np.ones(4))
        y = np.concatenate([[rng.uniform(800, 2500)], Y])
        par = rng.uniform(0.2, 3.0) if reactor else rng.uniform(1, 20) * P0
        fa, fb = a.rhs(par, y)[0], b.rhs(par, y)[0]
        g = a.rhs_gross(par, y)[0]
        assert np.all(np.abs(fa - fb) <= 1e-12 * g + 1e-30)
        Ja, Ga = a.jacobian(par, y, gross=True)
        Jb = b.jacobian(par, y)
        assert np.all(np.abs(Ja - Jb) <= 1e-11 * Ga + 1e-30)


@pytest.mark.parametrize("reactor", [0, 1])
def test_explicit_reverse_jacobian_complex_step(reactor):
    m = with_explicit_reverse(load_mechanism(CONFIGS["medium"]["mech"]))
    assert (m["rev"] == 2).sum() > 50
    om = OracleMech(m, reactor=reactor)
    if reactor:
        y, par = cv_states("medium", 2, seed_offset=4)
    else:
        y, par = synth.configs.reactor_states("medium", n=2, seed_offset=4)
    for i in range(2):
        J, G = om.jacobian(par[i], y[i], gross=True)
        _assert_matches_complex_step(om, par[i], y[i], J[0], G[0])


def test_reactor_and_reverse_inputs_validated():
    m = cyclic_network()
    with pytest.raises(ValueError):
        OracleMech(m, reactor=2)
    bad = dict(m)
    bad["rev"] = np.full(len(m["rev"]), 3, np.uint8)
    with pytest.raises(ValueError):
        OracleMech(bad)
