"""Constant-volume reactors and explicit reverse Arrhenius coefficients
(Sec. 3) on the GPU against the oracle, through the C ABI.

The bars are those of the constant-pressure path:
* RHS and Jacobian within 1e-12 of max(|oracle|, gross) + 1e-20;
* final states within |dT|/T <= 1e-6 and |dY_k| <= 1e-8 at rtol 1e-9,
  atol 1e-12, with equal statuses.

Inputs:
* constant volume: the workloads' compositions and T, with densities
  log-uniform on [0.1, 3] kg/m^3;
* explicit reverse: the 53-species mechanism with a quarter of its reversible
  reactions given explicit reverse coefficients fitted to its K_c rates.
"""
import numpy as np
import pytest

from synth.configs import CONFIGS, cv_states, load_mechanism, reactor_states
from conftest import state_errors
from oracle import ORA_RKF45, ORA_ROS4, OracleMech
from oracle.mechgen import with_explicit_reverse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


_cache = {}


def _case(ck, name, reactor, explicit):
    key = (name, reactor, explicit)
    if key not in _cache:
        m = load_mechanism(CONFIGS[name]["mech"])
        if explicit:
            m = with_explicit_reverse(m)
        _cache[key] = (m, ck.load_mechanism(m, reactor=reactor), OracleMech(m, reactor=reactor))
    return _cache[key]


def _inputs(name, reactor, n, seed_offset):
    if reactor:
        return cv_states(name, n, seed_offset=seed_offset)
    return reactor_states(name, n=n, seed_offset=seed_offset)


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


CASES = [("small", 1, False), ("medium", 1, False), ("large", 1, False), ("medium", 0, True),
         ("medium", 1, True)]


@pytest.mark.parametrize("name,reactor,explicit", CASES)
def test_rhs_matches_oracle(ck, name, reactor, explicit):
    m, gm, om = _case(ck, name, reactor, explicit)
    y, par = _inputs(name, reactor, 300, 51)
    out = torch.empty(y.shape, dtype=torch.float64, device="cuda")
    ck.rhs(gm, _dev(par), _dev(y), out)
    torch.cuda.synchronize()
    f = out.cpu().numpy()
    fo = om.rhs(par, y)
    g = om.rhs_gross(par, y)
    bound = 1e-12 * np.maximum(np.abs(fo), g) + 1e-20
    assert np.all(np.abs(f - fo) <= bound), np.max(np.abs(f - fo) / bound)


@pytest.mark.parametrize("name,reactor,explicit", CASES)
def test_jacobian_matches_oracle(ck, name, reactor, explicit):
    m, gm, om = _case(ck, name, reactor, explicit)
    y, par = _inputs(name, reactor, 12, 53)
    nn = y.shape[1]
    out = torch.empty((12, nn, nn), dtype=torch.float64, device="cuda")
    ck.jacobian(gm, _dev(par), _dev(y), out)
    torch.cuda.synchronize()
    J = out.cpu().numpy()
    Jo, G = om.jacobian(par, y, gross=True)
    bound = 1e-12 * np.maximum(np.abs(Jo), G) + 1e-20
    assert np.all(np.abs(J - Jo) <= bound), np.max(np.abs(J - Jo) / bound)


def _integrate(ck, gm, method, par, y, dt, **kw):
    yd = _dev(y)
    st = torch.empty(y.shape[0], dtype=torch.int32, device="cuda")
    fn = ck.integrate_ros4 if method == ORA_ROS4 else ck.integrate_rkf45
    fn(gm, _dev(par), yd, _dev(np.broadcast_to(dt, (y.shape[0],))), st, opts=ck.SolverOpts.make(**kw))
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy()


def _variant(reactor, explicit):
    return ("constant volume" if reactor else "constant pressure") + (", explicit reverse" if explicit else "")


@pytest.mark.parametrize("method,form", [(ORA_ROS4, 0), (ORA_RKF45, 1), (ORA_RKF45, 2)])
@pytest.mark.parametrize("name,reactor,explicit,n", [("small", 1, False, 256), ("medium", 1, False, 24),
                                                     ("large", 1, False, 6), ("medium", 0, True, 24),
                                                     ("medium", 1, True, 16)])
def test_integrate_matches_oracle(ck, method, form, name, reactor, explicit, n, parity_report):
    m, gm, om = _case(ck, name, reactor, explicit)
    y, par = _inputs(name, reactor, n, 57)
    dt = CONFIGS[name]["dt"]
    yg, stg = _integrate(ck, gm, method, par, y, dt, form=form)
    yo, _, sto, _ = om.integrate(method, par, y, dt)
    dTm, dYm = state_errors(yg, yo)
    parity_report.append({"case": "integrate", "workload": name, "variant": _variant(reactor, explicit),
                          "form": ("ros4" if method == ORA_ROS4 else f"rkf45 (form={form})"), "reactors": n,
                          "max_rel_dT": dTm, "max_abs_dY": dYm})
    assert np.array_equal(stg, sto) and np.all(stg == 0)
    assert np.max(np.abs(yg[:, 0] - yo[:, 0]) / yo[:, 0]) <= 1e-6
    assert np.max(np.abs(yg[:, 1:] - yo[:, 1:])) <= 1e-8


def test_cv_conserves_internal_energy_on_gpu(ck):
    m, gm, om = _case(ck, "medium", 1, False)
    y, rho = cv_states("medium", 32, seed_offset=59)
    yg, st = _integrate(ck, gm, ORA_ROS4, rho, y, 1e-5)
    assert np.all(st == 0)
    R = 8.314462618
    for i in range(32):
        u = []
        for v in (y[i], yg[i]):
            cp_R, h_RT, _ = om.thermo(v[0])
            uk = R * v[0] * (h_RT - 1.0) / m["mw"]
            u.append((np.sum(v[1:] * uk), np.sum(np.abs(v[1:] * uk))))
        assert abs(u[1][0] - u[0][0]) <= 1e-7 * max(u[0][1], u[1][1])


def test_loader_validates_new_fields(ck):
    m = load_mechanism(CONFIGS["small"]["mech"])
    with pytest.raises(ck.CKError, match="reactor"):
        ck.load_mechanism(m, reactor=2)
    bad = dict(m)
    bad["rev"] = np.asarray(m["rev"]).copy()
    bad["rev"][0] = 2
    with pytest.raises(ck.CKError, match="arrh_rev"):
        ck.load_mechanism(bad)


@pytest.mark.parametrize("name,reactor,explicit,n", [("small", 1, False, 64), ("medium", 1, True, 6)])
def test_fd_jacobian_ros4_on_variants(ck, name, reactor, explicit, n, parity_report):
    # the paper's forward-difference ROS4 (Sec. 5) on the Sec. 3 variants
    m, gm, om = _case(ck, name, reactor, explicit)
    y, par = _inputs(name, reactor, n, 61)
    dt = CONFIGS[name]["dt"]
    yg, stg = _integrate(ck, gm, ORA_ROS4, par, y, dt, jac=1)
    yo, _, sto, _ = om.integrate(ORA_ROS4, par, y, dt, jac=1)
    dTm, dYm = state_errors(yg, yo)
    parity_report.append({"case": "integrate", "workload": name, "variant": _variant(reactor, explicit),
                          "form": "ros4 (jac=1)", "reactors": n, "max_rel_dT": dTm, "max_abs_dY": dYm})
    assert np.array_equal(stg, sto) and np.all(stg == 0)
    assert np.max(np.abs(yg[:, 0] - yo[:, 0]) / yo[:, 0]) <= 1e-6
    assert np.max(np.abs(yg[:, 1:] - yo[:, 1:])) <= 1e-8


@pytest.mark.parametrize("precision", [1, 2])
def test_precision_form_on_constant_volume(ck, precision, parity_report):
    m, gm, om = _case(ck, "medium", 1, False)
    y, rho = _inputs("medium", 1, 16, 63)
    yg, stg = _integrate(ck, gm, ORA_ROS4, rho, y, 1e-5, precision=precision)
    yo, _, sto, _ = om.integrate(ORA_ROS4, rho, y, 1e-5)
    dTm, dYm = state_errors(yg, yo)
    parity_report.append({"case": "integrate", "workload": "medium", "variant": "constant volume",
                          "form": f"ros4 (precision={precision})", "reactors": 16, "max_rel_dT": dTm,
                          "max_abs_dY": dYm})
    assert np.array_equal(stg, sto) and np.all(stg == 0)
    assert np.max(np.abs(yg[:, 0] - yo[:, 0]) / yo[:, 0]) <= 1e-6
    assert np.max(np.abs(yg[:, 1:] - yo[:, 1:])) <= 1e-8
