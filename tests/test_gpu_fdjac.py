"""Forward-difference ROS4 variant (Sec. 5) on the GPU against the oracle.

Tolerances:
* Jacobian: a difference column is (f(y + s_j e_j) - f(y)) / s_j, so the
  RHS parity bar (1e-12 of the gross sum) divided by the increment bounds it:
  |gpu - oracle| <= 4e-12 gross_i / s_j + 1e-12 |J| + 1e-20;
* final states: the same bar as the analytic form (|dT|/T <= 1e-6,
  |dY_k| <= 1e-8 at rtol 1e-9, atol 1e-12), statuses equal.
"""
import numpy as np
import pytest

from synth.configs import CONFIGS, load_mechanism, reactor_states
from conftest import state_errors
from oracle import ORA_ROS4, OracleMech

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -52


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


_mechs = {}


def _mech(ck, name):
    if name not in _mechs:
        m = load_mechanism(CONFIGS[name]["mech"])
        _mechs[name] = (m, ck.load_mechanism(m), OracleMech(m))
    return _mechs[name]


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _increments(om, p, y, h, rtol, atol):
    f0 = om.rhs(p, y)
    w = 1.0 / (atol + rtol * np.abs(y))
    fn = np.sqrt(np.mean((f0 * w) ** 2, axis=1))
    n = y.shape[1]
    floor = np.where(fn != 0.0, 1000.0 * np.abs(h) * U * n * fn, 1.0)
    return np.maximum(2.0 ** -26 * np.abs(y), floor[:, None] / w)


@pytest.mark.parametrize("name,n", [("small", 64), ("medium", 24), ("large", 5)])
def test_jacobian_fd_matches_oracle(ck, name, n):
    m, gm, om = _mech(ck, name)
    y, p = reactor_states(name, n=n, seed_offset=31)
    h = 10.0 ** np.random.default_rng(3).uniform(-9, -5, n)
    rtol, atol = 1e-9, 1e-12
    nn = y.shape[1]
    out = torch.empty((n, nn, nn), dtype=torch.float64, device="cuda")
    ck.jacobian_fd(gm, _dev(p), _dev(y), _dev(h), out, rtol=rtol, atol=atol)
    torch.cuda.synchronize()
    J = out.cpu().numpy()
    Jo = om.jacobian_fd(p, y, h, rtol=rtol, atol=atol)
    s = _increments(om, p, y, h, rtol, atol)
    g = om.rhs_gross(p, y)
    bound = 4e-12 * g[:, :, None] / s[:, None, :] + 1e-12 * np.abs(Jo) + 1e-20
    err = np.abs(J - Jo)
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3g}"


def test_jacobian_fd_host_pointers(ck):
    m, gm, om = _mech(ck, "small")
    y, p = reactor_states("small", n=7, seed_offset=2)
    h = np.full(7, 1e-7)
    nn = y.shape[1]
    Jh = np.zeros((7, nn, nn))
    ck.jacobian_fd(gm, p, y, h, Jh)
    out = torch.empty((7, nn, nn), dtype=torch.float64, device="cuda")
    ck.jacobian_fd(gm, _dev(p), _dev(y), _dev(h), out)
    torch.cuda.synchronize()
    assert np.array_equal(Jh, out.cpu().numpy())


def _integrate(ck, gm, p, y, dt, **kw):
    yd = _dev(y)
    st = torch.empty(y.shape[0], dtype=torch.int32, device="cuda")
    steps = torch.empty((y.shape[0], 2), dtype=torch.int32, device="cuda")
    ck.integrate_ros4(gm, _dev(p), yd, _dev(np.broadcast_to(dt, (y.shape[0],))), st, steps=steps,
                      opts=ck.SolverOpts.make(**kw))
    torch.cuda.synchronize()
    return yd.cpu().numpy(), steps.cpu().numpy(), st.cpu().numpy()


def _assert_states_close(y, yo, st, sto, report=None, what=None):
    if report is not None:
        dTm, dYm = state_errors(y, yo)
        report.append(dict(what, max_rel_dT=dTm, max_abs_dY=dYm, statuses_equal=bool(np.array_equal(st, sto))))
    assert np.array_equal(st, sto)
    dT = np.abs(y[:, 0] - yo[:, 0]) / yo[:, 0]
    dY = np.abs(y[:, 1:] - yo[:, 1:])
    assert dT.max() <= 1e-6, dT.max()
    assert dY.max() <= 1e-8, dY.max()


@pytest.mark.parametrize("name,n", [("small", 512), ("medium", 16), ("large", 3)])
def test_ros4_fd_matches_oracle(ck, name, n, parity_report):
    m, gm, om = _mech(ck, name)
    cfg = CONFIGS[name]
    y, p = reactor_states(name, n=n, seed_offset=37)
    yg, sg, stg = _integrate(ck, gm, p, y, cfg["dt"], jac=1)
    yo, so, sto, _ = om.integrate(ORA_ROS4, p, y, cfg["dt"], jac=1)
    _assert_states_close(yg, yo, stg, sto, parity_report,
                         {"case": "integrate", "workload": name, "form": "ros4 (jac=1)", "reactors": n})
    assert np.all(stg == 0)
    assert np.abs(sg.sum(1) - so.sum(1)).max() <= 0.1 * so.sum(1).max() + 3


def test_fd_and_analytic_reach_the_same_state(ck):
    m, gm, om = _mech(ck, "medium")
    y, p = reactor_states("medium", n=64, seed_offset=41)
    ya, sa, sta = _integrate(ck, gm, p, y, 1e-5, jac=0)
    yf, sf, stf = _integrate(ck, gm, p, y, 1e-5, jac=1)
    assert np.all(sta == 0) and np.all(stf == 0)
    assert np.all(np.abs(ya - yf) <= 1e3 * (1e-9 * np.abs(ya) + 1e-12))


def test_jac_option_is_validated(ck):
    m, gm, om = _mech(ck, "small")
    y, p = reactor_states("small", n=4)
    yd = _dev(y)
    st = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(ck.CKError, match="jac"):
        ck.integrate_rkf45(gm, _dev(p), yd, _dev(np.full(4, 1e-5)), st, opts=ck.SolverOpts.make(jac=1))
    with pytest.raises(ck.CKError, match="jac"):
        ck.integrate_ros4(gm, _dev(p), yd, _dev(np.full(4, 1e-5)), st, opts=ck.SolverOpts.make(jac=2))


def test_fd_work_count(ck):
    m, gm, om = _mech(ck, "medium")
    w = ck.count_work(gm)
    n = len(m["mw"]) + 1
    # S+1 more RHS evaluations (Sec. 5) in place of the analytic Jacobian's work
    assert w["ros4_fd_step_fp64"] - w["ros4_step_fp64"] > n * w["rhs_fp64"] - w["jac_fp64"]
