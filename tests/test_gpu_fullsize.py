"""Parity at the workloads' full sizes, in the launch configuration the bench
times: the whole batch goes through one call, and a seeded sample of
reactors is checked against the oracle one by one (the oracle cannot
integrate the whole batch in test time).

Bars as in test_gpu_parity: RHS within 1e-12 of max(|oracle|, gross) +
1e-20; final states |dT|/T <= 1e-6 and |dY_k| <= 1e-8, equal statuses.
"""
import numpy as np
import pytest

from synth.configs import CONFIGS, load_mechanism, reactor_states
from conftest import state_errors
from oracle import ORA_RKF45, ORA_ROS4, OracleMech

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


def _full(name):
    cfg = CONFIGS[name]
    m = load_mechanism(cfg["mech"])
    y, p = reactor_states(name)  # the workload's full batch
    return cfg, m, y, p


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def _assert_states(yg, yo, stg, sto, report=None, what=None):
    if report is not None:
        dTm, dYm = state_errors(yg, yo)
        report.append(dict(what, max_rel_dT=dTm, max_abs_dY=dYm))
    assert np.array_equal(stg, sto)
    assert np.max(np.abs(yg[:, 0] - yo[:, 0]) / yo[:, 0]) <= 1e-6
    assert np.max(np.abs(yg[:, 1:] - yo[:, 1:])) <= 1e-8


def test_medium_full_batch_rhs_ros4_rkf45(ck, parity_report):
    cfg, m, y, p = _full("medium")
    n = y.shape[0]
    assert n == 131072
    gm = ck.load_mechanism(m)
    om = OracleMech(m)
    yd = torch.as_tensor(y, device="cuda")
    pd = torch.as_tensor(p, device="cuda")
    dt = torch.full((n,), cfg["dt"], dtype=torch.float64, device="cuda")
    # RHS over the whole batch, 256 sampled reactors
    f = torch.empty_like(yd)
    ck.rhs(gm, pd, yd, f)
    torch.cuda.synchronize()
    idx = _sample(n, 256, 71)
    fo = om.rhs(p[idx], y[idx])
    g = om.rhs_gross(p[idx], y[idx])
    bound = 1e-12 * np.maximum(np.abs(fo), g) + 1e-20
    assert np.all(np.abs(f.cpu().numpy()[idx] - fo) <= bound)
    # both integrators over the whole batch, 24 sampled reactors each
    for method, fn, seed in ((ORA_ROS4, ck.integrate_ros4, 72), (ORA_RKF45, ck.integrate_rkf45, 73)):
        yg = yd.clone()
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        fn(gm, pd, yg, dt, st)
        torch.cuda.synchronize()
        stg = st.cpu().numpy()
        assert np.all(stg == 0)
        idx = _sample(n, 24, seed)
        yo, _, sto, _ = om.integrate(method, p[idx], y[idx], cfg["dt"])
        _assert_states(yg.cpu().numpy()[idx], yo, stg[idx], sto, parity_report,
                       {"case": "integrate, full batch", "workload": "medium", "reactors": n, "sampled": 24,
                        "form": "ros4" if method == ORA_ROS4 else "rkf45"})


def test_large_full_batch_precision_form(ck, parity_report):
    # the precision form (FP32 LU and solves, one FP64 refinement) on the
    # whole 65536-reactor large batch, against the FP64 oracle and beside the
    # plain FP64 form on the same reactors
    cfg, m, y, p = _full("large")
    n = y.shape[0]
    assert n == 65536
    gm = ck.load_mechanism(m)
    om = OracleMech(m)
    idx = _sample(n, 8, 74)
    yo, _, sto, _ = om.integrate(ORA_ROS4, p[idx], y[idx], cfg["dt"])
    for prec in (1, 0):
        yg = torch.as_tensor(y, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        ck.integrate_ros4(gm, torch.as_tensor(p, device="cuda"), yg,
                          torch.full((n,), cfg["dt"], dtype=torch.float64, device="cuda"), st,
                          opts=ck.SolverOpts.make(precision=prec))
        torch.cuda.synchronize()
        stg = st.cpu().numpy()
        assert np.all(stg == 0)
        _assert_states(yg.cpu().numpy()[idx], yo, stg[idx], sto, parity_report,
                       {"case": "integrate, full batch", "workload": "large", "reactors": n, "sampled": 8,
                        "form": f"ros4 (precision={prec})" if prec else "ros4"})
