"""CUDA path against the CPU oracle, element by element, through the C ABI.

Tolerances (stated as error against the oracle):
* RHS and Jacobian: |gpu - oracle| <= 1e-12 * max(|oracle|, gross) + 1e-20,
  where gross is the same sum with every term in absolute value (the scale
  that cancellation near equilibrium leaves rounding errors at);
* final states: |dT|/T <= 1e-6 and |dY_k| <= 1e-8 at rtol 1e-9, atol 1e-12,
  statuses equal;
* LU: pivots identical, factors within 1e-13 relative to the matrix scale.
"""
import numpy as np
import pytest

import synth
from synth.configs import CONFIGS, load_mechanism, reactor_states
from synth.handmade import cyclic_network, linear_chain
from oracle import ORA_RKF45, ORA_ROS4, OracleMech
from conftest import plain_relative, state_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_STATE_T = 1e-6
ATOL_STATE_Y = 1e-8


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


_mechs = {}


def _mech(ck, name):
    if name not in _mechs:
        m = load_mechanism(CONFIGS[name]["mech"]) if name in CONFIGS else name
        _mechs[name] = (m, ck.load_mechanism(m), OracleMech(m))
    return _mechs[name]


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _gpu_rhs(ck, gm, p, y):
    out = torch.empty((y.shape[0], y.shape[1]), dtype=torch.float64, device="cuda")
    ck.rhs(gm, _dev(p), _dev(y), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _assert_rhs_close(f, fo, g, report=None, what=None):
    bound = 1e-12 * np.maximum(np.abs(fo), g) + 1e-20
    err = np.abs(f - fo)
    if report is not None:
        # the asserted bar scales by the gross rate (cancellation near
        # equilibrium); the plain relative error with the 1e-20 floor is
        # reported beside it
        report.append(dict(what, max_gross_ratio=float(np.max(err / bound)), **plain_relative(err, fo)))
    bad = err > bound
    assert not bad.any(), f"{bad.sum()} entries off; worst ratio {np.max(err / bound):.3g}"


@pytest.mark.parametrize("name,n", [("small", 1000), ("medium", 300), ("large", 161)])
def test_rhs_matches_oracle(ck, name, n, parity_report):
    m, gm, om = _mech(ck, name)
    y, p = reactor_states(name, n=n, seed_offset=17)
    f = _gpu_rhs(ck, gm, p, y)
    fo = om.rhs(p, y)
    g = om.rhs_gross(p, y)
    _assert_rhs_close(f, fo, g, parity_report, {"case": "rhs", "workload": name, "reactors": n})


@pytest.mark.parametrize("name", ["small", "medium", "large"])
def test_rhs_ragged_batches(ck, name):
    # k_rhs gives each thread several reactors; batches of 1 to 7 leave the
    # last group partly empty (it repeats the last reactor), and every
    # reactor must still match the oracle and the one-at-a-time result
    m, gm, om = _mech(ck, name)
    y, p = reactor_states(name, n=7, seed_offset=29)
    full = _gpu_rhs(ck, gm, p, y)
    for n in range(1, 8):
        f = _gpu_rhs(ck, gm, p[:n], y[:n])
        assert np.array_equal(f, full[:n])
        _assert_rhs_close(f, om.rhs(p[:n], y[:n]), om.rhs_gross(p[:n], y[:n]))


def test_rhs_temperature_sweep_crosses_thermo_ranges(ck):
    # the paper's RHS input (Sec. 5.1): uniform composition, T linear over
    # 500-1500 K, so lanes straddle the NASA-7 range boundary
    m, gm, om = _mech(ck, "medium")
    n = 777
    S = len(m["mw"])
    y = np.empty((n, S + 1))
    y[:, 0] = np.linspace(500.0, 1500.0, n)
    y[:, 1:] = 1.0 / S
    p = np.full(n, 101325.0)
    _assert_rhs_close(_gpu_rhs(ck, gm, p, y), om.rhs(p, y), om.rhs_gross(p, y))


@pytest.mark.parametrize("name,n", [("small", 70), ("medium", 40), ("large", 9)])
def test_jacobian_matches_oracle(ck, name, n, parity_report):
    m, gm, om = _mech(ck, name)
    y, p = reactor_states(name, n=n, seed_offset=23)
    nn = y.shape[1]
    out = torch.empty((n, nn, nn), dtype=torch.float64, device="cuda")
    ck.jacobian(gm, _dev(p), _dev(y), out)
    torch.cuda.synchronize()
    J = out.cpu().numpy()
    Jo, G = om.jacobian(p, y, gross=True)
    bound = 1e-12 * np.maximum(np.abs(Jo), G) + 1e-20
    err = np.abs(J - Jo)
    parity_report.append(dict(case="jacobian", workload=name, reactors=n, max_gross_ratio=float(np.max(err / bound)),
                              **plain_relative(err, Jo)))
    assert np.all(err <= bound), f"worst ratio {np.max(err / bound):.3g}"


@pytest.mark.parametrize("dim", [1, 2, 5, 11, 33, 54, 112])
def test_lu_matches_oracle_and_lapack(ck, oracle_lib, dim):
    rng = np.random.default_rng(dim)
    batch = 37
    A = rng.standard_normal((batch, dim, dim))
    b = rng.standard_normal((batch, dim))
    a_d = _dev(A)
    piv = torch.empty((batch, dim), dtype=torch.int32, device="cuda")
    info = torch.empty(batch, dtype=torch.int32, device="cuda")
    ck.lu_factor(a_d, piv, info)
    b_d = _dev(b)
    ck.lu_solve(a_d, piv, b_d)
    torch.cuda.synchronize()
    LU, P, I, X = a_d.cpu().numpy(), piv.cpu().numpy(), info.cpu().numpy(), b_d.cpu().numpy()
    assert np.all(I == 0)
    for k in range(batch):
        lu_o, piv_o, info_o = oracle_lib.lu_factor(A[k])
        assert np.array_equal(P[k], piv_o)
        scale = np.abs(A[k]).max()
        assert np.allclose(LU[k], lu_o, rtol=0, atol=1e-12 * scale * dim)
        xr = np.linalg.solve(A[k], b[k])
        assert np.allclose(X[k], xr, rtol=1e-9, atol=1e-9 * np.abs(xr).max())


def test_lu_reports_singular(ck):
    A = np.array([[[1.0, 2.0], [2.0, 4.0]], [[0.0, 1.0], [1.0, 0.0]]])
    a_d = _dev(A)
    piv = torch.empty((2, 2), dtype=torch.int32, device="cuda")
    info = torch.empty(2, dtype=torch.int32, device="cuda")
    ck.lu_factor(a_d, piv, info)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [2, 0]
    assert piv.cpu().numpy()[1, 0] == 1


@pytest.mark.parametrize("dim,k,rows", [(8, 0, (3, 5)), (11, 2, (9, 4, 6)), (54, 30, (43, 35, 38)),
                                         (54, 47, (53, 50)), (112, 0, (17, 97, 33)), (112, 64, (96, 81, 80))])
def test_lu_pivot_ties_take_the_first_row(ck, oracle_lib, dim, k, rows):
    # upper triangular in the columns before k, so steps 0..k-1 exchange
    # nothing and leave column k exactly as given; there the rows `rows`
    # share the largest magnitude (signs mixed), and the smallest of them
    # must become pivot k, as in the oracle, whichever lanes, tile slots and
    # warps hold them
    rng = np.random.default_rng(dim * 1000 + k)
    A = np.triu(rng.standard_normal((dim, dim))) + 4.0 * np.eye(dim)
    A[k + 1:, k] = rng.uniform(-1.0, 1.0, size=dim - k - 1)
    A[k, k] = 0.5
    for q, i in enumerate(rows):
        A[i, k] = 6.0 if q % 2 == 0 else -6.0
    a_d = _dev(A[None])
    piv = torch.empty((1, dim), dtype=torch.int32, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    ck.lu_factor(a_d, piv, info)
    torch.cuda.synchronize()
    _, piv_o, info_o = oracle_lib.lu_factor(A)
    P = piv.cpu().numpy()[0]
    assert info.cpu().tolist() == [0] and info_o == 0
    assert P[k] == min(rows) == piv_o[k]
    assert np.array_equal(P[:k], np.arange(k))


@pytest.mark.parametrize("dim,zero_at", [(54, 0), (54, 30), (112, 70), (11, 10)])
def test_lu_reports_a_late_singular_pivot(ck, dim, zero_at):
    # upper triangular: no row exchanges, and the column below a zero
    # diagonal entry is zero, so pivot zero_at is the first zero one
    rng = np.random.default_rng(dim + zero_at)
    A = np.triu(rng.standard_normal((dim, dim))) + 4.0 * np.eye(dim)
    A[zero_at, zero_at] = 0.0
    a_d = _dev(A[None])
    piv = torch.empty((1, dim), dtype=torch.int32, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    ck.lu_factor(a_d, piv, info)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [zero_at + 1]
    assert np.array_equal(piv.cpu().numpy()[0, :zero_at], np.arange(zero_at))


@pytest.mark.parametrize("dim", [11, 54, 112])
def test_lu_reports_non_finite_matrices(ck, dim):
    rng = np.random.default_rng(dim)
    A = rng.standard_normal((3, dim, dim)) + 4.0 * np.eye(dim)
    A[0, dim // 2, dim // 3] = np.nan
    A[1, dim - 1, 0] = np.inf
    a_d = _dev(A)
    piv = torch.empty((3, dim), dtype=torch.int32, device="cuda")
    info = torch.empty(3, dtype=torch.int32, device="cuda")
    ck.lu_factor(a_d, piv, info)
    torch.cuda.synchronize()
    I = info.cpu().tolist()
    assert I[0] != 0 and I[1] != 0 and I[2] == 0


def _integrate_gpu(ck, gm, method, p, y, dt, **kw):
    yd = _dev(y)
    st = torch.empty(y.shape[0], dtype=torch.int32, device="cuda")
    steps = torch.empty((y.shape[0], 2), dtype=torch.int32, device="cuda")
    h = _dev(np.zeros(y.shape[0]))
    fn = ck.integrate_ros4 if method == ORA_ROS4 else ck.integrate_rkf45
    fn(gm, _dev(p), yd, _dev(np.broadcast_to(dt, (y.shape[0],))), st, h_inout=h, steps=steps,
       opts=ck.SolverOpts.make(**kw))
    torch.cuda.synchronize()
    return yd.cpu().numpy(), steps.cpu().numpy(), st.cpu().numpy(), h.cpu().numpy()


def _assert_states_close(y, yo, st, sto, report=None, what=None):
    if report is not None:
        dTm, dYm = state_errors(y, yo)
        report.append(dict(what, max_rel_dT=dTm, max_abs_dY=dYm, statuses_equal=bool(np.array_equal(st, sto))))
    assert np.array_equal(st, sto)
    dT = np.abs(y[:, 0] - yo[:, 0]) / yo[:, 0]
    dY = np.abs(y[:, 1:] - yo[:, 1:])
    assert dT.max() <= RTOL_STATE_T, dT.max()
    assert dY.max() <= ATOL_STATE_Y, dY.max()


FORMS = [(ORA_ROS4, 0), (ORA_RKF45, 1), (ORA_RKF45, 2)]


def _form_name(method, **kw):
    base = "ros4" if method == ORA_ROS4 else "rkf45"
    tags = [f"{k}={v}" for k, v in sorted(kw.items()) if v]
    return base + (" (" + ", ".join(tags) + ")" if tags else "")


@pytest.mark.parametrize("method,form", FORMS)
def test_integrate_small_config_full(ck, method, form, parity_report):
    name = "small"
    m, gm, om = _mech(ck, name)
    cfg = CONFIGS[name]
    y, p = reactor_states(name)
    yg, sg, stg, hg = _integrate_gpu(ck, gm, method, p, y, cfg["dt"], form=form)
    yo, so, sto, ho = om.integrate(method, p, y, cfg["dt"], h_inout=np.zeros(len(p)))
    _assert_states_close(yg, yo, stg, sto, parity_report,
                         {"case": "integrate", "workload": name, "form": _form_name(method, form=form),
                          "reactors": len(p)})
    assert np.all(stg == 0)
    # step counts are reported, not required to match
    assert np.abs(sg.sum(1) - so.sum(1)).max() <= 0.1 * so.sum(1).max() + 3


@pytest.mark.parametrize("method,form", FORMS)
@pytest.mark.parametrize("name,n", [("medium", 48), ("large", 12)])
def test_integrate_sampled(ck, method, form, name, n, parity_report):
    m, gm, om = _mech(ck, name)
    cfg = CONFIGS[name]
    y, p = reactor_states(name, n=n, seed_offset=5)
    yg, sg, stg, _ = _integrate_gpu(ck, gm, method, p, y, cfg["dt"], form=form)
    yo, so, sto, _ = om.integrate(method, p, y, cfg["dt"])
    _assert_states_close(yg, yo, stg, sto, parity_report,
                         {"case": "integrate", "workload": name, "form": _form_name(method, form=form),
                          "reactors": n})


@pytest.mark.parametrize("method", [ORA_ROS4, ORA_RKF45])
def test_linear_chain_closed_form_on_gpu(ck, method):
    m = linear_chain(1e2, 1e4)
    gm = ck.load_mechanism(m)
    t = 1e-3
    y0 = np.array([[1000.0, 1.0, 0.0, 0.0]] * 3)
    y, steps, st, _ = _integrate_gpu(ck, gm, method, np.full(3, 101325.0), y0, t)
    ya = np.exp(-1e2 * t)
    yb = 1e2 / (1e4 - 1e2) * (np.exp(-1e2 * t) - np.exp(-1e4 * t))
    assert np.all(st == 0)
    assert np.max(np.abs(y[:, 1] - ya)) <= 1e-8 and np.max(np.abs(y[:, 2] - yb)) <= 1e-8
    assert np.max(np.abs(y[:, 0] - 1000.0)) <= 1e-9


def test_edge_cases(ck):
    m, gm, om = _mech(ck, "small")
    y, p = reactor_states("small", n=5, seed_offset=3)
    y[1, 3] = np.nan      # non-finite state
    y[2, 0] = -5.0        # T <= 0
    dt = np.array([1e-5, 1e-5, 1e-5, 0.0, 1e-5])
    p = p.copy()
    p[4] = 0.0            # p <= 0
    for method, form in FORMS:
        yg, sg, stg, _ = _integrate_gpu(ck, gm, method, p, y, dt, form=form)
        assert stg.tolist() == [0, 5, 5, 0, 5]
        assert sg[3].tolist() == [0, 0] and np.array_equal(yg[3], y[3])
    # max_steps
    yg, sg, stg, _ = _integrate_gpu(ck, gm, ORA_RKF45, p[:1], y[:1], 1e-4, max_steps=2)
    assert stg[0] == 1 and sg[0].sum() == 2
    # empty batch is a no-op
    e = torch.empty((0, y.shape[1]), dtype=torch.float64, device="cuda")
    ck.integrate_ros4(gm, torch.empty(0, dtype=torch.float64, device="cuda"), e,
                      torch.empty(0, dtype=torch.float64, device="cuda"),
                      torch.empty(0, dtype=torch.int32, device="cuda"))
    ck.rhs(gm, torch.empty(0, dtype=torch.float64, device="cuda"), e, e)


@pytest.mark.parametrize("n", [1, 31, 33, 129])
def test_ragged_batches_and_host_pointers(ck, n):
    m, gm, om = _mech(ck, "small")
    y, p = reactor_states("small", n=n, seed_offset=n)
    # host (numpy) arrays go through the library's staging path
    f_host = np.zeros_like(y)
    ck.rhs(gm, np.ascontiguousarray(p), np.ascontiguousarray(y), f_host)
    f_dev = _gpu_rhs(ck, gm, p, y)
    assert np.array_equal(f_host, f_dev)
    yh = y.copy()
    st = np.zeros(n, np.int32)
    ck.integrate_ros4(gm, np.ascontiguousarray(p), yh, np.full(n, 1e-5), st)
    yd, _, std, _ = _integrate_gpu(ck, gm, ORA_ROS4, p, y, 1e-5)
    assert np.array_equal(yh, yd) and np.array_equal(st, std)


def test_bitwise_deterministic(ck):
    m, gm, om = _mech(ck, "medium")
    y, p = reactor_states("medium", n=200, seed_offset=9)
    a = _integrate_gpu(ck, gm, ORA_ROS4, p, y, 1e-6)
    b = _integrate_gpu(ck, gm, ORA_ROS4, p, y, 1e-6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = _integrate_gpu(ck, gm, ORA_RKF45, p, y, 1e-6)
    d = _integrate_gpu(ck, gm, ORA_RKF45, p, y, 1e-6)
    assert np.array_equal(c[0], d[0])


def test_cyclic_network_equilibrium_on_gpu(ck):
    m = cyclic_network()
    gm = ck.load_mechanism(m)
    om = OracleMech(m)
    y = np.array([[1500.0, 0.7, 0.1, 0.2, 0.0], [1200.0, 0.0, 0.0, 0.0, 1.0]])
    p = np.array([101325.0, 3 * 101325.0])
    yg, _, stg, _ = _integrate_gpu(ck, gm, ORA_ROS4, p, y, 1e-2, rtol=1e-10, atol=1e-16, max_steps=1000000)
    yo, _, sto, _ = om.integrate(ORA_ROS4, p, y, 1e-2, rtol=1e-10, atol=1e-16, max_steps=1000000)
    _assert_states_close(yg, yo, stg, sto)


def test_work_counts_scale(ck):
    for name in ("small", "medium", "large"):
        m, gm, om = _mech(ck, name)
        w = ck.count_work(gm)
        n = len(m["mw"]) + 1
        assert w["lu_fp64"] > n ** 3 / 3
        assert w["ros4_step_fp64"] > w["lu_fp64"] + 3 * w["rhs_fp64"]
        assert w["rhs_exps"] >= len(m["rtype"])
        # the flop model: LU of an n x n matrix = n reciprocals, n(n-1)/2
        # multipliers and sum (n-k-1)^2 FMAs (2 flops each) ~ 2n^3/3; a solve
        # pair n(n-1) FMAs and n products ~ 2n^2
        assert w["lu_flops"] == n + n * (n - 1) / 2 + 2 * (n - 1) * n * (2 * n - 1) / 6
        assert w["solve_flops"] == 2 * n * (n - 1) + n
        assert w["ros4_step_flops"] == w["ros4_jeval_flops"] + w["ros4_attempt_flops"]
        assert w["ros4_attempt_flops"] > 2 * w["rhs_flops"] + w["lu_flops"] + 4 * w["solve_flops"]
        assert w["ros4_jeval_flops"] > w["rhs_flops"] + 2 * (n - 1) ** 2  # the species block, twice
        # one ln T and the exponentials of every RHS
        assert w["rhs_transc"] == w["rhs_exps"] + 1
        assert w["rkf45_step_flops"] > 6 * w["rhs_flops"]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name,n", [("small", 128), ("medium", 48), ("large", 16)])
def test_ros4_precision_form_matches_fp64_oracle(ck, name, n, precision, parity_report):
    # FP32 LU and stage solves with one or two FP64 refinement steps per
    # solve; the final states must meet the same bar as the FP64 form
    m, gm, om = _mech(ck, name)
    cfg = CONFIGS[name]
    y, p = reactor_states(name, n=n, seed_offset=29)
    yg, sg, stg, _ = _integrate_gpu(ck, gm, ORA_ROS4, p, y, cfg["dt"], precision=precision)
    yo, so, sto, _ = om.integrate(ORA_ROS4, p, y, cfg["dt"])
    _assert_states_close(yg, yo, stg, sto, parity_report,
                         {"case": "integrate", "workload": name,
                          "form": _form_name(ORA_ROS4, precision=precision), "reactors": n})


def test_precision_option_is_validated(ck):
    m, gm, om = _mech(ck, "small")
    y, p = reactor_states("small", n=4)
    with pytest.raises(ck.CKError, match="precision"):
        _integrate_gpu(ck, gm, ORA_RKF45, p, y, 1e-5, precision=1)
