"""Request server (ck_server_*): results in a mix equal results alone, and
admission, cancellation and bounded waits behave as documented."""
import numpy as np
import pytest

from synth.configs import CONFIGS, load_mechanism, reactor_states

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


@pytest.fixture(scope="module")
def mechs(ck):
    return {name: ck.load_mechanism(load_mechanism(CONFIGS[name]["mech"])) for name in ("small", "medium", "large")}


def _alone(ck, gm, method, p, y, dt, opts):
    yd = torch.as_tensor(y, device="cuda").clone()
    st = torch.empty(len(p), dtype=torch.int32, device="cuda")
    steps = torch.empty((len(p), 2), dtype=torch.int32, device="cuda")
    fn = ck.integrate_ros4 if method == 0 else ck.integrate_rkf45
    fn(gm, torch.as_tensor(p, device="cuda"), yd, torch.as_tensor(dt, device="cuda"), st, steps=steps, opts=opts)
    torch.cuda.synchronize()
    return yd.cpu().numpy(), st.cpu().numpy(), steps.cpu().numpy()


def test_results_in_the_mix_equal_results_alone(ck, mechs):
    rng = np.random.default_rng(2004)
    reqs = []
    for k, (name, method, n, prec, host) in enumerate([
            ("small", 1, 700, 0, True), ("medium", 0, 300, 1, False), ("large", 0, 40, 1, True),
            ("medium", 1, 500, 0, False), ("small", 0, 900, 0, False), ("large", 1, 60, 0, True)]):
        y, p = reactor_states(name, n=n, seed_offset=100 + k)
        dt = 10.0 ** rng.uniform(-6, -5, n)
        opts = ck.SolverOpts.make(precision=prec)
        reqs.append((name, method, y, p, dt, opts, host))
    srv = ck.Server(hbm_budget_bytes=1 << 30, streams=3, chunk_reactors=128)
    tickets, outs = [], []
    for name, method, y, p, dt, opts, host in reqs:
        if host:
            yy = y.copy()
            st = np.zeros(len(p), np.int32)
            steps = np.zeros((len(p), 2), np.int32)
            t = srv.submit(mechs[name], method, np.ascontiguousarray(p), yy, np.ascontiguousarray(dt), st, steps, opts)
        else:
            yy = torch.as_tensor(y, device="cuda").clone()
            st = torch.empty(len(p), dtype=torch.int32, device="cuda")
            steps = torch.empty((len(p), 2), dtype=torch.int32, device="cuda")
            t = srv.submit(mechs[name], method, torch.as_tensor(p, device="cuda"), yy,
                           torch.as_tensor(dt, device="cuda"), st, steps, opts)
        tickets.append(t)
        outs.append((yy, st, steps))
    for t in tickets:
        srv.wait(t, 600.0)
        assert srv.poll(t) == 1
    torch.cuda.synchronize()
    for (name, method, y, p, dt, opts, host), (yy, st, steps) in zip(reqs, outs):
        ya, sa, stepsa = _alone(ck, mechs[name], method, p, y, dt, opts)
        got = yy if host else yy.cpu().numpy()
        gst = st if host else st.cpu().numpy()
        gsteps = steps if host else steps.cpu().numpy()
        assert np.array_equal(got, ya), name      # bitwise: same kernel, reactors independent
        assert np.array_equal(gst, sa) and np.array_equal(gsteps, stepsa)
        assert np.all(sa == 0)
    info = srv.stats()
    assert info["completed"] == len(reqs) and info["bytes_in_use"] == info["reserved"] > 0
    for t in tickets:
        srv.release(t)
    srv.close()


def test_serving_trace_matches_oracle(ck, mechs, parity_report):
    # a seeded trace shaped like the serving workload: each request a batch on
    # one of the three mechanisms, dt log-uniform on [1e-6, 1e-4] s, ROS4 in
    # the precision form or RKF45 50/50, all in flight together on three
    # streams in chunks of 128; request sizes are scaled to 64-512 cells so
    # the oracle can follow a sample of every request
    from oracle import OracleMech
    from conftest import state_errors
    rng = np.random.default_rng(2104)
    names = ["small", "medium", "large"]
    reqs = []
    for k in range(10):
        name = names[int(rng.integers(3))]
        n = int(round(10 ** rng.uniform(np.log10(64), np.log10(512))))
        method = int(rng.integers(2))
        dt = 10.0 ** rng.uniform(-6, -4)
        y, p = reactor_states(name, n=n, seed_offset=300 + k)
        opts = ck.SolverOpts.make(precision=1 if method == 0 else 0)
        reqs.append((name, method, y, p, dt, opts, bool(k % 2)))
    srv = ck.Server(hbm_budget_bytes=1 << 30, streams=3, chunk_reactors=128)
    outs = []
    for name, method, y, p, dt, opts, host in reqs:
        n = len(p)
        if host:
            yy, st = y.copy(), np.zeros(n, np.int32)
            t = srv.submit(mechs[name], method, np.ascontiguousarray(p), yy, np.full(n, dt), st, None, opts)
        else:
            yy = torch.as_tensor(y, device="cuda").clone()
            st = torch.empty(n, dtype=torch.int32, device="cuda")
            t = srv.submit(mechs[name], method, torch.as_tensor(p, device="cuda"), yy,
                           torch.full((n,), dt, dtype=torch.float64, device="cuda"), st, None, opts)
        outs.append((t, yy, st))
    for t, _, _ in outs:
        srv.wait(t, 600.0)
    torch.cuda.synchronize()
    oms = {}
    for (name, method, y, p, dt, opts, host), (t, yy, st) in zip(reqs, outs):
        got = yy if host else yy.cpu().numpy()
        gst = st if host else st.cpu().numpy()
        idx = np.sort(rng.choice(len(p), size=min(12, len(p)), replace=False))
        om = oms.setdefault(name, OracleMech(load_mechanism(CONFIGS[name]["mech"])))
        yo, _, sto, _ = om.integrate(method, p[idx], y[idx], dt)
        dTm, dYm = state_errors(got[idx], yo)
        parity_report.append({"case": "serving trace", "workload": name,
                              "form": "ros4 (precision=1)" if method == 0 else "rkf45", "reactors": len(p),
                              "sampled": len(idx), "dt": dt, "max_rel_dT": dTm, "max_abs_dY": dYm})
        assert np.array_equal(gst[idx], sto) and np.all(gst == 0)
        assert dTm <= 1e-6 and dYm <= 1e-8, (name, method, dTm, dYm)
    srv.close()


def test_admission_cancel_and_timeout(ck, mechs):
    y, p = reactor_states("medium", n=256, seed_offset=7)
    per = (y.shape[1] * 8 + 28)
    probe = ck.Server(hbm_budget_bytes=1 << 30, streams=1)
    reserved = probe.stats()["reserved"]   # the stream's solver scratch, inside the budget
    probe.close()
    with pytest.raises(ck.CKError, match="reserve"):
        ck.Server(hbm_budget_bytes=reserved, streams=1)
    srv = ck.Server(hbm_budget_bytes=reserved + per * 300, streams=1, chunk_reactors=64)
    # a request larger than the whole budget is refused
    big_y = np.zeros((400, y.shape[1]))
    with pytest.raises(ck.CKError, match="budget"):
        srv.submit(mechs["medium"], 0, np.ones(400), big_y, np.ones(400), np.zeros(400, np.int32))
    # the second request waits for memory behind the first
    a = dict(p=np.ascontiguousarray(p), y=y.copy(), dt=np.full(256, 1e-5), st=np.zeros(256, np.int32))
    b = dict(p=np.ascontiguousarray(p), y=y.copy(), dt=np.full(256, 1e-5), st=np.zeros(256, np.int32))
    ta = srv.submit(mechs["medium"], 0, a["p"], a["y"], a["dt"], a["st"])
    tb = srv.submit(mechs["medium"], 0, b["p"], b["y"], b["dt"], b["st"])
    with pytest.raises(ck.CKError, match="timeout"):
        srv.wait(tb, 0.0)
    srv.cancel(tb)
    assert srv.poll(tb) == 3
    srv.wait(ta, 600.0)
    assert srv.poll(ta) == 1 and np.all(a["st"] == 0)
    assert np.array_equal(b["y"], y)  # the cancelled request never ran
    srv.close()
