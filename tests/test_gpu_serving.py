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
    assert info["completed"] == len(reqs) and info["bytes_in_use"] == 0
    for t in tickets:
        srv.release(t)
    srv.close()


def test_admission_cancel_and_timeout(ck, mechs):
    y, p = reactor_states("medium", n=256, seed_offset=7)
    per = (y.shape[1] * 8 + 28)
    srv = ck.Server(hbm_budget_bytes=per * 300, streams=1, chunk_reactors=64)
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
