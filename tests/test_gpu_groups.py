"""Mixed batches (ck_integrate_groups) and the autotuner."""
import numpy as np
import pytest

from synth.configs import CONFIGS, load_mechanism, mixed_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


def _dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("use_graph", [False, True])
def test_groups_equal_separate_calls(ck, method, use_graph):
    groups = mixed_batch(n=600, seed=11)
    mechs = {nm: ck.load_mechanism(load_mechanism(CONFIGS[nm]["mech"])) for nm, *_ in groups}
    specs, refs = [], []
    for nm, y, p, dt in groups:
        opts = ck.SolverOpts.make(form=2)
        yy, st = _dev(y), torch.empty(len(p), dtype=torch.int32, device="cuda")
        specs.append(dict(mech=mechs[nm], p=_dev(p), y=yy, dt=_dev(dt), status=st, opts=opts))
        yr, sr = _dev(y), torch.empty(len(p), dtype=torch.int32, device="cuda")
        fn = ck.integrate_ros4 if method == 0 else ck.integrate_rkf45
        fn(mechs[nm], _dev(p), yr, _dev(dt), sr, opts=opts)
        refs.append((yr, sr))
    for rep in range(2):  # the second graph call replays the captured graph
        for sp, (nm, y, p, dt) in zip(specs, groups):
            sp["y"].copy_(_dev(y))
        ck.integrate_groups(method, specs, use_graph=use_graph)
        torch.cuda.synchronize()
        for sp, (yr, sr) in zip(specs, refs):
            assert torch.equal(sp["y"], yr) and torch.equal(sp["status"], sr)
            assert bool((sr == 0).all())
    ck.graph_cache_clear()


def test_groups_reject_host_arrays(ck):
    nm, y, p, dt = mixed_batch(n=64, seed=3)[0]
    gm = ck.load_mechanism(load_mechanism(CONFIGS[nm]["mech"]))
    with pytest.raises(ck.CKError, match="device pointers"):
        ck.integrate_groups(1, [dict(mech=gm, p=p, y=y.copy(), dt=dt, status=np.zeros(len(p), np.int32))])


def test_autotuner_picks_a_valid_shape(ck, tmp_path):
    from paper_1608_05794_gb300 import autotune
    nm, y, p, dt = mixed_batch(n=800, seed=5)[1]
    m = load_mechanism(CONFIGS[nm]["mech"])
    gm = ck.load_mechanism(m)
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(gm, m, 1, _dev(p), _dev(y), _dev(dt), cache=cache, sample=256)
    assert best in autotune.candidates(1, gm.S)
    assert autotune.tune(gm, m, 1, _dev(p), _dev(y), _dev(dt), cache=cache, sample=256) == best  # cached


def test_group_order_tuner_picks_and_caches(ck, tmp_path):
    # concurrent and sequential group launches give the same bits; the tuner
    # times both and caches its choice
    from paper_1608_05794_gb300 import autotune
    groups = mixed_batch(n=300, seed=13)
    mds = [load_mechanism(CONFIGS[nm]["mech"]) for nm, *_ in groups]
    specs = [dict(mech=ck.load_mechanism(md), p=_dev(p), y=_dev(y), dt=_dev(dt),
                  status=torch.empty(len(p), dtype=torch.int32, device="cuda"), opts=ck.SolverOpts.make(form=2))
             for md, (nm, y, p, dt) in zip(mds, groups)]
    cache = str(tmp_path / "tune.json")
    seq = autotune.tune_groups(1, specs, mds, cache=cache)
    assert isinstance(seq, bool)
    for sp, (nm, y, p, dt) in zip(specs, groups):
        assert torch.equal(sp["y"], _dev(y))  # the inputs are restored
    assert autotune.tune_groups(1, specs, mds, cache=cache) == seq
    out = []
    for flag in (False, True):
        ck.integrate_groups(1, specs, use_graph=True, sequential=flag)
        torch.cuda.synchronize()
        out.append([sp["y"].clone() for sp in specs])
        for sp, (nm, y, p, dt) in zip(specs, groups):
            sp["y"].copy_(_dev(y))
    assert all(torch.equal(a, b) for a, b in zip(*out))
    ck.graph_cache_clear()
