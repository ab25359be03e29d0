"""The mixed batching workload through ck_integrate_groups against the oracle.

The batching form integrates the three mechanisms in one call: every group is
a persistent work-queue kernel on a forked branch, captured in a CUDA graph
and replayed.  Its inputs are the stiffest the library sees: half of every
group's reactors start from the stored near-ignition states, temperatures run
from 900 to 2800 K and dt is log-uniform on [1e-6, 1e-4] s on the 10-, 53-
and 111-species mechanisms, the uneven per-reactor work of the divergence
study (Sec. 5.2, Eq. waste).  Every reactor of a seeded 240-reactor mixed
batch is compared with the oracle at the bars of the plain form: |dT|/T <=
1e-6, |dY_k| <= 1e-8 at rtol 1e-9, atol 1e-12, statuses equal.
"""
import numpy as np
import pytest

from conftest import state_errors
from oracle import ORA_RKF45, ORA_ROS4, OracleMech
from synth.configs import CONFIGS, ignition_states, load_mechanism, mixed_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_MIXED, SEED = 240, 77


@pytest.fixture(scope="module")
def ck():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1608_05794_gb300.ck as ck
    return ck


@pytest.fixture(scope="module")
def mixed():
    """The seeded mixed batch and the oracle's final states for both methods."""
    groups = mixed_batch(n=N_MIXED, seed=SEED)
    out = []
    for nm, y, p, dt in groups:
        m = load_mechanism(CONFIGS[nm]["mech"])
        om = OracleMech(m)
        ora = {meth: om.integrate(meth, p, y, dt)[::2] for meth in (ORA_ROS4, ORA_RKF45)}  # (y, status)
        out.append(dict(name=nm, m=m, y=y, p=p, dt=dt, oracle=ora))
    return out


def test_mixed_batch_covers_the_stiff_inputs(mixed):
    # the inputs the batching form is for: near-ignition states in every
    # group, the coldest temperatures and the longest steps on the two large
    # mechanisms
    for g in mixed:
        yi, _ = ignition_states(g["name"])
        from_ignition = sum(any(np.array_equal(row, s) for s in yi) for row in g["y"])
        assert from_ignition >= len(g["y"]) // 2
    big = [g for g in mixed if g["name"] in ("medium", "large")]
    assert min(g["y"][:, 0].min() for g in mixed) < 950.0
    assert max(g["dt"].max() for g in big) > 5e-5
    assert all((g["dt"] > 3e-5).sum() >= 3 for g in big)


FORMS = [(ORA_ROS4, {}), (ORA_ROS4, {"precision": 1}), (ORA_RKF45, {"form": 2}), (ORA_RKF45, {"form": 1})]


@pytest.mark.parametrize("method,kw", FORMS)
def test_graph_groups_match_oracle(ck, mixed, method, kw, parity_report):
    mechs = [ck.load_mechanism(g["m"]) for g in mixed]
    specs = []
    for g, gm in zip(mixed, mechs):
        specs.append(dict(mech=gm, p=torch.as_tensor(g["p"], device="cuda"),
                          y=torch.as_tensor(g["y"], device="cuda").clone(),
                          dt=torch.as_tensor(g["dt"], device="cuda"),
                          status=torch.empty(len(g["p"]), dtype=torch.int32, device="cuda"),
                          opts=ck.SolverOpts.make(**kw)))
    for rep in range(2):  # capture, then replay the captured graph
        for sp, g in zip(specs, mixed):
            sp["y"].copy_(torch.as_tensor(g["y"], device="cuda"))
        ck.integrate_groups(method, specs, use_graph=True)
        torch.cuda.synchronize()
        for sp, g in zip(specs, mixed):
            yg, stg = sp["y"].cpu().numpy(), sp["status"].cpu().numpy()
            yo, sto = g["oracle"][method]
            dTm, dYm = state_errors(yg, yo)
            if rep == 1:
                tags = ", ".join(f"{k}={v}" for k, v in kw.items())
                parity_report.append({"case": "integrate, mixed batch (graph groups)", "workload": g["name"],
                                      "form": ("ros4" if method == ORA_ROS4 else "rkf45") + (f" ({tags})" if tags else ""),
                                      "reactors": len(g["p"]), "max_rel_dT": dTm, "max_abs_dY": dYm})
            assert np.array_equal(stg, sto), g["name"]
            assert np.all(stg == 0)
            assert dTm <= 1e-6 and dYm <= 1e-8, (g["name"], dTm, dYm)
    ck.graph_cache_clear()


def test_sequential_groups_match_oracle(ck, mixed):
    # the groups launched one after another on the caller's stream
    mechs = [ck.load_mechanism(g["m"]) for g in mixed]
    specs = [dict(mech=gm, p=torch.as_tensor(g["p"], device="cuda"), y=torch.as_tensor(g["y"], device="cuda").clone(),
                  dt=torch.as_tensor(g["dt"], device="cuda"),
                  status=torch.empty(len(g["p"]), dtype=torch.int32, device="cuda"))
             for g, gm in zip(mixed, mechs)]
    ck.integrate_groups(ORA_ROS4, specs, use_graph=True, sequential=True)
    torch.cuda.synchronize()
    for sp, g in zip(specs, mixed):
        yo, sto = g["oracle"][ORA_ROS4]
        dTm, dYm = state_errors(sp["y"].cpu().numpy(), yo)
        assert np.array_equal(sp["status"].cpu().numpy(), sto)
        assert dTm <= 1e-6 and dYm <= 1e-8
    ck.graph_cache_clear()
