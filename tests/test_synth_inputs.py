"""Structure of the stored synthetic mechanisms and the seeded states."""
import numpy as np
import pytest

from synth.configs import CONFIGS, load_mechanism, reactor_states


@pytest.mark.parametrize("name", ["small", "medium", "large"])
def test_mechanism_structure(name):
    cfg = CONFIGS[name]
    m = load_mechanism(cfg["mech"])
    S, R = cfg["n_species"], cfg["n_reactions"]
    assert m["mw"].shape == (S,) and m["reac"].shape == (R, 3) and m["nasa"].shape == (S, 2, 7)
    assert int((m["rtype"] == 1).sum()) == cfg["n_thirdbody"]
    assert int((m["rtype"] == 2).sum()) == cfg["n_falloff"]
    assert np.all(m["rev"] == 1)
    used = np.zeros(S, bool)
    for i in range(R):
        a = [s for s in m["reac"][i] if s >= 0]
        b = [s for s in m["prod"][i] if s >= 0]
        assert 1 <= len(a) <= 3 and 1 <= len(b) <= 3
        # atom balance
        assert np.array_equal(m["elem"][a].sum(0), m["elem"][b].sum(0))
        if m["rtype"][i] in (1, 2):
            assert len(a) != len(b)
        used[a] = True
        used[b] = True
    assert used.all()
    # molar masses follow the compositions
    masses = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999}
    W = m["elem"] @ np.array([masses[e] for e in m["elements"]]) * 1e-3
    assert np.allclose(W, m["mw"], rtol=1e-15)
    # parameter ranges
    assert np.all((m["arrh"][:, 1] >= -1) & (m["arrh"][:, 1] <= 2))
    assert np.all((m["arrh"][:, 2] >= 0) & (m["arrh"][:, 2] <= 200e3))
    assert np.all((m["nasa"][:, 1, 0] >= 2.5) & (m["nasa"][:, 1, 0] <= 6.0))


def test_states_seeded_and_normalised():
    y1, p1 = reactor_states("small", n=64)
    y2, p2 = reactor_states("small", n=64)
    assert np.array_equal(y1, y2) and np.array_equal(p1, p2)
    assert np.allclose(y1[:, 1:].sum(1), 1.0, rtol=0, atol=1e-15)
    assert np.all(y1[:, 1:] >= 0)
    assert np.all((y1[:, 0] >= 1000) & (y1[:, 0] <= 2500))
    assert np.all((p1 >= 101325) & (p1 <= 20 * 101325))


def test_mixed_workload_structure():
    from synth.configs import ignition_states, mixed_batch
    groups = mixed_batch(n=2000, seed=1)
    assert [g[0] for g in groups] == ["small", "medium", "large"]
    assert [len(g[2]) for g in groups] == [1000, 700, 300]
    for name, y, p, dt in groups:
        assert np.all((dt >= 1e-6) & (dt <= 1e-4))
        assert np.allclose(y[:, 1:].sum(1), 1.0, atol=1e-12)
        yi, pi = ignition_states(name)
        # half of every group comes from the stored near-ignition states
        hit = sum(any(np.array_equal(row, t) for t in yi) for row in y)
        assert hit == len(y) // 2
