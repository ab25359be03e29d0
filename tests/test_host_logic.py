"""Host-side logic that needs no GPU: the divergence measure of the batch
bench (Eq. waste), the autotuner's candidate shapes and cache key."""
import numpy as np
import pytest

import bench
from synth.configs import CONFIGS, load_mechanism


def test_waste_closed_forms():
    # equal step counts in every warp-sized group: nothing wasted
    w = bench.waste(np.full(64, 7))
    assert w["P"] == 32 and w["mean"] == 0.0 and w["frac_below_1pct"] == 1.0
    # one reactor of 32 takes twice the steps: W = 1 - (31 + 2) / (32 * 2)
    s = np.ones(32)
    s[5] = 2
    assert bench.waste(s)["mean"] == pytest.approx(1.0 - 33.0 / 64.0)
    # a ragged tail shorter than P is left out; fewer than P reactors give no groups
    assert bench.waste(np.concatenate([np.full(32, 3), [1, 9]]))["mean"] == 0.0
    assert bench.waste(np.ones(10))["mean"] is None


def test_autotune_candidates_are_valid_options():
    ck = pytest.importorskip("paper_1608_05794_gb300.ck")
    from paper_1608_05794_gb300 import autotune
    fields = {k for k, _ in ck.SolverOpts._fields_}
    for method in (0, 1):
        for S in (10, 53, 111):
            cands = autotune.candidates(method, S)
            assert cands, (method, S)
            for c in cands:
                assert set(c) <= fields
                o = ck.SolverOpts.make(**c)
                assert o.variant >= 0 and o.form in (0, 1, 2) and o.team in (0, 8, 16)
                if o.team == 16:
                    assert S + 1 <= 112


def test_autotune_key_separates_rate_forms_and_reactors():
    pytest.importorskip("paper_1608_05794_gb300.ck")
    from paper_1608_05794_gb300 import autotune
    from oracle.mechgen import with_explicit_reverse
    m = load_mechanism(CONFIGS["small"]["mech"])
    d0 = autotune.mech_digest(m)
    assert d0 == autotune.mech_digest(load_mechanism(CONFIGS["small"]["mech"]))
    assert autotune.mech_digest(m, reactor=1) != d0
    assert autotune.mech_digest(with_explicit_reverse(m)) != d0
