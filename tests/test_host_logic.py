"""Host-side logic that needs no GPU: the divergence measure of the batch
bench (Eq. waste), the autotuner's candidate shapes and cache key, the
bench's work model and roofline arithmetic, the serving trace and its
latency-bound test, and the clock summary."""
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


def _work():
    # a stand-in for ck_count_work's output (only the fields the model reads)
    return dict(n_species=53, rhs_flops=100.0, rhs_transc=10.0, ros4_jeval_flops=1000.0, ros4_attempt_flops=3000.0,
                rkf45_step_flops=700.0, ros4_fd_jeval_flops=5500.0, rhs_fp64=80.0, jac_fp64=400.0,
                ros4_step_fp64=2500.0, rkf45_step_fp64=500.0, ros4_fd_step_fp64=6400.0)


def test_ros4_work_charges_one_jacobian_per_accepted_step():
    w = _work()
    steps = np.array([[10, 0], [8, 2]])      # 20 attempts, 18 accepted
    r = bench.ros4_work(w, steps)
    assert r["attempts"] == 20 and r["jacobians"] == 18
    assert r["flops"] == 18 * 1000.0 + 20 * 3000.0 + 4 * 100.0            # + 2 RHS of EstimateH0 each
    assert r["transc"] == (18 + 2 * 20 + 4) * 10.0
    assert r["fp64_instr"] == 18 * 480.0 + 20 * (2500.0 - 480.0) + 4 * 80.0
    assert bench.ros4_work(w, steps, h0_estimated=False)["flops"] == 18 * 1000.0 + 20 * 3000.0


def test_ros4_work_forward_differences_redo_the_columns_after_a_rejection():
    w = _work()
    r = bench.ros4_work(w, np.array([[8, 2]]), h0_estimated=False, fd=True)
    assert r["jacobians"] == 10
    # f(y) and 54 columns at each of the 8 new states; the 54 columns alone after each rejection
    assert r["flops"] == 8 * 5500.0 + 2 * (5500.0 - 100.0) + 10 * 3000.0
    assert r["transc"] == (8 * 55 + 2 * 54 + 2 * 10) * 10.0


def test_roofline_rate_arithmetic():
    peaks = {"fp64_flops_per_s": 1e12, "w_exp": 16.0}
    r = bench.roofline_rate({"flops": 6e11, "transc": 1e10, "fp64_instr": 2e11}, 1.0, peaks)
    assert r["tflops"] == pytest.approx(0.76) and r["frac"] == pytest.approx(0.76)
    assert r["fp64_issue_frac"] == pytest.approx(0.4)
    assert bench.rkf45_work(_work(), np.array([[3, 1]]))["flops"] == 4 * 700.0 + 2 * 100.0


def test_serving_trace_is_seeded_and_in_range():
    a, b = bench.make_trace(50), bench.make_trace(50)
    assert a == b
    lo, hi = bench.SERVE_CELLS
    for r in a:
        assert r["name"] in ("small", "medium", "large") and lo <= r["n"] <= hi
        assert 1e-6 <= r["dt"] <= 1e-4 and r["method"] in (0, 1)
    arr = bench.poisson_arrivals(20000, 50.0)
    assert np.all(np.diff(arr) > 0) and np.mean(np.diff(arr)) == pytest.approx(1 / 50.0, rel=0.03)


def test_bounded_p99_detects_a_growing_queue():
    arr = np.arange(100.0)
    assert bench.bounded_p99(np.full(100, 0.3), arr)
    assert not bench.bounded_p99(0.1 + 0.5 * arr, arr)   # every request waits longer than the last
    assert bench.bounded_p99(np.array([1.0, 2.0]), arr[:2])


def test_clock_summary():
    lines = ["1980, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "2070, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active", "garbage"]
    c = bench.summarize_clocks(lines)
    assert c["sm_mhz"] == pytest.approx(2025.0) and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 2
    assert bench.summarize_clocks([]) is None
