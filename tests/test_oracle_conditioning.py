"""Conditioning of the ROS4 iteration matrix along real trajectories: the
evidence behind the precision form's choice of FP32 over BF16 factors.

The stages of ROS4 (Sec. 2) solve M u = b with M = I/(h gamma) - J.  An LU
factored in a low precision with unit roundoff u_f and refined against M in
FP64 reduces the error by about kappa u_f per refinement step, and the
FP64 residual of every step costs n^2 FMAs on the FP64 pipe, the scarce unit
of this path; the factorization itself runs on other pipes in either case.

The oracle integrates seeded medium and large reactors; stopping it after k
attempted steps (max_steps = k) returns the state and the step size of the
(k+1)-th attempt, i.e. the (y, h) pairs the driver visits.  At each pair:
* the 2-norm condition number of M, raw and after one sweep of row and
  column equilibration (which partial pivoting would be given in the low
  precision form);
* the refinement steps needed to reach FP64 accuracy (1e-15 relative) at
  the equilibrated kappa: (kappa u_f)^(k+1) <= 1e-15.
The checks: FP32 (u = 2^-24) converges everywhere in at most 2 steps (the
precision form runs 1 or 2), while BF16 (u = 2^-8) needs at least 4 more
steps at every pair; and raw, unequilibrated BF16 refinement would diverge
(kappa u >= 1) at most pairs.  So BF16 tiles would add FP64 residual work
where FP32 factors add none, whatever the tensor cores save.
"""
import numpy as np
import pytest

from oracle import ORA_ROS4, OracleMech
from synth.configs import CONFIGS, load_mechanism, reactor_states

GAMMA = 0.57282  # App. C
U_FP32, U_BF16 = 2.0 ** -24, 2.0 ** -8


def _visited_pairs(name, n_reactors, seed_offset, n_points=8):
    cfg = CONFIGS[name]
    om = OracleMech(load_mechanism(cfg["mech"]))
    y, p = reactor_states(name, n=n_reactors, seed_offset=seed_offset)
    out = []
    for i in range(n_reactors):
        _, s, st, _ = om.integrate(ORA_ROS4, p[i:i + 1], y[i:i + 1], cfg["dt"], h_inout=np.zeros(1))
        assert st[0] == 0
        total = int(s.sum())
        for k in sorted(set([1, 2] + [int(x) for x in np.geomspace(3, total, n_points)])):
            yk, _, stk, hk = om.integrate(ORA_ROS4, p[i:i + 1], y[i:i + 1], cfg["dt"], h_inout=np.zeros(1),
                                          max_steps=k)
            if stk[0] == 0:  # reached dt within k attempts
                break
            J = om.jacobian(p[i:i + 1], yk)[0]
            out.append(np.eye(J.shape[0]) / (hk[0] * GAMMA) - J)
    return out


def _equilibrate(M):
    r = 1.0 / np.abs(M).max(axis=1)
    Mr = M * r[:, None]
    c = 1.0 / np.abs(Mr).max(axis=0)
    return Mr * c[None, :]


def _steps_to_fp64(kappa, u):
    rho = kappa * u
    if rho >= 1.0:
        return np.inf
    return max(0, int(np.ceil(np.log(1e-15) / np.log(rho))) - 1)


@pytest.mark.parametrize("name,n", [("medium", 4), ("large", 3)])
def test_fp32_factors_dominate_bf16(name, n):
    mats = _visited_pairs(name, n, seed_offset=91)
    assert len(mats) >= 10 * n // 2
    raw = np.array([np.linalg.cond(M) for M in mats])
    eq = np.array([np.linalg.cond(_equilibrate(M)) for M in mats])
    k32 = np.array([_steps_to_fp64(k, U_FP32) for k in eq])
    k16 = np.array([_steps_to_fp64(k, U_BF16) for k in eq])
    # the badly scaled raw matrices: BF16 refinement without equilibration
    # diverges at most visited pairs (median kappa above 2^8)
    assert np.median(raw) * U_BF16 >= 1.0
    # equilibrated, the matrices are well conditioned ...
    assert eq.max() < 50.0
    # ... FP32 reaches FP64 accuracy in at most two refinement steps ...
    assert k32.max() <= 2
    # ... while BF16 needs at least four more FP64 residuals at every pair
    assert np.all(k16 >= k32 + 4)
