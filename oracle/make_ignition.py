"""Near-ignition reactor states for the mixed workload (TEST INFRASTRUCTURE).

For each stored mechanism, seeded blends (T U[900, 2800] K, p U[1, 20] atm)
are integrated with the oracle's ROS4 on a log-spaced time grid up to
T_HORIZON.  The ignition time t_ign is where dT/dt peaks; a state is sampled
at t drawn uniformly from [0.5, 1.0] t_ign.  The synthetic mechanisms have
no chain-branching induction period, so for most blends dT/dt is largest at
t = 0; the heat-release event then has no interior peak, and its time scale
is taken as the half-width t_half (where dT/dt first falls below half its
initial value), with t drawn from [0.5, 1.0] t_half.  The states are written
to synth/data/ignition_<mech>.npz.  Only synth (random draws) and oracle
(integration) are called.

Run: python -m oracle.make_ignition
"""
from __future__ import annotations

import sys

import numpy as np

import synth
from synth.configs import CONFIGS, DATA_DIR, load_mechanism

from .oracle import ORA_ROS4, OracleMech

T_HORIZON = 1e-3
N_GRID = 60
PER_MECH = 24
RTOL, ATOL = 1e-7, 1e-12


def ignition_states(name: str, seed: int, count: int = PER_MECH):
    cfg = CONFIGS[name]
    m = load_mechanism(cfg["mech"])
    om = OracleMech(m)
    rng = np.random.default_rng(seed)
    grid = np.concatenate([[0.0], np.geomspace(1e-8, T_HORIZON, N_GRID)])
    out_y, out_p, out_t = [], [], []
    tries = 0
    while len(out_y) < count and tries < 20 * count:
        batch = 16
        tries += batch
        y0, p = synth.draw_states(rng, m["names"], m["elem"], m["mw"], m["elements"], batch, (900.0, 2800.0),
                                  (1.0, 20.0))
        # march every blend along the grid, recording dT/dt at each point
        y = y0.copy()
        dTdt = np.zeros((batch, len(grid)))
        dTdt[:, 0] = om.rhs(p, y)[:, 0]
        ok = np.ones(batch, bool)
        for g in range(1, len(grid)):
            y, steps, st, _ = om.integrate(ORA_ROS4, p, y, grid[g] - grid[g - 1], rtol=RTOL, atol=ATOL)
            ok &= st == 0
            dTdt[:, g] = om.rhs(p, y)[:, 0]
        for i in range(batch):
            if not ok[i] or len(out_y) >= count:
                continue
            gi = int(np.argmax(dTdt[i]))
            if gi == len(grid) - 1 or not (dTdt[i, 0] > 0.0):
                continue
            if gi == 0:
                below = np.flatnonzero(dTdt[i] < 0.5 * dTdt[i, 0])
                if len(below) == 0:
                    continue
                gi = int(below[0])
            t_ign = grid[gi]
            ts = rng.uniform(0.5, 1.0) * t_ign
            ys, _, st, _ = om.integrate(ORA_ROS4, p[i:i + 1], y0[i:i + 1], ts, rtol=RTOL, atol=ATOL)
            if st[0] != 0:
                continue
            out_y.append(ys[0])
            out_p.append(p[i])
            out_t.append(t_ign)
    return np.array(out_y), np.array(out_p), np.array(out_t)


def main(names=None):
    import os
    for k, name in enumerate(["small", "medium", "large"]):
        if names and name not in names:
            continue
        y, p, t = ignition_states(name, 3000 + k)
        path = os.path.join(DATA_DIR, f"ignition_{CONFIGS[name]['mech']}.npz")
        np.savez(path, y=y, p=p, t_ign=t)
        print(f"{name}: {len(y)} near-ignition states, t_ign from {t.min():.2e} to {t.max():.2e} s -> {path}",
              flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or None)
