"""Write the shaped synthetic mechanisms to ``synth/data`` (TEST INFRASTRUCTURE).

Run once: ``python -m oracle.make_inputs`` (``python -m oracle.make_inputs
explicit_reverse`` writes the explicit-reverse variant of the medium
mechanism).  Calls only ``synth`` (random
draws) and ``oracle`` (shaping).  Prints the spectral radius of the analytic
Jacobian at a few seeded states of each workload as a stiffness report.
"""
from __future__ import annotations

import sys

import numpy as np

import synth
from synth.configs import CONFIGS, save_mechanism

from .mechgen import make_mechanism
from .oracle import OracleMech


def write_explicit_reverse():
    """The medium mechanism with explicit reverse coefficients on a quarter of
    its reversible reactions (oracle.mechgen.with_explicit_reverse), stored
    for the rate-form variant of the benchmark."""
    from synth.configs import EXPLICIT_REVERSE_MECH, load_mechanism
    from .mechgen import with_explicit_reverse
    m = with_explicit_reverse(load_mechanism(CONFIGS["medium"]["mech"]))
    print(f"  wrote {save_mechanism(EXPLICIT_REVERSE_MECH, m)} ({int((m['rev'] == 2).sum())} explicit reverse)")


def main(names=None):
    if names and "explicit_reverse" in names:
        write_explicit_reverse()
        names = [n for n in names if n != "explicit_reverse"]
        if not names:
            return
    for cname, cfg in CONFIGS.items():
        if names and cname not in names:
            continue
        print(f"{cname}: {cfg['mech']}")
        m = make_mechanism(cfg["n_species"], cfg["n_reactions"], cfg["n_thirdbody"], cfg["n_falloff"],
                           cfg["elements"], cfg["mech_seed"])
        path = save_mechanism(cfg["mech"], m)
        print(f"  wrote {path}")
        om = OracleMech(m)
        rng = np.random.default_rng(7)
        y, p = synth.draw_states(rng, m["names"], m["elem"], m["mw"], m["elements"], 8,
                                 cfg["t_range"], cfg["p_range_atm"])
        J = om.jacobian(p, y)
        rad = [np.abs(np.linalg.eigvals(J[i])).max() for i in range(len(p))]
        print("  spectral radius of J at 8 states: " + " ".join(f"{r:.2e}" for r in rad))


if __name__ == "__main__":
    main(sys.argv[1:] or None)
