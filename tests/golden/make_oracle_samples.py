"""Write tests/golden/oracle_samples.npz: the oracle's final states for seeded
samples of the workloads' reactors, the expected values that bench.py
compares the GPU forms with (bench.py reads this file; it runs no oracle code
outside its CPU-baseline leg).

Run from the repository root:  python tests/golden/make_oracle_samples.py

Contents, per key prefix <workload>_<method>:
  idx     the sampled reactor indices of the workload's full batch
          (synth.configs.reactor_states, seed offset 0);
  y       the oracle's final states after integrating each over the
          workload's dt at rtol 1e-9, atol 1e-12 (ROS4: Sec. 2, App. C;
          Algorithm 1);
  status  the oracle's per-reactor statuses.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ORA_ROS4, OracleMech  # noqa: E402
from synth.configs import CONFIGS, load_mechanism, reactor_states  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_samples.npz")

# (workload, method, sample size, seed of the index draw)
SAMPLES = [("large", ORA_ROS4, 16, 4401)]


def main():
    out = {}
    for name, method, k, seed in SAMPLES:
        cfg = CONFIGS[name]
        y, p = reactor_states(name)
        idx = np.sort(np.random.default_rng(seed).choice(len(p), size=k, replace=False))
        om = OracleMech(load_mechanism(cfg["mech"]))
        yo, _, st, _ = om.integrate(method, p[idx], y[idx], cfg["dt"])
        tag = f"{name}_{'ros4' if method == ORA_ROS4 else 'rkf45'}"
        out[f"{tag}_idx"] = idx
        out[f"{tag}_y"] = yo
        out[f"{tag}_status"] = st
        print(tag, "statuses", np.bincount(st))
    np.savez(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
