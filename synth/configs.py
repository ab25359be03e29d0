"""Named synthetic workloads and loading of the stored mechanisms.

Mechanism sizes follow Table 1 of the paper (H2/CO 14/38 is replaced by a
10-species H/O/N stand-in; GRI-Mech 3.0 53/325; USC Mech II 111/784).  The
shaped mechanisms are stored as ``synth/data/<name>.npz``; they are written by
``oracle/make_inputs.py``.
"""
from __future__ import annotations

import os

import numpy as np

DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")

# name -> description of one workload
CONFIGS = {
    "small": dict(mech="mech_s10", n_species=10, n_reactions=20, n_thirdbody=2, n_falloff=1,
                  elements=["H", "O", "N"], mech_seed=1010, n_reactors=512, state_seed=2000,
                  t_range=(1000.0, 2500.0), p_range_atm=(1.0, 20.0), dt=1e-4),
    "medium": dict(mech="mech_s53", n_species=53, n_reactions=325, n_thirdbody=30, n_falloff=20,
                   elements=["C", "H", "O", "N"], mech_seed=1053, n_reactors=131072, state_seed=2001,
                   t_range=(1000.0, 2500.0), p_range_atm=(1.0, 20.0), dt=1e-5, rhs_repeats=1000),
    "large": dict(mech="mech_s111", n_species=111, n_reactions=784, n_thirdbody=72, n_falloff=48,
                  elements=["C", "H", "O", "N"], mech_seed=1111, n_reactors=65536, state_seed=2002,
                  t_range=(900.0, 2800.0), p_range_atm=(1.0, 20.0), dt=1e-5),
}

MECH_KEYS = ("names", "elements", "elem", "mw", "nasa", "tmid", "reac", "prod", "arrh",
             "rtype", "rev", "arrh0", "eff_ptr", "eff_sp", "eff_val")


def mechanism_path(name: str) -> str:
    return os.path.join(DATA_DIR, name + ".npz")


def load_mechanism(name: str) -> dict:
    """Load a stored mechanism as a dict of numpy arrays.

    Keys: names[S], elements[E], elem[S,E] int32 atom counts, mw[S] kg/mol,
    nasa[S,2,7] (index 0 = low range, 1 = high range), tmid[S] K,
    reac[R,3] / prod[R,3] species slots (-1 padded; a species repeated in
    slots has that stoichiometric coefficient), arrh[R,3] (A SI, beta,
    Ea J/mol), rtype[R] (0 elementary, 1 third-body, 2 Lindemann), rev[R]
    (1 reversible through K_c, 0 irreversible), arrh0[R,3] low-pressure limit
    for type 2, eff_ptr[R+1] / eff_sp / eff_val CSR third-body efficiencies
    (species not listed have efficiency 1).
    """
    path = mechanism_path(name)
    with np.load(path, allow_pickle=False) as z:
        m = {k: z[k] for k in z.files}
    m["names"] = [str(s) for s in m["names"]]
    m["elements"] = [str(s) for s in m["elements"]]
    return m


def save_mechanism(name: str, m: dict) -> str:
    os.makedirs(DATA_DIR, exist_ok=True)
    path = mechanism_path(name)
    out = {k: m[k] for k in MECH_KEYS}
    if "arrh_rev" in m:  # explicit reverse Arrhenius coefficients (rev == 2)
        out["arrh_rev"] = m["arrh_rev"]
    out["names"] = np.array(m["names"], dtype="U16")
    out["elements"] = np.array(m["elements"], dtype="U4")
    np.savez(path, **out)
    return path


def reactor_states(cfg_name: str, n: int | None = None, seed_offset: int = 0):
    """Seeded reactor states (y[n, S+1], p[n]) for a named workload."""
    from .draw import draw_states
    cfg = CONFIGS[cfg_name]
    m = load_mechanism(cfg["mech"])
    rng = np.random.default_rng(cfg["state_seed"] + seed_offset)
    nn = cfg["n_reactors"] if n is None else n
    return draw_states(rng, m["names"], m["elem"], m["mw"], m["elements"], nn,
                       cfg["t_range"], cfg["p_range_atm"])


def cv_states(cfg_name: str, n: int, seed_offset: int = 0):
    """Seeded constant-volume reactor states (y[n, S+1], rho[n]) for a named
    workload's mechanism: compositions and T as in reactor_states, densities
    log-uniform on [0.1, 3] kg/m^3 (seed state_seed + 7000 + seed_offset)."""
    from .draw import draw_densities
    y, _ = reactor_states(cfg_name, n=n, seed_offset=seed_offset)
    rng = np.random.default_rng(CONFIGS[cfg_name]["state_seed"] + 7000 + seed_offset)
    return y, draw_densities(rng, n)


# The medium mechanism with a quarter of its reversible reactions on explicit
# reverse Arrhenius coefficients (rev == 2, Sec. 3), stored by
# ``python -m oracle.make_inputs explicit_reverse``.
EXPLICIT_REVERSE_MECH = "mech_s53_rev"

# Mixed workload: the three mechanisms in one batch (50/35/15 split of
# 200000 reactors), T U[900, 2800] K, half the reactors of each mechanism
# drawn from its near-ignition states, dt log-uniform on [1e-6, 1e-4] s.
MIXED = dict(n_reactors=200000, split=(("small", 0.50), ("medium", 0.35), ("large", 0.15)), seed=2003,
             t_range=(900.0, 2800.0), p_range_atm=(1.0, 20.0), dt_range=(1e-6, 1e-4))


def ignition_states(cfg_name: str):
    """Stored near-ignition states (y, p) of a workload's mechanism."""
    path = os.path.join(DATA_DIR, f"ignition_{CONFIGS[cfg_name]['mech']}.npz")
    with np.load(path) as z:
        return z["y"], z["p"]


def mixed_batch(n: int | None = None, seed: int | None = None):
    """Groups of the mixed workload: list of (cfg_name, y, p, dt)."""
    from .draw import draw_states
    total = MIXED["n_reactors"] if n is None else n
    rng = np.random.default_rng(MIXED["seed"] if seed is None else seed)
    counts = [int(round(total * f)) for _, f in MIXED["split"]]
    counts[-1] = total - sum(counts[:-1])
    groups = []
    for (name, _), cnt in zip(MIXED["split"], counts):
        m = load_mechanism(CONFIGS[name]["mech"])
        half = cnt // 2
        y1, p1 = draw_states(rng, m["names"], m["elem"], m["mw"], m["elements"], cnt - half, MIXED["t_range"],
                             MIXED["p_range_atm"])
        yi, pi = ignition_states(name)
        idx = rng.integers(len(yi), size=half)
        y = np.concatenate([y1, yi[idx]])
        p = np.concatenate([p1, pi[idx]])
        perm = rng.permutation(cnt)
        dt = 10.0 ** rng.uniform(np.log10(MIXED["dt_range"][0]), np.log10(MIXED["dt_range"][1]), cnt)
        groups.append((name, np.ascontiguousarray(y[perm]), np.ascontiguousarray(p[perm]), dt))
    return groups
