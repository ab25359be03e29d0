"""Seeded synthetic inputs for batched constant-pressure reactor workloads.

This package holds random draws only: species compositions, atom-balanced
reaction structure, raw Arrhenius / fall-off / efficiency parameters, raw
NASA-7 coefficient draws and reactor states.  It evaluates no rate,
thermodynamic or integration formula of the method (Sec. 3 of Stone,
Alferman & Niemeyer, arXiv 1608.05794): the shaping of a drawn mechanism
(thermo continuity at T_mid, heat-capacity bounds, the stiffness cap) is done
by ``oracle/mechgen.py`` and its result is stored under ``synth/data``.

Both the CPU oracle and the CUDA library consume what this package returns;
neither imports the other.
"""
from .draw import (  # noqa: F401
    ATM,
    ELEMENT_MASS_G,
    draw_species,
    draw_reactions,
    draw_arrhenius,
    draw_thermo_raw,
    draw_states,
    draw_efficiencies,
    draw_densities,
    pick_reactions,
)
from .configs import CONFIGS, load_mechanism, mechanism_path  # noqa: F401
