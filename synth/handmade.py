"""Hand-built mechanisms with closed-form behaviour (test inputs).

Each function returns a mechanism dict in the layout of
``synth.load_mechanism``.  They contain data only.
"""
from __future__ import annotations

import numpy as np


def _const_cp_nasa(S, a1=3.5, a6=-1000.0, a7=5.0):
    nasa = np.zeros((S, 2, 7))
    nasa[:, :, 0] = a1
    nasa[:, :, 5] = a6
    nasa[:, :, 6] = a7
    return nasa


def linear_chain(k1: float, k2: float, a6=None) -> dict:
    """A -> B -> C, three isomers (same composition, same molar mass, same
    constant cp/R = 3.5), irreversible, beta = 0, Ea = 0.  With Y_A(0) = 1:
    Y_A = exp(-k1 t), Y_B = k1/(k2-k1) (exp(-k1 t) - exp(-k2 t)), Y_C = 1 - Y_A - Y_B.
    a6 (optional, per species, K): the enthalpy offsets H_k/R = 3.5 T + a6_k;
    equal offsets (the default) release no heat, so T stays constant."""
    S = 3
    elem = np.array([[1, 1], [1, 1], [1, 1]], np.int32)  # C1 O1 each
    mw = np.full(S, 28.010e-3)
    reac = np.array([[0, -1, -1], [1, -1, -1]], np.int32)
    prod = np.array([[1, -1, -1], [2, -1, -1]], np.int32)
    arrh = np.array([[k1, 0.0, 0.0], [k2, 0.0, 0.0]])
    nasa = _const_cp_nasa(S)
    if a6 is not None:
        nasa[:, :, 5] = np.asarray(a6, float)[:, None]
    return dict(names=["A", "B", "C"], elements=["C", "O"], elem=elem, mw=mw,
                nasa=nasa, tmid=np.full(S, 1000.0), reac=reac, prod=prod, arrh=arrh,
                rtype=np.zeros(2, np.uint8), rev=np.zeros(2, np.uint8), arrh0=np.zeros((2, 3)),
                eff_ptr=np.zeros(3, np.int32), eff_sp=np.zeros(0, np.int32), eff_val=np.zeros(0))


def const_cp_species(a1=4.0, a6=-2500.0, a7=12.0) -> dict:
    """One inert species with a constant heat capacity (a2..a5 = 0) and a
    trivial mechanism (no reactions)."""
    return dict(names=["X"], elements=["N"], elem=np.array([[2]], np.int32), mw=np.array([28.014e-3]),
                nasa=_const_cp_nasa(1, a1, a6, a7), tmid=np.array([1000.0]),
                reac=np.zeros((0, 3), np.int32), prod=np.zeros((0, 3), np.int32), arrh=np.zeros((0, 3)),
                rtype=np.zeros(0, np.uint8), rev=np.zeros(0, np.uint8), arrh0=np.zeros((0, 3)),
                eff_ptr=np.zeros(1, np.int32), eff_sp=np.zeros(0, np.int32), eff_val=np.zeros(0))


def cyclic_network() -> dict:
    """Fast reversible network with a cycle and molecularity changes.

    Species: isomers A, B, C (composition N1 O1) and dimer D (N2 O2), with
    constant-cp thermo of distinct enthalpies and entropies.  Reactions:
    A<=>B, B<=>C, A<=>C (a cycle: the three K_c must agree for a detailed
    equilibrium), 2A(+M)<=>D (third-body), B+C(+M)<=>D (Lindemann), 2C<=>D.
    Every reaction is reversible through K_c; equilibrium is reached within
    about 1e-3 s at 1500 K and 1 atm.
    """
    elem = np.array([[1, 1], [1, 1], [1, 1], [2, 2]], np.int32)  # N O
    mw = elem.astype(float) @ np.array([14.007e-3, 15.999e-3])
    nasa = np.zeros((4, 2, 7))
    nasa[:, :, 0] = np.array([3.5, 3.6, 3.4, 4.8])[:, None]
    nasa[:, :, 5] = np.array([9000.0, 7500.0, 10500.0, -15000.0])[:, None]  # H/R offsets (K)
    nasa[:, :, 6] = np.array([25.0, 23.5, 26.0, 47.0])[:, None]
    reac = np.array([[0, -1, -1], [1, -1, -1], [0, -1, -1], [0, 0, -1], [1, 2, -1], [2, 2, -1]], np.int32)
    prod = np.array([[1, -1, -1], [2, -1, -1], [2, -1, -1], [3, -1, -1], [3, -1, -1], [3, -1, -1]], np.int32)
    arrh = np.array([[2e5, 0.2, 8e3], [1e5, 0.0, 5e3], [5e4, 0.5, 12e3],
                     [1e2, 0.0, 0.0], [5e4, 0.3, 4e3], [2e4, 0.0, 2e3]])
    arrh0 = np.zeros((6, 3))
    arrh0[4] = [5e2, 0.0, 1e3]
    rtype = np.array([0, 0, 0, 1, 2, 0], np.uint8)
    eff_ptr = np.array([0, 0, 0, 0, 2, 4, 4], np.int32)
    eff_sp = np.array([1, 3, 0, 2], np.int32)
    eff_val = np.array([2.5, 0.5, 1.7, 3.0])
    return dict(names=["A", "B", "C", "D"], elements=["N", "O"], elem=elem, mw=mw, nasa=nasa,
                tmid=np.full(4, 1000.0), reac=reac, prod=prod, arrh=arrh, rtype=rtype,
                rev=np.ones(6, np.uint8), arrh0=arrh0, eff_ptr=eff_ptr, eff_sp=eff_sp,
                eff_val=eff_val)


T_PIN = 1000.0  # K: the temperature the round values of rate_pins() are placed at


def rate_pins() -> dict:
    """Three reactions whose rate coefficients take closed forms (test input).

    Isomers A, B (N1 O1) and dimer D (N2 O2) with constant heat capacities
    (cp/R = 3.5, 3.5, 7.0, so every ln T term of the Gibbs energies of
    reaction cancels) and enthalpy / entropy offsets chosen so that, with
    T0 = T_PIN:
      A <=> B       k_f = 2 T exp(-T0 ln2 / T)            (A = 2, beta = 1, Ea = R T0 ln 2)
                    K_c = 3 * 2^(T0/T)                    (dS/R = ln 3, dH/R = -T0 ln 2, dnu = 0)
      2A (+M) <=> D third body, k_f = 50 (constant),       K_c = 5 R T / p0     (dnu = -1)
      A + B (+M) <=> D Lindemann, k_inf = 1000, k0 = 10 T^-1 exp(-T0 ln4 / T),
                    K_c = (5/3) 2^(-T0/T) R T / p0
    so that at T0: k_f(A<=>B) = T0, K_c = 6; k0 = 10 / (4 T0); and at 2 T0:
    k_f = 2 sqrt(2) T0, K_c = 3 sqrt(2), k0 the same 10 / (4 T0)."""
    ln2, ln3, ln5 = np.log(2.0), np.log(3.0), np.log(5.0)
    R = 8.314462618
    elem = np.array([[1, 1], [1, 1], [2, 2]], np.int32)  # N O
    mw = elem.astype(float) @ np.array([14.007e-3, 15.999e-3])
    nasa = np.zeros((3, 2, 7))
    a6A, a7A = 1000.0, 20.0
    nasa[:, :, 0] = np.array([3.5, 3.5, 7.0])[:, None]
    nasa[:, :, 5] = np.array([a6A, a6A - T_PIN * ln2, 2 * a6A])[:, None]
    nasa[:, :, 6] = np.array([a7A, a7A + ln3, 2 * a7A + ln5])[:, None]
    reac = np.array([[0, -1, -1], [0, 0, -1], [0, 1, -1]], np.int32)
    prod = np.array([[1, -1, -1], [2, -1, -1], [2, -1, -1]], np.int32)
    arrh = np.array([[2.0, 1.0, R * T_PIN * ln2], [50.0, 0.0, 0.0], [1000.0, 0.0, 0.0]])
    arrh0 = np.zeros((3, 3))
    arrh0[2] = [10.0, -1.0, R * T_PIN * 2 * ln2]
    return dict(names=["A", "B", "D"], elements=["N", "O"], elem=elem, mw=mw, nasa=nasa,
                tmid=np.full(3, 1000.0), reac=reac, prod=prod, arrh=arrh,
                rtype=np.array([0, 1, 2], np.uint8), rev=np.ones(3, np.uint8), arrh0=arrh0,
                eff_ptr=np.zeros(4, np.int32), eff_sp=np.zeros(0, np.int32), eff_val=np.zeros(0))
