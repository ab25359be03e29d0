"""Shaping of synthetic mechanisms with the oracle (TEST INFRASTRUCTURE).

``synth`` draws raw random parameters; this module turns them into a usable
mechanism by evaluating the oracle's own NASA-7 polynomials (Eq. tfits) and
rate coefficients (Eqs. kfor, kc, krev):

* thermo: the low-range a2..a5 are perturbed high-range ones, and the
  low-range a1, a6, a7 are solved so that cp, H and S are continuous at
  T_mid; a species is redrawn until 2.5 <= cp/R <= 3 atoms + 3 on
  [300, 3500] K; a6 and a7 are then shifted in both ranges so that H(298 K)
  equals the drawn heat of formation and S(298 K)/R the drawn entropy;
* stiffness cap: a candidate reaction is kept only if every forward and
  reverse pseudo-first-order rate k C^(m-1) (times [M] <= 6 C for third-body
  reactions; min(k_inf, k0 [M]) for fall-off) stays below ``lam_cap`` on
  800-3000 K at 20 atm, C = p/(R T).  Its Arrhenius parameters are redrawn a
  few times before the reaction itself is discarded.  Without such a cap the
  stated parameter ranges give pseudo-first-order rates near 1e16 1/s, where
  an explicit method cannot run.

The result is written to ``synth/data`` by ``oracle/make_inputs.py`` and read
by both the oracle and the CUDA library.
"""
from __future__ import annotations

import numpy as np

import synth
from synth.draw import draw_arrhenius, draw_efficiencies, draw_reactions, draw_species, draw_thermo_raw, redraw_high

from .oracle import OracleMech

R_GAS = 8.314462618
T_MID = 1000.0
T_GRID_CAP = np.linspace(800.0, 3000.0, 23)
P_CAP = 20.0 * synth.ATM
CP_GRID = np.linspace(300.0, 3500.0, 33)


def _thermo_mech(S, nasa, tmid):
    """An oracle mechanism with S species and no reactions (for thermo only)."""
    z = np.zeros((0, 3))
    return OracleMech(dict(mw=np.ones(S), nasa=nasa, tmid=tmid, reac=np.zeros((0, 3), np.int32),
                           prod=np.zeros((0, 3), np.int32), arrh=z, rtype=np.zeros(0, np.int32),
                           rev=np.zeros(0, np.int32), arrh0=z, eff_ptr=np.zeros(1, np.int32),
                           eff_sp=np.zeros(0, np.int32), eff_val=np.zeros(0)))


def shape_thermo(rng, names, elem, raw):
    """Continuous two-range NASA-7 coefficients [S,2,7] with bounded cp."""
    S = len(names)
    atoms = elem.sum(axis=1)
    high = raw["high"].copy()
    dlow = raw["dlow"].copy()
    nasa = np.zeros((S, 2, 7))
    for k in range(S):
        for _ in range(1000):
            a_hi = np.zeros(7)
            a_hi[:5] = high[k]
            a_lo = np.zeros(7)
            a_lo[1:5] = high[k, 1:5] + dlow[k]
            # evaluate each range alone at T_mid (tmid far away selects one range)
            one = np.zeros((1, 2, 7))
            one[0, 0] = a_lo
            one[0, 1] = a_hi
            lo_only = _thermo_mech(1, one, np.array([1e30]))
            hi_only = _thermo_mech(1, one, np.array([0.0]))
            cpH, hH, sH = hi_only.thermo(T_MID)
            cpL, hL, sL = lo_only.thermo(T_MID)
            a_lo[0] = cpH[0] - cpL[0]
            one[0, 0] = a_lo
            lo_only = _thermo_mech(1, one, np.array([1e30]))
            cpL, hL, sL = lo_only.thermo(T_MID)
            a_lo[5] = (hH[0] - hL[0]) * T_MID
            a_lo[6] = sH[0] - sL[0]
            one[0, 0] = a_lo
            both = _thermo_mech(1, one, np.array([T_MID]))
            cps = np.array([both.thermo(T)[0][0] for T in CP_GRID])
            if cps.min() >= 2.5 and cps.max() <= 3.0 * atoms[k] + 3.0:
                break
            high[k] = redraw_high(rng)
            dlow[k] = dlow[k] * 0.5
        else:
            raise RuntimeError(f"cp bounds unreachable for species {names[k]}")
        # anchor H(298) and S(298)
        both = _thermo_mech(1, one, np.array([T_MID]))
        _, h298, s298 = both.thermo(298.15)
        d6 = raw["dhf298"][k] / R_GAS - h298[0] * 298.15
        d7 = raw["s298_r"][k] - s298[0]
        one[0, :, 5] += d6
        one[0, :, 6] += d7
        nasa[k] = one[0]
    return nasa, np.full(S, T_MID)


class CapCheck:
    """Stiffness-cap acceptance of candidate reactions (see module doc)."""

    def __init__(self, rng, S, mw, nasa, tmid, lam_cap, arrh_tries=40):
        self.rng = rng
        self.S = S
        self.mw = mw
        self.nasa = nasa
        self.tmid = tmid
        self.lam_cap = lam_cap
        self.arrh_tries = arrh_tries
        self.candidates = 0
        self.rejected = 0

    def _max_rates(self, a, b, rtype, arrh, arrh0):
        reac = -np.ones((1, 3), np.int32)
        prod = -np.ones((1, 3), np.int32)
        reac[0, : len(a)] = a
        prod[0, : len(b)] = b
        om = OracleMech(dict(mw=self.mw, nasa=self.nasa, tmid=self.tmid, reac=reac, prod=prod,
                             arrh=arrh[None, :], rtype=np.array([rtype], np.int32),
                             rev=np.ones(1, np.int32), arrh0=arrh0[None, :],
                             eff_ptr=np.zeros(2, np.int32), eff_sp=np.zeros(0, np.int32),
                             eff_val=np.zeros(0)))
        worst = 0.0
        for T in T_GRID_CAP:
            kf, kc, kr, k0 = om.rate_coeffs(T)
            C = P_CAP / (R_GAS * T)
            M = 6.0 * C if rtype in (1, 2) else C
            if rtype == 1:
                ef, er = kf[0] * M, kr[0] * M
            elif rtype == 2:
                c = (k0[0] * M / kf[0]) / (1.0 + k0[0] * M / kf[0])
                ef, er = kf[0] * c, kr[0] * c
            else:
                ef, er = kf[0], kr[0]
            worst = max(worst, ef * C ** (len(a) - 1), er * C ** (len(b) - 1))
            if not np.isfinite(worst):
                return np.inf
        return worst

    def __call__(self, a, b, rtype):
        self.candidates += 1
        for _ in range(self.arrh_tries):
            arrh, arrh0 = draw_arrhenius(self.rng, len(a), rtype)
            if self._max_rates(a, b, rtype, arrh, arrh0) <= self.lam_cap:
                return arrh, arrh0
        self.rejected += 1
        return None


def make_mechanism(n_species, n_reactions, n_thirdbody, n_falloff, elements, seed, lam_cap=1e8,
                   verbose=True):
    """Draw and shape one synthetic mechanism (dict of arrays, see
    ``synth.load_mechanism``)."""
    rng = np.random.default_rng(seed)
    for attempt in range(50):
        names, elem, mw = draw_species(rng, n_species, elements)
        raw = draw_thermo_raw(rng, names)
        nasa, tmid = shape_thermo(rng, names, elem, raw)
        cap = CapCheck(rng, n_species, mw, nasa, tmid, lam_cap)
        try:
            reac, prod, rtype, params = draw_reactions(rng, elem, n_reactions, n_thirdbody, n_falloff,
                                                       accept=cap)
        except (ValueError, RuntimeError) as e:
            if verbose:
                print(f"  redraw species set ({e})")
            continue
        break
    else:
        raise RuntimeError("could not draw a mechanism")
    arrh = np.array([p[0] for p in params])
    arrh0 = np.array([p[1] for p in params])
    eff_ptr, eff_sp, eff_val = draw_efficiencies(rng, n_species, rtype)
    m = dict(names=names, elements=list(elements), elem=elem, mw=mw, nasa=nasa, tmid=tmid,
             reac=reac, prod=prod, arrh=arrh, rtype=rtype, rev=np.ones(len(rtype), np.uint8),
             arrh0=arrh0, eff_ptr=eff_ptr, eff_sp=eff_sp, eff_val=eff_val)
    if verbose:
        print(f"  {n_species} species, {len(rtype)} reactions; cap {lam_cap:g}/s rejected "
              f"{cap.rejected} of {cap.candidates} candidate reactions")
    return m


def with_explicit_reverse(m: dict, frac: float = 0.25, seed: int = 4242,
                          temps=(1000.0, 1700.0, 2500.0)) -> dict:
    """A copy of mechanism m in which a random fraction of the reversible
    reactions carries explicit reverse Arrhenius coefficients (Sec. 3)
    instead of K_c.  Each explicit triple (A_r, beta_r, Ea_r) interpolates
    the K_c-based reverse rate ln k_r(T) = ln A_r + beta_r ln T - Ea_r/(R T)
    exactly at three temperatures, so the reverse rates (and the stiffness
    cap they obey) stay close to the original ones.  Test input only."""
    rng = np.random.default_rng(seed)
    picked = synth.pick_reactions(rng, m["rev"], frac)
    om = OracleMech(m)
    lnkr = np.array([np.log(om.rate_coeffs(T)[2][picked]) for T in temps])  # [3, k]
    R_GAS = 8.314462618
    A = np.array([[1.0, np.log(T), -1.0 / (R_GAS * T)] for T in temps])
    coef = np.linalg.solve(A, lnkr)  # rows: ln A_r, beta_r, Ea_r
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    out["rev"] = np.asarray(m["rev"]).astype(np.uint8).copy()
    out["rev"][picked] = 2
    arrh_rev = np.zeros((len(m["rev"]), 3))
    arrh_rev[picked, 0] = np.exp(coef[0])
    arrh_rev[picked, 1] = coef[1]
    arrh_rev[picked, 2] = coef[2]
    out["arrh_rev"] = arrh_rev
    return out
