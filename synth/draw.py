"""Random draws for synthetic mechanisms and reactor states.

Everything here is a draw from ``numpy.random.Generator`` plus bookkeeping
(atom balance of multisets, unit conversion of pre-exponential factors,
normalisation of mass fractions).  No rate coefficient, thermodynamic
polynomial or ODE right-hand side is evaluated in this module.

The parameter distributions follow the workloads of Sec. 5 of the paper
(mechanism sizes of Table 1; N_reac roughly 5 N_sp, Sec. 4) with the ranges
stated for the synthetic stand-ins: A log-uniform on [1e6, 1e14] in
cm-mol-s units, beta uniform on [-1, 2], Ea uniform on [0, 200] kJ/mol,
NASA-7 high-range a1 uniform on [2.5, 6].
"""
from __future__ import annotations

import itertools

import numpy as np

ATM = 101325.0  # Pa per standard atmosphere (unit conversion only)

# Standard atomic masses in g/mol (IUPAC conventional values).
ELEMENT_MASS_G = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999}

# Simple molecules every mechanism carries (element -> count).
_BASE_SPECIES = {
    "H2": {"H": 2},
    "O2": {"O": 2},
    "N2": {"N": 2},
    "H2O": {"H": 2, "O": 1},
    "CO": {"C": 1, "O": 1},
    "CO2": {"C": 1, "O": 2},
}
# Upper bounds on atoms of each element in a random species.
_MAX_ATOMS = {"C": 3, "H": 4, "O": 3, "N": 2}
_MAX_TOTAL_ATOMS = 8


def _name(comp: dict[str, int], elements: list[str]) -> str:
    s = "".join(f"{e}{comp[e] if comp[e] > 1 else ''}" for e in elements if comp.get(e, 0) > 0)
    return s or "X"


def draw_species(rng: np.random.Generator, n_species: int, elements: list[str]):
    """Draw ``n_species`` distinct compositions over ``elements``.

    Returns (names, elem_count[S, E] int32, mw[S] kg/mol).  The base
    molecules H2, O2, N2, H2O (and CO, CO2 when carbon is present) come first;
    the rest are unique random compositions with at most 8 atoms.
    """
    comps: list[dict[str, int]] = []
    names: list[str] = []
    for nm, c in _BASE_SPECIES.items():
        if all(e in elements for e in c):
            comps.append({e: c.get(e, 0) for e in elements})
            names.append(nm)
    # Light radicals make balanced reactions plentiful; they are drawn like the
    # rest but offered first.
    seen = {tuple(c[e] for e in elements) for c in comps}
    tries = 0
    while len(comps) < n_species:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not draw enough distinct species")
        c = {e: int(rng.integers(0, _MAX_ATOMS[e] + 1)) for e in elements}
        tot = sum(c.values())
        if tot == 0 or tot > _MAX_TOTAL_ATOMS:
            continue
        key = tuple(c[e] for e in elements)
        if key in seen:
            continue
        seen.add(key)
        comps.append(c)
        names.append(_name(c, elements))
    comps = comps[:n_species]
    names = names[:n_species]
    elem = np.array([[c[e] for e in elements] for c in comps], dtype=np.int32)
    masses = np.array([ELEMENT_MASS_G[e] for e in elements]) * 1e-3  # kg/mol
    mw = elem.astype(np.float64) @ masses
    return names, elem, mw


def _multisets(n_species: int, max_size: int = 3):
    out = []
    for m in range(1, max_size + 1):
        out.extend(itertools.combinations_with_replacement(range(n_species), m))
    return out


def _balanced_partners(elem: np.ndarray):
    """Map every multiset of 1-3 species to the multisets with the same atom
    vector and no species in common (the candidate reverse sides)."""
    S = elem.shape[0]
    atoms = {}
    for m in _multisets(S):
        key = tuple(int(v) for v in elem[list(m)].sum(axis=0))
        atoms.setdefault(key, []).append(m)
    partners = {}
    for group in atoms.values():
        if len(group) < 2:
            continue
        for a in group:
            cands = [b for b in group if not (set(a) & set(b))]
            if cands:
                partners[a] = cands
    return partners


def draw_reactions(rng: np.random.Generator, elem: np.ndarray, n_reactions: int,
                   n_thirdbody: int, n_falloff: int, accept=None, max_tries: int = 400000):
    """Draw ``n_reactions`` atom-balanced reactions reactants -> products.

    Each side is a multiset of 1-3 species (so stoichiometric coefficients are
    at most 3); both sides carry the same atom vector, share no species, and no
    reaction (or its reverse) repeats.  Every species appears in at least one
    reaction.  ``n_thirdbody`` reactions are third-body (type 1) and
    ``n_falloff`` Lindemann fall-off (type 2); both are drawn from reactions
    whose two sides differ in molecularity.

    ``accept(reac, prod, rtype)`` (optional) returns the reaction's rate
    parameters, or None to discard the candidate; the caller uses it to shape
    the draw.  Returns (reac[R,3], prod[R,3] int32 padded with -1, rtype[R]
    uint8, params list).
    """
    S = elem.shape[0]
    partners = _balanced_partners(elem)
    keys = list(partners.keys())
    if not keys:
        raise RuntimeError("no balanced reactions exist for this species set")
    by_species = {k: [a for a in keys if k in a] for k in range(S)}
    missing = [k for k in range(S) if not by_species[k]]
    if missing:
        raise ValueError(f"species {missing} cannot appear in any balanced reaction")
    uneq_keys = [a for a in keys if any(len(b) != len(a) for b in partners[a])]

    chosen: list[tuple] = []
    params: list = []
    seen = set()
    tries = [0]

    def attempt(pool, rtype, need_unequal):
        tries[0] += 1
        if tries[0] > max_tries:
            raise RuntimeError("could not draw enough acceptable reactions")
        a = pool[int(rng.integers(len(pool)))]
        cands = partners[a]
        if need_unequal:
            cands = [b for b in cands if len(b) != len(a)]
            if not cands:
                return False
        b = cands[int(rng.integers(len(cands)))]
        if (a, b) in seen or (b, a) in seen:
            return False
        par = accept(a, b, rtype) if accept is not None else None
        if accept is not None and par is None:
            return False
        seen.add((a, b))
        chosen.append((a, b, rtype))
        params.append(par)
        return True

    covered = np.zeros(S, bool)
    for k in rng.permutation(S):
        if covered[k]:
            continue
        while not attempt(by_species[int(k)], 0, False):
            pass
        for s in chosen[-1][0] + chosen[-1][1]:
            covered[s] = True
    if not uneq_keys and (n_thirdbody + n_falloff) > 0:
        raise RuntimeError("no reactions with unequal molecularity")
    for rtype, count in ((1, n_thirdbody), (2, n_falloff)):
        for _ in range(count):
            while not attempt(uneq_keys, rtype, True):
                pass
    while len(chosen) < n_reactions:
        attempt(keys, 0, False)
    if len(chosen) > n_reactions:
        raise RuntimeError("coverage needs more reactions than requested")
    perm = rng.permutation(len(chosen))
    chosen = [chosen[i] for i in perm]
    params = [params[i] for i in perm]
    R = len(chosen)
    reac = -np.ones((R, 3), np.int32)
    prod = -np.ones((R, 3), np.int32)
    rtype = np.zeros(R, np.uint8)
    for i, (a, b, t) in enumerate(chosen):
        reac[i, : len(a)] = a
        prod[i, : len(b)] = b
        rtype[i] = t
    return reac, prod, rtype, params


def draw_arrhenius(rng: np.random.Generator, n_reac_side: int, rtype: int):
    """Draw one reaction's rate parameters.

    Returns (arrh[3], arrh0[3]) in SI units: A in (m^3/mol)^(order-1)/s,
    beta, Ea in J/mol.  ``order`` is the reactant molecularity, plus one for a
    third-body reaction.  For a Lindemann reaction ``arrh`` is the
    high-pressure limit and ``arrh0`` the low-pressure limit, whose A is
    10^U(2,6) times larger in units one order higher and whose Ea is uniform
    on [0, Ea].  A in cm-mol-s units is log-uniform on [1e6, 1e14].
    """
    order = n_reac_side + (1 if rtype == 1 else 0)
    a_cgs = 10.0 ** rng.uniform(6.0, 14.0)
    beta = rng.uniform(-1.0, 2.0)
    ea = rng.uniform(0.0, 200e3)
    arrh = np.array([a_cgs * (1e-6) ** (order - 1), beta, ea])
    arrh0 = np.zeros(3)
    if rtype == 2:
        a0_cgs = a_cgs * 10.0 ** rng.uniform(2.0, 6.0)
        arrh0 = np.array([a0_cgs * (1e-6) ** order, rng.uniform(-1.0, 2.0), rng.uniform(0.0, ea)])
    return arrh, arrh0


def draw_efficiencies(rng: np.random.Generator, n_species: int, rtype: np.ndarray):
    """Third-body efficiencies in CSR form: 3 species per type-1/2 reaction,
    each uniform on [0.4, 6]; every other species has efficiency 1."""
    ptr = [0]
    sp: list[int] = []
    val: list[float] = []
    for t in rtype:
        if t in (1, 2):
            pick = np.sort(rng.choice(n_species, size=min(3, n_species), replace=False))
            sp.extend(int(k) for k in pick)
            val.extend(float(v) for v in rng.uniform(0.4, 6.0, size=len(pick)))
        ptr.append(len(sp))
    return np.array(ptr, np.int32), np.array(sp, np.int32), np.array(val, np.float64)


def draw_thermo_raw(rng: np.random.Generator, names: list[str]):
    """Raw NASA-7 draws per species (not yet continuous at T_mid).

    Returns dict with ``high`` [S,5] (a1..a5 of the high range), ``dlow``
    [S,4] (perturbations of a2..a5 for the low range), ``dhf298`` [S] J/mol
    (zero for H2, O2, N2) and ``s298_r`` [S] (S(298 K)/R).
    """
    S = len(names)
    high = np.empty((S, 5))
    high[:, 0] = rng.uniform(2.5, 6.0, S)
    high[:, 1] = rng.uniform(-1e-3, 3e-3, S)
    high[:, 2] = rng.uniform(-1e-6, 1e-6, S)
    high[:, 3] = rng.uniform(-1e-10, 1e-10, S)
    high[:, 4] = rng.uniform(-1e-14, 1e-14, S)
    dlow = np.empty((S, 4))
    dlow[:, 0] = rng.uniform(-1e-3, 1e-3, S)
    dlow[:, 1] = rng.uniform(-1e-6, 1e-6, S)
    dlow[:, 2] = rng.uniform(-3e-10, 3e-10, S)
    dlow[:, 3] = rng.uniform(-3e-14, 3e-14, S)
    dhf = rng.uniform(-400e3, 400e3, S)
    for i, nm in enumerate(names):
        if nm in ("H2", "O2", "N2"):
            dhf[i] = 0.0
    s298 = rng.uniform(20.0, 40.0, S)
    return {"high": high, "dlow": dlow, "dhf298": dhf, "s298_r": s298}


def redraw_high(rng: np.random.Generator):
    """One fresh high-range a1..a5 draw (used when a species' heat capacity
    falls outside its bounds)."""
    return np.array([rng.uniform(2.5, 6.0), rng.uniform(-1e-3, 3e-3), rng.uniform(-1e-6, 1e-6),
                     rng.uniform(-1e-10, 1e-10), rng.uniform(-1e-14, 1e-14)])


def _groups(names: list[str], elem: np.ndarray, elements: list[str]):
    """Split species into fuel / oxidizer / product groups for blends."""
    idx = {e: i for i, e in enumerate(elements)}
    S = len(names)
    o2 = names.index("O2")
    n2 = names.index("N2")
    c = elem[:, idx["C"]] if "C" in idx else np.zeros(S, np.int32)
    h = elem[:, idx["H"]]
    o = elem[:, idx["O"]]
    # fuel: species with C or H and no O, richest in C then H (up to 3)
    cand = [k for k in range(S) if o[k] == 0 and (c[k] + h[k]) > 0]
    cand.sort(key=lambda k: (-int(c[k]), -int(h[k]), k))
    fuel = cand[:3] if cand else [names.index("H2")]
    oxid = [o2, n2]
    prod = [k for k in range(S) if k not in fuel and k not in oxid]
    return fuel, oxid, prod


def draw_states(rng: np.random.Generator, names, elem, mw, elements, n: int,
                t_range=(1000.0, 2500.0), p_range_atm=(1.0, 20.0)):
    """Reactor states: T and p uniform on their ranges, Y a random blend.

    Y: Dirichlet(1,1,1) weights over {fuel, oxidizer, products}; oxidizer is
    O2 + N2 at 3.76:1 molar; fuel and product mass is spread over their
    species with uniform random weights.  Returns (y[n, S+1] with column 0 = T
    in K, p[n] in Pa).
    """
    S = len(names)
    fuel, oxid, prod = _groups(names, elem, elements)
    T = rng.uniform(t_range[0], t_range[1], n)
    p = rng.uniform(p_range_atm[0], p_range_atm[1], n) * ATM
    w = rng.dirichlet([1.0, 1.0, 1.0], n)
    Y = np.zeros((n, S))
    fw = rng.uniform(0.0, 1.0, (n, len(fuel)))
    fw /= fw.sum(axis=1, keepdims=True)
    Y[:, fuel] += w[:, :1] * fw
    air = np.array([1.0 * mw[oxid[0]], 3.76 * mw[oxid[1]]])
    air /= air.sum()
    Y[:, oxid] += w[:, 1:2] * air[None, :]
    if prod:
        pw = rng.uniform(0.0, 1.0, (n, len(prod)))
        pw /= pw.sum(axis=1, keepdims=True)
        Y[:, prod] += w[:, 2:3] * pw
    else:
        Y[:, fuel] += w[:, 2:3] * fw
    Y /= Y.sum(axis=1, keepdims=True)
    y = np.empty((n, S + 1))
    y[:, 0] = T
    y[:, 1:] = Y
    return y, p


def draw_densities(rng: np.random.Generator, n: int, rho_range=(0.1, 3.0)) -> np.ndarray:
    """Fixed densities of constant-volume reactors, log-uniform in kg/m^3
    (0.1-3 kg/m^3 spans about 0.3-25 atm over 1000-2500 K)."""
    lo, hi = np.log(rho_range[0]), np.log(rho_range[1])
    return np.exp(rng.uniform(lo, hi, n))


def pick_reactions(rng: np.random.Generator, rev: np.ndarray, frac: float) -> np.ndarray:
    """A random subset (fraction frac) of the reversible reactions."""
    idx = np.flatnonzero(np.asarray(rev) != 0)
    k = int(round(frac * len(idx)))
    return np.sort(rng.choice(idx, size=k, replace=False)) if k else np.zeros(0, int)
