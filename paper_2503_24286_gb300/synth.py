"""Seeded synthetic mechanisms and thermochemical states.

This module only *draws* data: species compositions, NASA-7 coefficient sets,
reaction shapes and rate parameters, and random states (T, p, Y).  It holds
none of the arithmetic the library evaluates (no rate constants, equilibrium
constants, production rates, energies or densities); both the CUDA library and
the CPU oracle read what it writes and evaluate the method independently.

Mechanism shape follows the problem statement of the paper's formulation
appendix (Sec. A.1, Eqs. for reactions / mass action / Arrhenius / Troe falloff
and the NASA polynomials of Sec. A.1); parameter distributions are those of the
synthetic workloads:

* elements with standard atomic weights; species of small compositions;
* two-range NASA-7 fits (T_mid = 1000 K) to smooth positive cp/R curves built
  from rigid-rotor / harmonic-oscillator (Einstein-function) models, with cp
  continuous to first derivative and h, s continuous at T_mid;
* element-balanced reversible reactions with 1-3 species a side (coefficients
  1 or 2, order <= 3), optional third-body efficiencies U[0.5, 12] on up to 8
  species, Troe falloff, and duplicate pairs;
* states: T ~ U, p ~ U (atm), Y ~ Dirichlet(0.5);
* transport fits of the form the paper's mixture-averaged model takes (Sec. A.2):
  species viscosity sqrt(T) (sum_m b_m ln^m T)^2, conductivity
  sqrt(T) sum_m c_m ln^m T and binary diffusivity sqrt(T) sum_m a_m ln^m T,
  m = 0..4, least-squares fitted on [250, 3600] K to Chapman-Enskog-type model
  curves (Lennard-Jones parameters drawn per species, Neufeld-Janzen-Aziz
  collision integrals, Eucken-type conductivity, diffusivity at 1 atm).  The
  model curves are only the fitting targets; the library and the oracle
  evaluate the fits and the mixture rules.

The text format written by :func:`write_mechanism` is the interchange format
of the library (``pyro_mech_load``) and the oracle; see ``MECH_FORMAT``.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

ATOMIC_WEIGHTS: Dict[str, float] = {
    "H": 1.008,
    "C": 12.011,
    "N": 14.007,
    "O": 15.999,
    "Ar": 39.95,
}

# Element-reference forms (formation enthalpy zero).
REFERENCE_FORMS: Dict[str, Dict[str, int]] = {
    "H": {"H": 2},
    "O": {"O": 2},
    "N": {"N": 2},
    "C": {"C": 1},
    "Ar": {"Ar": 1},
}

T_LOW, T_MID, T_HIGH = 200.0, 1000.0, 3500.0
ONE_ATM = 101325.0

MECH_FORMAT = """\
pyro-mech 1
name <text>
elements <E>
element <symbol> <atomic weight>                       (E lines)
species <N>
species <name> <n> <sym> <count> ... <sym> <count>      (N lines, composition)
thermo <k> <T_low> <T_mid> <T_high> <a1..a7 low> <a1..a7 high>   (N lines)
reactions <M>
reaction <kind> rev <0|1> dup <0|1> reac <n> <k> <nu> ... prod <n> <k> <nu> ...
         arr <A> <b> <theta>
         [eff <n> <k> <eps> ...] [low <A0> <b0> <theta0>] [troe <a> <T3> <T1> [<T2>]]
         [sri <a> <b> <c> [<d> <e>]] [plog <n> <p> <A> <b> <theta> ...] end
[transport <N>                                           (optional section)
 tspecies <k> <b0..b4> <c0..c4>                          (N lines: viscosity, conductivity)
 tbinary <k> <j> <a0..a4>                                (k < j, N(N-1)/2 lines: diffusivity)]
kind in {arrhenius, threebody, falloff, plog}; theta = Ea/R in K; SI kmol units.
A falloff reaction carries troe or sri data (neither: Lindemann); a plog
reaction lists its pressure nodes (Pa, increasing) and its arr data is unused.
All reals are written with 17 significant digits (exact round trip).
"""


@dataclass
class Species:
    name: str
    composition: Dict[str, int]
    nasa_low: List[float]
    nasa_high: List[float]
    t_low: float = T_LOW
    t_mid: float = T_MID
    t_high: float = T_HIGH
    h298: Optional[float] = None    # h(298.15 K)/R [K] the fit was anchored to (not in the file)
    s298: Optional[float] = None    # s(298.15 K)/R the fit was anchored to (not in the file)


@dataclass
class Reaction:
    kind: str                                   # arrhenius | threebody | falloff
    reactants: List[Tuple[int, int]]            # (species index, coefficient)
    products: List[Tuple[int, int]]
    A: float
    b: float
    theta: float                                # activation temperature Ea/R [K]
    reversible: bool = True
    duplicate: bool = False
    efficiencies: Dict[int, float] = field(default_factory=dict)
    low: Optional[Tuple[float, float, float]] = None       # k0 (A0, b0, theta0)
    troe: Optional[Tuple[float, ...]] = None               # (a, T3, T1[, T2])
    sri: Optional[Tuple[float, ...]] = None                # falloff SRI (a, b, c[, d, e])
    plog: Optional[List[Tuple[float, float, float, float]]] = None   # kind plog: (p [Pa], A, b, theta)


@dataclass
class Transport:
    """Polynomial transport fits (Sec. A.2), coefficients of ln^m T, m = 0..4."""
    visc: np.ndarray       # [N, 5]: mu_k = sqrt(T) (sum_m b_km ln^m T)^2        [Pa s]
    cond: np.ndarray       # [N, 5]: kappa_k = sqrt(T) sum_m c_km ln^m T          [W/(m K)]
    diff: np.ndarray       # [N, N, 5] symmetric: D_kj = sqrt(T) sum_m a_kjm ln^m T  [m^2/s]


@dataclass
class Mechanism:
    name: str
    elements: List[Tuple[str, float]]
    species: List[Species]
    reactions: List[Reaction]
    transport: Optional[Transport] = None

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return len(self.reactions)


# ----------------------------------------------------------------------------
# Workload table (synthetic stand-ins for the paper's H2/air and GRI-3.0-sized
# mechanisms).
# ----------------------------------------------------------------------------

CONFIGS = {
    0: dict(name="h2air-10sp", mech=0, elements=["H", "O", "N"], n_species=10,
            n_reactions=21, n_threebody=4, n_falloff=2, n_dup_pairs=0,
            inert=[{"N": 2}], n_points=4096, T=(300.0, 2500.0), p_atm=(1.0, 1.0)),
    1: dict(name="gri-53sp", mech=1, elements=["C", "H", "O", "N", "Ar"], n_species=53,
            n_reactions=325, n_threebody=30, n_falloff=25, n_dup_pairs=28,
            inert=[{"Ar": 1}], n_points=2 ** 22, T=(300.0, 2800.0), p_atm=(0.5, 20.0)),
    2: dict(name="gri-53sp-jacobian", mech=1, n_points=2 ** 20,
            T=(300.0, 2800.0), p_atm=(0.5, 20.0)),
    3: dict(name="gri-53sp-learned-guess", mech=1, n_points=2 ** 22, n_train=2 ** 24,
            T=(300.0, 2800.0), p_atm=(0.5, 20.0)),
    4: dict(name="large-160sp", mech=4, elements=["C", "H", "O", "N"], n_species=160,
            n_reactions=1100, n_threebody=80, n_falloff=60, n_dup_pairs=0,
            inert=[], n_points=2 ** 21, T=(300.0, 2800.0), p_atm=(1.0, 40.0)),
    # Crank-Nicolson step (Sec. A.3.2) on the 53-species mechanism.  The synthetic
    # kinetics (log10 A up to 16, b up to 3, random formation enthalpies) put the
    # fastest chemical time scales near 1e-40 s at 2000-2800 K, so the step size
    # is set on that scale: dt = 3e-41 s gives dt |lambda_max| from ~1e-3 up to
    # ~10 across the states (the stiff regime an implicit step is for) while the
    # Newton iteration from Y^m still converges for every state of the batch.
    5: dict(name="gri-53sp-crank-nicolson", mech=1, n_points=2 ** 18, T=(2000.0, 2800.0),
            p_atm=(0.5, 20.0), dt=3.0e-41),
    # the same for the 10-species mechanism (fastest scales ~1e-31 s at 1500-2500 K)
    6: dict(name="h2air-10sp-crank-nicolson", mech=0, n_points=4096, T=(1500.0, 2500.0),
            p_atm=(1.0, 1.0), dt=1.0e-31),
    # other pressure-dependent forms: the 53-species mechanism with 10 of its Troe
    # falloff reactions given SRI data instead and 20 plain reactions turned into
    # PLOG reactions (3-5 pressure nodes between 0.1 and 100 atm)
    7: dict(name="gri-53sp-pdep", mech=7, base=1, n_sri=10, n_plog=20, n_points=2 ** 22,
            T=(300.0, 2800.0), p_atm=(0.5, 20.0)),
    # Crank-Nicolson step on the 160-species mechanism (161 x 161 Newton systems with
    # the temperature row folded out: 160 x 160).  Its gross rates reach ~1e42
    # kmol/m^3/s at 2000-2800 K, six orders above the 53-species mechanism's, so
    # the step is dt = 1e-46 s (T moves by up to ~10 K, Newton converges in 3-7 steps).
    8: dict(name="large-160sp-crank-nicolson", mech=4, n_points=2 ** 14, T=(2000.0, 2800.0),
            p_atm=(1.0, 40.0), dt=1.0e-46),
}
PDEP_SEED_OFFSET = 2000

MECH_SEED_BASE = 2503
STATE_SEED_BASE = 24286


TRANSPORT_SEED_OFFSET = 1000


def config_mechanism(index: int) -> Mechanism:
    """The synthetic mechanism of workload ``index`` (seed 2503 + mechanism index),
    with transport fits drawn from a separate stream (seed 3503 + mechanism index)."""
    cfg = CONFIGS[index]
    m = CONFIGS[cfg["mech"]]
    if "base" in m:
        return pressure_dependent_variant(config_mechanism(m["base"]), m["n_sri"], m["n_plog"],
                                          MECH_SEED_BASE + PDEP_SEED_OFFSET + cfg["mech"], m["name"])
    mech = generate_mechanism(
        name=m["name"], elements=m["elements"], n_species=m["n_species"],
        n_reactions=m["n_reactions"], n_threebody=m["n_threebody"],
        n_falloff=m["n_falloff"], n_dup_pairs=m["n_dup_pairs"], inert=m["inert"],
        seed=MECH_SEED_BASE + cfg["mech"])
    mech.transport = generate_transport(mech, MECH_SEED_BASE + TRANSPORT_SEED_OFFSET + cfg["mech"])
    return mech


# ----------------------------------------------------------------------------
# Species
# ----------------------------------------------------------------------------

# small molecules placed before the random fill (H2/air and C1-C2/N chemistry)
PRESET_FORMULAS = ["OH", "H2O", "HO2", "H2O2", "CH", "CH2", "CH3", "CH4", "CO", "CO2",
                   "HCO", "CH2O", "CH3O", "CH3OH", "C2H2", "C2H4", "C2H6", "NH", "NO",
                   "NO2", "N2O", "HCN", "HNO", "C2H3", "C2H5", "HCCO", "CH2CO", "NH2",
                   "NH3", "CN"]


def parse_formula(f: str) -> Dict[str, int]:
    """'CH2O' -> {'C': 1, 'H': 2, 'O': 1}."""
    out: Dict[str, int] = {}
    i = 0
    while i < len(f):
        e = f[i]
        i += 1
        if i < len(f) and f[i].islower():
            e += f[i]
            i += 1
        j = i
        while j < len(f) and f[j].isdigit():
            j += 1
        out[e] = out.get(e, 0) + (int(f[i:j]) if j > i else 1)
        i = j
    return out


_COUNT_LIMITS = {"C": 3, "H": 8, "O": 3, "N": 2, "Ar": 0}
_COUNT_LIMITS_LARGE = {"C": 7, "H": 16, "O": 4, "N": 3, "Ar": 0}


def _formula(comp: Dict[str, int], order: Sequence[str]) -> str:
    s = ""
    for e in order:
        c = comp.get(e, 0)
        if c:
            s += e + (str(c) if c > 1 else "")
    return s


def _draw_compositions(rng: np.random.Generator, elements: List[str], n: int,
                       inert: List[Dict[str, int]]) -> List[Dict[str, int]]:
    comps: List[Dict[str, int]] = []
    seen = set()

    def add(c):
        key = tuple(sorted(c.items()))
        if key not in seen:
            seen.add(key)
            comps.append(dict(c))

    # inert species first, then element references, atoms and common molecules
    for c in inert:
        add(c)
    for e in elements:
        add(REFERENCE_FORMS[e])
    for e in elements:
        if e != "Ar":
            add({e: 1})
    for f in PRESET_FORMULAS:
        c = parse_formula(f)
        if set(c) <= set(elements) and len(comps) < n:
            add(c)
    limits = _COUNT_LIMITS if n <= 60 else _COUNT_LIMITS_LARGE
    active = [e for e in elements if e != "Ar"]
    tries = 0
    while len(comps) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not draw enough distinct compositions")
        c = {}
        for e in active:
            lim = limits[e]
            # geometric-ish preference for small counts
            k = int(min(lim, rng.geometric(0.45) - 1))
            if k:
                c[e] = k
        tot = sum(c.values())
        if tot < 2 or tot > (9 if n <= 60 else 14):
            continue
        add(c)
    return comps[:n]


def _einstein(x: np.ndarray) -> np.ndarray:
    ex = np.exp(-x)
    return x * x * ex / (1.0 - ex) ** 2


def _cp_model(rng: np.random.Generator, comp: Dict[str, int]):
    """A smooth positive cp/R(T) curve: translation + rotation + harmonic modes."""
    n_atoms = sum(comp.values())
    if n_atoms == 1:
        return lambda T: np.full_like(np.asarray(T, dtype=float), 2.5)
    linear = n_atoms == 2 or rng.random() < 0.2
    rot = 1.0 if linear else 1.5
    n_vib = 3 * n_atoms - (5 if linear else 6)
    thetas = rng.uniform(400.0, 5000.0, size=n_vib)

    def cp(T):
        T = np.asarray(T, dtype=float)
        out = np.full_like(T, 2.5 + rot)
        for th in thetas:
            out = out + _einstein(th / T)
        return out
    return cp


def _fit_nasa(cp, h298: float, s298: float) -> Tuple[List[float], List[float]]:
    """Least-squares NASA-7 fit of cp/R with C1 continuity of cp at T_mid and
    C0 continuity of h and s at T_mid (data preparation, not library arithmetic)."""
    Tl = np.linspace(T_LOW, T_MID, 161)
    V = np.vander(Tl, 5, increasing=True)
    lo = np.linalg.lstsq(V, cp(Tl), rcond=None)[0]
    # value and slope of the low fit at T_mid
    c_mid = sum(lo[m] * T_MID ** m for m in range(5))
    d_mid = sum(m * lo[m] * T_MID ** (m - 1) for m in range(1, 5))
    Th = np.linspace(T_MID, T_HIGH, 201)
    u = Th - T_MID
    # cp_hi = c_mid + d_mid u + u^2 (q0 + q1 u + q2 u^2)
    B = np.stack([u ** 2, u ** 3, u ** 4], axis=1)
    q = np.linalg.lstsq(B, cp(Th) - c_mid - d_mid * u, rcond=None)[0]
    # expand the polynomial in u = T - T_mid to monomials in T
    poly_u = np.array([c_mid, d_mid, q[0], q[1], q[2]])
    hi = np.zeros(5)
    for m, cm in enumerate(poly_u):
        for i in range(m + 1):
            hi[i] += cm * math.comb(m, i) * (-T_MID) ** (m - i)
    # integration constants from h(298.15), s(298.15) and continuity at T_mid
    def h_int(a, T):  # integral of cp/R dT, without constant
        return sum(a[m] * T ** (m + 1) / (m + 1) for m in range(5))

    def s_int(a, T):  # integral of cp/(R T) dT, without constant
        return a[0] * math.log(T) + sum(a[m] * T ** m / m for m in range(1, 5))
    T0 = 298.15
    a6_lo = h298 - h_int(lo, T0)
    a7_lo = s298 - s_int(lo, T0)
    a6_hi = h_int(lo, T_MID) + a6_lo - h_int(hi, T_MID)
    a7_hi = s_int(lo, T_MID) + a7_lo - s_int(hi, T_MID)
    return ([float(x) for x in lo] + [float(a6_lo), float(a7_lo)],
            [float(x) for x in hi] + [float(a6_hi), float(a7_hi)])


def _cp_poly_min(a_lo, a_hi) -> float:
    T1 = np.linspace(100.0, T_MID, 400)
    T2 = np.linspace(T_MID, 5000.0, 800)
    c1 = sum(a_lo[m] * T1 ** m for m in range(5))
    c2 = sum(a_hi[m] * T2 ** m for m in range(5))
    return float(min(c1.min(), c2.min()))


# ----------------------------------------------------------------------------
# Reactions
# ----------------------------------------------------------------------------

def _side_multisets(reactive: List[int], max_order: int):
    """All multisets of reactive species with order <= max_order, coefficients 1-2."""
    out = []
    for order in range(1, max_order + 1):
        for combo in itertools.combinations_with_replacement(reactive, order):
            counts: Dict[int, int] = {}
            for k in combo:
                counts[k] = counts.get(k, 0) + 1
            if max(counts.values()) > 2:
                continue
            out.append(tuple(sorted(counts.items())))
    return out


def _element_key(side, comps, elements):
    v = [0] * len(elements)
    for k, nu in side:
        for i, e in enumerate(elements):
            v[i] += nu * comps[k].get(e, 0)
    return tuple(v)


def generate_mechanism(name: str, elements: List[str], n_species: int, n_reactions: int,
                       n_threebody: int, n_falloff: int, n_dup_pairs: int,
                       inert: List[Dict[str, int]], seed: int) -> Mechanism:
    rng = np.random.default_rng(seed)
    comps = _draw_compositions(rng, elements, n_species, inert)
    order = [e for e in ["C", "H", "O", "N", "Ar"] if e in elements]
    names = [_formula(c, order) for c in comps]
    refs = [tuple(sorted(REFERENCE_FORMS[e].items())) for e in elements]

    species: List[Species] = []
    for c, nm in zip(comps, names):
        key = tuple(sorted(c.items()))
        h298 = 0.0 if key in refs else float(rng.uniform(-3.0e4, 3.0e4))
        s298 = float(rng.uniform(15.0, 35.0))
        for _ in range(100):
            cp = _cp_model(rng, c)
            lo, hi = _fit_nasa(cp, h298, s298)
            if _cp_poly_min(lo, hi) >= 1.5:
                break
        else:
            raise RuntimeError("NASA fit with cp/R >= 1.5 not found")
        species.append(Species(nm, c, lo, hi, h298=h298, s298=s298))

    inert_keys = [tuple(sorted(c.items())) for c in inert]
    reactive = [k for k, c in enumerate(comps) if tuple(sorted(c.items())) not in inert_keys]

    # candidate sides grouped by element vector; a reaction pairs two disjoint
    # sides of one group (exact integer element balance)
    groups: Dict[Tuple[int, ...], List] = {}
    for side in _side_multisets(reactive, 3):
        groups.setdefault(_element_key(side, comps, elements), []).append(side)
    # pools of groups per (reactant order, product order)
    by_orders: Dict[Tuple[int, int], List[Tuple[List, List]]] = {}
    for g in groups.values():
        if len(g) < 2:
            continue
        by_o: Dict[int, List] = {}
        for sd in g:
            by_o.setdefault(sum(n for _, n in sd), []).append(sd)
        for o1 in by_o:
            for o2 in by_o:
                if o1 == o2 and len(by_o[o1]) < 2:
                    continue
                by_orders.setdefault((o1, o2), []).append((by_o[o1], by_o[o2]))
    used = set()

    def take(weights):
        keys = [k for k in weights if k in by_orders]
        w = np.array([weights[k] for k in keys], dtype=float)
        w /= w.sum()
        for _ in range(200000):
            o = keys[int(rng.choice(len(keys), p=w))]
            pool = by_orders[o]
            ga, gb = pool[int(rng.integers(len(pool)))]
            a = ga[int(rng.integers(len(ga)))]
            b = gb[int(rng.integers(len(gb)))]
            if a == b or set(k for k, _ in a) & set(k for k, _ in b):
                continue
            key = (a, b) if a < b else (b, a)
            if key in used:
                continue
            used.add(key)
            return [tuple(x) for x in a], [tuple(x) for x in b]
        raise RuntimeError("not enough element-balanced reaction shapes")

    pairs3 = {(2, 2): 0.55, (1, 2): 0.1, (2, 1): 0.1, (2, 3): 0.1, (3, 2): 0.1, (3, 3): 0.05}
    pairs2 = {(1, 2): 0.4, (2, 1): 0.4, (2, 2): 0.2}

    def arrhenius():
        return (float(10.0 ** rng.uniform(8.0, 16.0)), float(rng.uniform(-2.0, 3.0)),
                float(rng.uniform(0.0, 3.0e4)))

    def efficiencies():
        n_eff = min(n_species, 8)
        idx = rng.choice(n_species, size=n_eff, replace=False)
        return {int(k): float(rng.uniform(0.5, 12.0)) for k in sorted(idx)}

    reactions: List[Reaction] = []
    n_plain = n_reactions - n_threebody - n_falloff - 2 * n_dup_pairs
    if n_plain < 0:
        raise ValueError("reaction counts do not add up")
    for _ in range(n_threebody):
        r, p = take(pairs2)
        A, b, th = arrhenius()
        reactions.append(Reaction("threebody", r, p, A, b, th, efficiencies=efficiencies()))
    for i in range(n_falloff):
        r, p = take(pairs2)
        A, b, th = arrhenius()
        low = (float(A * 10.0 ** rng.uniform(2.0, 5.0)), float(rng.uniform(-2.0, 0.0)),
               float(rng.uniform(0.0, 1.0e4)))
        troe = [float(rng.uniform(0.1, 0.9)), float(rng.uniform(30.0, 300.0)),
                float(rng.uniform(500.0, 3000.0))]
        if i % 2 == 0:
            troe.append(float(rng.uniform(3000.0, 8000.0)))
        reactions.append(Reaction("falloff", r, p, A, b, th, efficiencies=efficiencies(),
                                  low=low, troe=tuple(troe)))
    for _ in range(n_dup_pairs):
        r, p = take(pairs3)
        for _k in range(2):
            A, b, th = arrhenius()
            reactions.append(Reaction("arrhenius", r, p, A, b, th, duplicate=True))
    for _ in range(n_plain):
        r, p = take(pairs3)
        A, b, th = arrhenius()
        reactions.append(Reaction("arrhenius", r, p, A, b, th))
    # interleave kinds deterministically (a mechanism file is not sorted by kind)
    perm = rng.permutation(len(reactions))
    # keep duplicate pairs adjacent
    order_r: List[int] = []
    placed = set()
    for i in perm:
        if i in placed:
            continue
        rx = reactions[i]
        order_r.append(int(i))
        placed.add(int(i))
        if rx.duplicate:
            # its partner shares stoichiometry
            for j in range(len(reactions)):
                if j not in placed and reactions[j].duplicate and \
                        reactions[j].reactants == rx.reactants and reactions[j].products == rx.products:
                    order_r.append(j)
                    placed.add(j)
                    break
    reactions = [reactions[i] for i in order_r]
    elems = [(e, ATOMIC_WEIGHTS[e]) for e in elements]
    return Mechanism(name, elems, species, reactions)


def pressure_dependent_variant(base: Mechanism, n_sri: int, n_plog: int, seed: int, name: str) -> Mechanism:
    """A copy of ``base`` with the first ``n_sri`` Troe falloff reactions given SRI
    data (a ~ U[0.1, 2], b ~ U[100, 1000] K, c ~ U[100, 3000] K; d ~ U[0.5, 2],
    e ~ U[-0.5, 0.5] on every other one) and the first ``n_plog`` plain
    non-duplicate reactions turned into PLOG reactions with 3-5 pressure nodes
    log-uniform in [0.1, 100] atm, each node's Arrhenius data the reaction's own
    with A x 10^U[-1, 1], b + U[-0.3, 0.3], theta + U[-1000, 1000] K (>= 0)."""
    import copy
    rng = np.random.default_rng(seed)
    mech = copy.deepcopy(base)
    mech.name = name
    falloff = [r for r in mech.reactions if r.kind == "falloff" and r.troe is not None]
    for q, r in enumerate(falloff[:n_sri]):
        a, b, c = float(rng.uniform(0.1, 2.0)), float(rng.uniform(100.0, 1000.0)), float(rng.uniform(100.0, 3000.0))
        r.troe = None
        r.sri = (a, b, c, float(rng.uniform(0.5, 2.0)), float(rng.uniform(-0.5, 0.5))) if q % 2 == 0 else (a, b, c)
    plain = [r for r in mech.reactions if r.kind == "arrhenius" and not r.duplicate]
    for r in plain[:n_plog]:
        nn = int(rng.integers(3, 6))
        lp = np.sort(rng.uniform(np.log(0.1), np.log(100.0), size=nn))
        nodes = []
        for q in range(nn):
            nodes.append((float(np.exp(lp[q]) * ONE_ATM), float(r.A * 10.0 ** rng.uniform(-1.0, 1.0)),
                          float(r.b + rng.uniform(-0.3, 0.3)), float(max(0.0, r.theta + rng.uniform(-1000.0, 1000.0)))))
        r.kind = "plog"
        r.plog = nodes
    return mech


# ----------------------------------------------------------------------------
# Transport fits
# ----------------------------------------------------------------------------

R_UNIV = 8314.462618          # J/(kmol K), for the Eucken-type model only
TR_FIT_T = (250.0, 3600.0)


def _omega22(ts: np.ndarray) -> np.ndarray:
    """Reduced collision integral Omega(2,2)* of the Lennard-Jones potential
    (Neufeld, Janzen and Aziz, J. Chem. Phys. 57, 1100 (1972))."""
    return 1.16145 * ts ** -0.14874 + 0.52487 * np.exp(-0.77320 * ts) + 2.16178 * np.exp(-2.43787 * ts)


def _omega11(ts: np.ndarray) -> np.ndarray:
    """Reduced collision integral Omega(1,1)* (same reference)."""
    return (1.06036 * ts ** -0.15610 + 0.19300 * np.exp(-0.47635 * ts) + 1.03587 * np.exp(-1.52996 * ts)
            + 1.76474 * np.exp(-3.89411 * ts))


@dataclass
class TransportModel:
    """Per-species model parameters the fits are drawn from (not in the file)."""
    W: np.ndarray          # kg/kmol
    sigma: np.ndarray      # Lennard-Jones diameter [Angstrom]
    eps: np.ndarray        # well depth / k_B [K]
    cint: np.ndarray       # internal-mode weight of the conductivity model
    theta: np.ndarray      # internal-mode temperature of the conductivity model [K]

    def viscosity(self, T: np.ndarray) -> np.ndarray:
        """[N, nT] Chapman-Enskog viscosity [Pa s]."""
        T = np.asarray(T, dtype=float)
        ts = T[None, :] / self.eps[:, None]
        return 2.6693e-6 * np.sqrt(self.W[:, None] * T[None, :]) / (self.sigma[:, None] ** 2 * _omega22(ts))

    def conductivity(self, T: np.ndarray) -> np.ndarray:
        """[N, nT] Eucken-type conductivity [W/(m K)]: (mu/W) R (15/4 + internal part)."""
        T = np.asarray(T, dtype=float)
        f = 3.75 + self.cint[:, None] * (1.0 - np.exp(-T[None, :] / self.theta[:, None]))
        return self.viscosity(T) / self.W[:, None] * R_UNIV * f

    def diffusivity(self, T: np.ndarray) -> np.ndarray:
        """[N, N, nT] Chapman-Enskog binary diffusivity at 1 atm [m^2/s]."""
        T = np.asarray(T, dtype=float)
        sig = 0.5 * (self.sigma[:, None] + self.sigma[None, :])
        eps = np.sqrt(self.eps[:, None] * self.eps[None, :])
        wr = 1.0 / self.W[:, None] + 1.0 / self.W[None, :]
        ts = T[None, None, :] / eps[:, :, None]
        return 1.8583e-7 * np.sqrt(T[None, None, :] ** 3 * wr[:, :, None]) / (sig[:, :, None] ** 2 * _omega11(ts))


def transport_model(mech: Mechanism, seed: int) -> TransportModel:
    """Seeded Lennard-Jones and conductivity-model parameters of every species."""
    rng = np.random.default_rng(seed)
    ew = dict(mech.elements)
    W = np.array([sum(c * ew[e] for e, c in s.composition.items()) for s in mech.species])
    atoms = np.array([sum(s.composition.values()) for s in mech.species], dtype=float)
    sigma = 2.6 + 0.45 * np.sqrt(atoms) + rng.uniform(-0.2, 0.2, size=atoms.size)
    eps = (90.0 + 55.0 * atoms ** 0.7) * rng.uniform(0.7, 1.3, size=atoms.size)
    cint = np.where(atoms > 1, rng.uniform(0.5, 4.0, size=atoms.size), 0.0)
    theta = rng.uniform(300.0, 2000.0, size=atoms.size)
    return TransportModel(W, sigma, eps, cint, theta)


def _fit_lnT(T: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Least-squares coefficients of sum_m c_m ln^m T (m = 0..4), rows of y fitted independently."""
    V = np.vander(np.log(T), 5, increasing=True)
    c, *_ = np.linalg.lstsq(V, y.T, rcond=None)
    return np.ascontiguousarray(c.T)


def generate_transport(mech: Mechanism, seed: int) -> Transport:
    """Transport fits of every species and species pair (Sec. A.2 forms)."""
    mdl = transport_model(mech, seed)
    T = np.exp(np.linspace(math.log(TR_FIT_T[0]), math.log(TR_FIT_T[1]), 48))
    sq = np.sqrt(T)[None, :]
    visc = _fit_lnT(T, np.sqrt(mdl.viscosity(T) / sq))
    cond = _fit_lnT(T, mdl.conductivity(T) / sq)
    N = mech.n_species
    D = mdl.diffusivity(T) / sq[None]
    diff = _fit_lnT(T, D.reshape(N * N, -1)).reshape(N, N, 5)
    diff = 0.5 * (diff + diff.transpose(1, 0, 2))          # exactly symmetric
    diff[np.arange(N), np.arange(N)] = 0.0                  # self-diffusion is not used (j != k)
    return Transport(visc, cond, diff)


# ----------------------------------------------------------------------------
# File format
# ----------------------------------------------------------------------------

def _f(x: float) -> str:
    return "%.17g" % x


def write_mechanism(mech: Mechanism, path: str) -> None:
    lines = ["pyro-mech 1", "name " + mech.name, "elements %d" % len(mech.elements)]
    for e, w in mech.elements:
        lines.append("element %s %s" % (e, _f(w)))
    lines.append("species %d" % mech.n_species)
    for s in mech.species:
        items = [(e, c) for e, c in s.composition.items() if c]
        lines.append("species %s %d %s" % (s.name, len(items),
                                           " ".join("%s %d" % (e, c) for e, c in items)))
    for k, s in enumerate(mech.species):
        lines.append("thermo %d %s %s %s %s %s" % (
            k, _f(s.t_low), _f(s.t_mid), _f(s.t_high),
            " ".join(_f(a) for a in s.nasa_low), " ".join(_f(a) for a in s.nasa_high)))
    lines.append("reactions %d" % mech.n_reactions)
    for r in mech.reactions:
        parts = ["reaction", r.kind, "rev", "1" if r.reversible else "0",
                 "dup", "1" if r.duplicate else "0",
                 "reac", str(len(r.reactants))]
        for k, nu in r.reactants:
            parts += [str(k), str(nu)]
        parts += ["prod", str(len(r.products))]
        for k, nu in r.products:
            parts += [str(k), str(nu)]
        parts += ["arr", _f(r.A), _f(r.b), _f(r.theta)]
        if r.efficiencies:
            parts += ["eff", str(len(r.efficiencies))]
            for k, e in sorted(r.efficiencies.items()):
                parts += [str(k), _f(e)]
        if r.low is not None:
            parts += ["low"] + [_f(x) for x in r.low]
        if r.troe is not None:
            parts += ["troe"] + [_f(x) for x in r.troe]
        if r.sri is not None:
            parts += ["sri"] + [_f(x) for x in r.sri]
        if r.plog is not None:
            parts += ["plog", str(len(r.plog))]
            for node in r.plog:
                parts += [_f(x) for x in node]
        parts.append("end")
        lines.append(" ".join(parts))
    tr = mech.transport
    if tr is not None:
        lines.append("transport %d" % mech.n_species)
        for k in range(mech.n_species):
            lines.append("tspecies %d %s %s" % (k, " ".join(_f(x) for x in tr.visc[k]),
                                                " ".join(_f(x) for x in tr.cond[k])))
        for k in range(mech.n_species):
            for j in range(k + 1, mech.n_species):
                lines.append("tbinary %d %d %s" % (k, j, " ".join(_f(x) for x in tr.diff[k, j])))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def read_mechanism(path: str) -> Mechanism:
    """Parse the text format back into a :class:`Mechanism` (used by tooling and tests)."""
    with open(path) as f:
        toks = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    it = iter(toks)
    hdr = next(it)
    if hdr[:2] != ["pyro-mech", "1"]:
        raise ValueError("not a pyro-mech v1 file")
    name = " ".join(next(it)[1:])
    ne = int(next(it)[1])
    elements = []
    for _ in range(ne):
        t = next(it)
        elements.append((t[1], float(t[2])))
    ns = int(next(it)[1])
    sp = []
    for _ in range(ns):
        t = next(it)
        n = int(t[2])
        comp = {t[3 + 2 * i]: int(t[4 + 2 * i]) for i in range(n)}
        sp.append([t[1], comp])
    species = []
    for k in range(ns):
        t = next(it)
        v = [float(x) for x in t[2:]]
        species.append(Species(sp[k][0], sp[k][1], v[3:10], v[10:17], v[0], v[1], v[2]))
    nr = int(next(it)[1])
    reactions = []
    for _ in range(nr):
        t = next(it)
        kind = t[1]
        i = 2
        rev = dup = False
        reac, prod = [], []
        A = b = th = 0.0
        eff, low, troe, sri, plog = {}, None, None, None, None
        while t[i] != "end":
            key = t[i]
            if key == "rev":
                rev = t[i + 1] == "1"; i += 2
            elif key == "dup":
                dup = t[i + 1] == "1"; i += 2
            elif key in ("reac", "prod"):
                n = int(t[i + 1]); lst = []
                for j in range(n):
                    lst.append((int(t[i + 2 + 2 * j]), int(t[i + 3 + 2 * j])))
                (reac if key == "reac" else prod).extend(lst)
                i += 2 + 2 * n
            elif key == "arr":
                A, b, th = float(t[i + 1]), float(t[i + 2]), float(t[i + 3]); i += 4
            elif key == "eff":
                n = int(t[i + 1])
                for j in range(n):
                    eff[int(t[i + 2 + 2 * j])] = float(t[i + 3 + 2 * j])
                i += 2 + 2 * n
            elif key == "low":
                low = (float(t[i + 1]), float(t[i + 2]), float(t[i + 3])); i += 4
            elif key in ("troe", "sri"):
                j = i + 1; vals = []
                while t[j] not in ("end", "eff", "low", "troe", "sri", "plog"):
                    vals.append(float(t[j])); j += 1
                if key == "troe":
                    troe = tuple(vals)
                else:
                    sri = tuple(vals)
                i = j
            elif key == "plog":
                n = int(t[i + 1])
                plog = [tuple(float(x) for x in t[i + 2 + 4 * q:i + 6 + 4 * q]) for q in range(n)]
                i += 2 + 4 * n
            else:
                raise ValueError("unknown reaction key " + key)
        reactions.append(Reaction(kind, reac, prod, A, b, th, rev, dup, eff, low, troe, sri, plog))
    transport = None
    t = next(it, None)
    if t is not None and t[0] == "transport":
        visc, cond = np.zeros((ns, 5)), np.zeros((ns, 5))
        diff = np.zeros((ns, ns, 5))
        for _ in range(ns):
            t = next(it)
            k = int(t[1])
            visc[k] = [float(x) for x in t[2:7]]
            cond[k] = [float(x) for x in t[7:12]]
        for _ in range(ns * (ns - 1) // 2):
            t = next(it)
            k, j = int(t[1]), int(t[2])
            diff[k, j] = diff[j, k] = [float(x) for x in t[3:8]]
        transport = Transport(visc, cond, diff)
    return Mechanism(name, elements, species, reactions, transport)


# ----------------------------------------------------------------------------
# States
# ----------------------------------------------------------------------------

@dataclass
class States:
    T: np.ndarray          # [n] K
    p: np.ndarray          # [n] Pa
    Y: np.ndarray          # [N, n] mass fractions, species-major (SoA)


def generate_states(n_species: int, n: int, T_range=(300.0, 2800.0), p_atm=(1.0, 1.0),
                    seed: int = 0, alpha: float = 0.5) -> States:
    """Random states: T ~ U(T_range), p ~ U(p_atm) atm, Y ~ Dirichlet(alpha)."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(T_range[0], T_range[1], size=n)
    p = rng.uniform(p_atm[0], p_atm[1], size=n) * ONE_ATM
    G = rng.gamma(alpha, 1.0, size=(n_species, n))
    Y = G / G.sum(axis=0, keepdims=True)
    return States(T, p, np.ascontiguousarray(Y))


def config_states(index: int, n: Optional[int] = None, offset_seed: int = 0) -> States:
    """States of workload ``index`` (seed 24286 + index), optionally fewer points."""
    cfg = CONFIGS[index]
    mech_cfg = CONFIGS[cfg["mech"]]
    if "base" in mech_cfg:
        mech_cfg = CONFIGS[mech_cfg["base"]]
    n = cfg["n_points"] if n is None else n
    return generate_states(mech_cfg["n_species"], n, cfg["T"], cfg["p_atm"],
                           seed=STATE_SEED_BASE + index + offset_seed)


def generate_states_torch(n_species: int, n: int, T_range, p_atm, seed: int, device):
    """Same distributions drawn with torch's generator on ``device`` (large workloads)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    T = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    T = T_range[0] + (T_range[1] - T_range[0]) * T
    p = torch.rand(n, generator=g, device=device, dtype=torch.float64)
    p = (p_atm[0] + (p_atm[1] - p_atm[0]) * p) * ONE_ATM
    conc = torch.full((n_species, n), 0.5, device=device, dtype=torch.float64)
    G = torch._standard_gamma(conc, generator=g) if hasattr(torch, "_standard_gamma") else None
    if G is None:  # pragma: no cover
        raise RuntimeError("torch._standard_gamma unavailable")
    Y = G / G.sum(dim=0, keepdim=True)
    return T, p, Y.contiguous()
