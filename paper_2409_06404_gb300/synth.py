"""Seeded synthetic mechanisms and thermochemical states.

This module only *draws inputs*: element compositions, Arrhenius/Troe parameters,
third-body efficiencies, polynomial fits of smooth heat-capacity and transport curves,
and point states (T, p, Y_k) shaped like the spectral-element workloads of the paper
(polynomial order 7, 8^3 = 512 Gauss-Lobatto-Legendre points per hexahedral element,
Sec. 3.2-3.3).  It contains none of the thermochemistry that the library evaluates:
no rate constant, equilibrium constant, rate of progress, production rate, mixture rule
or transport formula.  Both the CPU oracle (``oracle/``) and the CUDA path receive the
arrays produced here, and nothing else is shared between them.

Everything is deterministic in the seed (numpy PCG64).

Units are SI throughout: K, Pa, kg/mol, J/mol, m^3/mol/s (for order-2 reactions).

Mechanism conventions (the reading of the paper's "Cantera format" mechanism input,
Sec. 2, which the paper does not spell out):
  * NASA-7 polynomials, two ranges split at ``T_mid`` (1000 K), coefficients a1..a7.
  * Every reaction is reversible; the reverse rate follows from equilibrium.
  * ``rtype`` 0 = elementary, 1 = third-body (rate of progress multiplied by [M]),
    2 = Troe falloff (k_inf from lnA/beta/Ea, k_0 from lnA0/beta0/Ea0).
  * Third-body efficiencies ``eff[r, k]`` (default 1) are used for rtype 1 and 2.
  * Transport: ln(mu_k), ln(lambda_k), ln(D_jk at p_ref) are cubic polynomials in ln T,
    coefficients stored lowest order first; D pairs j<k packed row-major
    (pair index of (j, k), j<k: j*K - j*(j+1)/2 + (k - j - 1)).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, fields

import numpy as np
from numpy.polynomial import Polynomial

# IUPAC standard atomic weights, kg/mol
ATOMIC_WEIGHT = {"H": 1.008e-3, "C": 12.011e-3, "N": 14.007e-3, "O": 15.999e-3}
# Molar gas constant (J/mol/K), used only to express sampled formation enthalpies in kelvin
_R_GAS = 8.314462618
_T_REF = 298.15
P_ATM = 101325.0

MAX_SIDE = 3  # at most 3 molecules on each side of a generated reaction


@dataclass
class Mechanism:
    """A synthetic reaction mechanism as plain numpy arrays (host memory)."""

    K: int
    R: int
    elements: tuple
    W: np.ndarray          # [K] kg/mol
    atoms: np.ndarray      # [K, n_elem] int32
    nasa_lo: np.ndarray    # [K, 7] a1..a7 for T <= T_mid
    nasa_hi: np.ndarray    # [K, 7] a1..a7 for T > T_mid
    T_mid: np.ndarray      # [K]
    T_lo: np.ndarray       # [K] nominal validity range (not enforced)
    T_hi: np.ndarray       # [K]
    reac_ptr: np.ndarray   # [R+1] int32, CSR over reactant entries
    reac_sp: np.ndarray    # int32 species index
    reac_nu: np.ndarray    # int32 stoichiometric coefficient (>0)
    prod_ptr: np.ndarray   # [R+1]
    prod_sp: np.ndarray
    prod_nu: np.ndarray
    rtype: np.ndarray      # [R] int32: 0 elementary, 1 third-body, 2 Troe
    lnA: np.ndarray        # [R] ln A (high-pressure limit for Troe)
    beta: np.ndarray       # [R]
    Ea: np.ndarray         # [R] J/mol
    lnA0: np.ndarray       # [R] low-pressure limit (Troe rows only, else 0)
    beta0: np.ndarray      # [R]
    Ea0: np.ndarray        # [R]
    troe: np.ndarray       # [R, 4] a, T3, T1, T2 (T2 <= 0: term absent); Troe rows only
    eff: np.ndarray        # [R, K] third-body efficiencies (used for rtype 1, 2)
    mu_fit: np.ndarray     # [K, 4]
    lam_fit: np.ndarray    # [K, 4]
    D_fit: np.ndarray      # [K(K-1)/2, 4], pairs j<k, at p_ref
    p_ref: float = P_ATM

    @property
    def n_elem(self) -> int:
        return len(self.elements)

    def arrays(self) -> dict:
        return {f.name: getattr(self, f.name) for f in fields(self)}

    def copy(self) -> "Mechanism":
        kw = {}
        for f in fields(self):
            v = getattr(self, f.name)
            kw[f.name] = v.copy() if isinstance(v, np.ndarray) else v
        return Mechanism(**kw)


# --------------------------------------------------------------------------------------
# species
# --------------------------------------------------------------------------------------
def _species_atoms(rng, K, n_elem, max_count=2):
    vecs = [v for v in itertools.product(range(max_count + 1), repeat=n_elem) if sum(v) > 0]
    vecs = np.array(vecs, dtype=np.int32)
    if K <= len(vecs):
        idx = rng.choice(len(vecs), size=K, replace=False)
    else:  # more species than compositions: the surplus are isomers
        extra = rng.choice(len(vecs), size=K - len(vecs), replace=True)
        idx = np.concatenate([rng.permutation(len(vecs)), extra])
    return vecs[idx]


def _fit_cp(rng, n_atoms, T_mid):
    """Fit two quartic polynomials (in T) to a smooth sigmoid c_p/R curve, continuous at T_mid."""
    c0 = rng.uniform(2.5, 4.5)
    dc = rng.uniform(0.5, 1.5) * n_atoms
    Tc = rng.uniform(500.0, 2000.0)
    w = rng.uniform(200.0, 800.0)

    def curve(T):
        return c0 + dc / (1.0 + np.exp(-(T - Tc) / w))

    s = 1000.0  # fit in t = T/s for conditioning
    Tl = np.linspace(300.0, T_mid, 141)
    bl = np.linalg.lstsq(np.vander(Tl / s, 5, increasing=True), curve(Tl), rcond=None)[0]
    v_mid = Polynomial(bl)(T_mid / s)
    Th = np.linspace(T_mid, 3500.0, 251)
    th = Th / s
    tm = T_mid / s
    Vh = np.stack([th ** m - tm ** m for m in range(1, 5)], axis=1)
    ch = np.linalg.lstsq(Vh, curve(Th) - v_mid, rcond=None)[0]
    bh = np.concatenate([[v_mid - sum(ch[m - 1] * tm ** m for m in range(1, 5))], ch])
    scale = s ** -np.arange(5.0)
    return bl * scale, bh * scale


def _antiderivatives(cp_coef):
    """H(T) = int cp/R dT and S(T) = int cp/(R T) dT with zero integration constants."""
    P = Polynomial(cp_coef)
    H = P.integ()
    rest = Polynomial(cp_coef[1:]).integ()   # int (cp/R - a1)/T dT
    a1 = cp_coef[0]
    return (lambda T: H(T)), (lambda T: a1 * np.log(T) + rest(T))


def _nasa(rng, n_atoms, hf, s298, T_mid):
    lo, hi = _fit_cp(rng, n_atoms, T_mid)
    H_lo, S_lo = _antiderivatives(lo)
    H_hi, S_hi = _antiderivatives(hi)
    a6_lo = hf / _R_GAS - H_lo(_T_REF)
    a7_lo = s298 - S_lo(_T_REF)
    a6_hi = a6_lo + H_lo(T_mid) - H_hi(T_mid)
    a7_hi = a7_lo + S_lo(T_mid) - S_hi(T_mid)
    return np.concatenate([lo, [a6_lo, a7_lo]]), np.concatenate([hi, [a6_hi, a7_hi]])


def _log_cubic(rng, ln_v300, e_lo, e_hi):
    """Coefficients (in ln T, lowest order first) of ln v = ln v300 + e u + c2 u^2 + c3 u^3, u = ln(T/300)."""
    e = rng.uniform(e_lo, e_hi)
    c2 = rng.uniform(-0.02, 0.02)
    c3 = rng.uniform(-0.005, 0.005)
    P = Polynomial([ln_v300, e, c2, c3])(Polynomial([-np.log(300.0), 1.0]))
    c = np.zeros(4)
    c[: len(P.coef)] = P.coef
    return c


# --------------------------------------------------------------------------------------
# reactions
# --------------------------------------------------------------------------------------
def _multisets(atoms):
    """All multisets of 1..MAX_SIDE species, grouped by total atom vector."""
    K = atoms.shape[0]
    sets, keys = [], []
    for size in range(1, MAX_SIDE + 1):
        for c in itertools.combinations_with_replacement(range(K), size):
            sets.append(c)
    pad = np.full((len(sets), MAX_SIDE), -1, dtype=np.int64)
    for i, c in enumerate(sets):
        pad[i, : len(c)] = c
    atoms_pad = np.vstack([atoms, np.zeros((1, atoms.shape[1]), dtype=atoms.dtype)])
    vec = atoms_pad[pad].sum(axis=1)  # index -1 hits the zero row
    _, inv = np.unique(vec, axis=0, return_inverse=True)
    inv = inv.ravel()
    groups = {}
    for i, g in enumerate(inv):
        groups.setdefault(int(g), []).append(i)
    return sets, inv, groups


def _entries(ms):
    sp, nu = np.unique(np.array(ms, dtype=np.int64), return_counts=True)
    return list(zip(sp.tolist(), nu.tolist()))


def _reactions(rng, atoms, hf, R, n_tb, n_troe, max_dh=4.0e5):
    sets, inv, groups = _multisets(atoms)
    sizes = np.array([len(s) for s in sets])
    singles = [i for i, s in enumerate(sets) if len(s) == 1]
    nonsingle = np.flatnonzero(sizes >= 2)
    used = set()
    out = []

    def accept(a, b):
        key = (min(a, b), max(a, b))
        if a == b or key in used:
            return False
        dh = sum(hf[s] for s in sets[b]) - sum(hf[s] for s in sets[a])
        if abs(dh) > max_dh:
            return False
        used.add(key)
        return True

    def draw_falloff_like():
        # A + B (+M) <=> AB (+M), random direction; any balanced reaction if none is left
        for _ in range(2000):
            a = singles[rng.integers(len(singles))]
            partners = [j for j in groups[int(inv[a])] if sizes[j] == 2]
            if not partners:
                continue
            b = partners[rng.integers(len(partners))]
            if rng.random() < 0.5:
                a, b = b, a
            if accept(a, b):
                return a, b
        return draw_elementary()

    def draw_elementary():
        for _ in range(100000):
            a = int(nonsingle[rng.integers(len(nonsingle))]) if rng.random() < 0.85 else \
                singles[rng.integers(len(singles))]
            cand = [j for j in groups[int(inv[a])] if j != a]
            if not cand:
                continue
            b = cand[rng.integers(len(cand))]
            if rng.random() < 0.5:
                a, b = b, a
            if accept(a, b):
                return a, b
        raise RuntimeError("could not draw an elementary reaction")

    kinds = [0] * (R - n_tb - n_troe) + [1] * n_tb + [2] * n_troe
    for kind in kinds:
        a, b = draw_falloff_like() if kind else draw_elementary()
        out.append((kind, _entries(sets[a]), _entries(sets[b])))
    order = rng.permutation(len(out))
    return [out[i] for i in order]


def _log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def make_mechanism(K, R, n_tb, n_troe, elements=("C", "H", "O", "N"), seed=0, T_mid=1000.0):
    """Draw a synthetic element-balanced mechanism (see module docstring for the conventions).

    Arrhenius parameters: A log-uniform in [1e6, 1e16], beta uniform in [-2, 2],
    Ea uniform in [0, 200] kJ/mol; Troe rows draw k_0 and k_inf from the same
    distributions and a ~ U[0.1, 0.9], T3 ~ logU[30, 1000] K, T1 ~ logU[1000, 1e4] K,
    T2 ~ logU[1000, 1e4] K with probability 1/2 (else absent).  Third-body rows get
    U[0.5, 12] efficiencies on a random subset of 2..6 species (others 1).
    Formation enthalpies h_f(298) ~ U[-400, 400] kJ/mol, s(298)/R ~ U[20, 35]; reactions
    whose sum of nu*h_f exceeds 400 kJ/mol in magnitude are redrawn, which keeps the
    equilibrium constants within about 1e+-130 over 300..3500 K.
    """
    if R < n_tb + n_troe:
        raise ValueError("R must cover the third-body and Troe reactions")
    rng = np.random.Generator(np.random.PCG64(seed))
    ne = len(elements)
    atoms = _species_atoms(rng, K, ne)
    W = atoms @ np.array([ATOMIC_WEIGHT[e] for e in elements])
    n_atoms = atoms.sum(axis=1)

    hf = rng.uniform(-4.0e5, 4.0e5, K)
    s298 = rng.uniform(20.0, 35.0, K)
    nasa_lo = np.zeros((K, 7))
    nasa_hi = np.zeros((K, 7))
    for k in range(K):
        nasa_lo[k], nasa_hi[k] = _nasa(rng, n_atoms[k], hf[k], s298[k], T_mid)

    rx = _reactions(rng, atoms, hf, R, n_tb, n_troe)
    reac_ptr, reac_sp, reac_nu = [0], [], []
    prod_ptr, prod_sp, prod_nu = [0], [], []
    rtype = np.zeros(R, np.int32)
    for r, (kind, reac, prod) in enumerate(rx):
        rtype[r] = kind
        for s, n in reac:
            reac_sp.append(s)
            reac_nu.append(n)
        for s, n in prod:
            prod_sp.append(s)
            prod_nu.append(n)
        reac_ptr.append(len(reac_sp))
        prod_ptr.append(len(prod_sp))

    lnA = np.log(_log_uniform(rng, 1e6, 1e16, R))
    beta = rng.uniform(-2.0, 2.0, R)
    Ea = rng.uniform(0.0, 2.0e5, R)
    lnA0 = np.zeros(R)
    beta0 = np.zeros(R)
    Ea0 = np.zeros(R)
    troe = np.zeros((R, 4))
    eff = np.ones((R, K))
    for r in range(R):
        if rtype[r] == 2:
            lnA0[r] = np.log(_log_uniform(rng, 1e6, 1e16))
            beta0[r] = rng.uniform(-2.0, 2.0)
            Ea0[r] = rng.uniform(0.0, 2.0e5)
            troe[r, 0] = rng.uniform(0.1, 0.9)
            troe[r, 1] = _log_uniform(rng, 30.0, 1000.0)
            troe[r, 2] = _log_uniform(rng, 1000.0, 1.0e4)
            troe[r, 3] = _log_uniform(rng, 1000.0, 1.0e4) if rng.random() < 0.5 else 0.0
        if rtype[r] != 0:
            m = int(rng.integers(2, min(6, K) + 1))
            sel = rng.choice(K, size=m, replace=False)
            eff[r, sel] = rng.uniform(0.5, 12.0, m)

    mu_fit = np.stack([_log_cubic(rng, np.log(_log_uniform(rng, 8e-6, 2e-5)), 0.6, 0.8) for _ in range(K)])
    lam_fit = np.stack([_log_cubic(rng, np.log(_log_uniform(rng, 0.01, 0.2)), 0.7, 0.9) for _ in range(K)])
    P = K * (K - 1) // 2
    D_fit = np.stack([_log_cubic(rng, np.log(_log_uniform(rng, 5e-6, 8e-5)), 1.6, 1.8) for _ in range(P)]) \
        if P else np.zeros((0, 4))

    i32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    f64 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return Mechanism(
        K=K, R=R, elements=tuple(elements), W=f64(W), atoms=i32(atoms),
        nasa_lo=f64(nasa_lo), nasa_hi=f64(nasa_hi), T_mid=f64(np.full(K, T_mid)),
        T_lo=f64(np.full(K, 300.0)), T_hi=f64(np.full(K, 3500.0)),
        reac_ptr=i32(reac_ptr), reac_sp=i32(reac_sp), reac_nu=i32(reac_nu),
        prod_ptr=i32(prod_ptr), prod_sp=i32(prod_sp), prod_nu=i32(prod_nu),
        rtype=i32(rtype), lnA=f64(lnA), beta=f64(beta), Ea=f64(Ea),
        lnA0=f64(lnA0), beta0=f64(beta0), Ea0=f64(Ea0), troe=f64(troe), eff=f64(eff),
        mu_fit=f64(mu_fit), lam_fit=f64(lam_fit), D_fit=f64(D_fit), p_ref=P_ATM,
    )


def mechanism_from_arrays(**kw) -> Mechanism:
    """Build a Mechanism from explicit arrays (used for hand-made tiny mechanisms in tests)."""
    K = int(kw["K"])
    R = int(kw["R"])
    d = dict(
        elements=("X",), T_mid=np.full(K, 1000.0), T_lo=np.full(K, 300.0), T_hi=np.full(K, 3500.0),
        lnA0=np.zeros(R), beta0=np.zeros(R), Ea0=np.zeros(R), troe=np.zeros((R, 4)),
        eff=np.ones((R, K)), mu_fit=np.zeros((K, 4)), lam_fit=np.zeros((K, 4)),
        D_fit=np.zeros((K * (K - 1) // 2, 4)), p_ref=P_ATM, atoms=np.ones((K, 1), np.int32),
        rtype=np.zeros(R, np.int32),
    )
    d.update(kw)
    ints = {"atoms", "reac_ptr", "reac_sp", "reac_nu", "prod_ptr", "prod_sp", "prod_nu", "rtype"}
    out = {}
    for f in fields(Mechanism):
        v = d[f.name]
        if f.name in ints:
            v = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
        elif f.name in ("K", "R"):
            v = int(v)
        elif f.name == "p_ref":
            v = float(v)
        elif f.name == "elements":
            v = tuple(v)
        else:
            v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
        out[f.name] = v
    return Mechanism(**out)


# --------------------------------------------------------------------------------------
# states
# --------------------------------------------------------------------------------------
def gll_nodes(order=7):
    """Gauss-Lobatto-Legendre nodes of the given polynomial order, mapped to [0, 1]."""
    from numpy.polynomial import legendre as L
    inner = L.Legendre.basis(order).deriv().roots()
    x = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return 0.5 * (x + 1.0)


def _dirichlet(rng, alpha, K, n):
    g = rng.gamma(alpha, 1.0, size=(K, n))
    g /= g.sum(axis=0, keepdims=True)
    return g


@dataclass
class States:
    T: np.ndarray   # [n]
    p: np.ndarray   # [n]
    Y: np.ndarray   # [K, n] (row stride n)

    @property
    def n(self):
        return self.T.shape[0]


def states_uniform(K, n, seed, T_lo=300.0, T_hi=2500.0, p=P_ATM, alpha=0.5) -> States:
    """T ~ U[T_lo, T_hi], constant p, Y ~ Dirichlet(alpha)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T = rng.uniform(T_lo, T_hi, n)
    Y = _dirichlet(rng, alpha, K, n)
    return States(T=T, p=np.full(n, float(p)), Y=np.ascontiguousarray(Y))


def states_flame(K, n_elements, seed, order=7, p=P_ATM, alpha=0.3, noise=0.05,
                 T_u=300.0, dT=950.0, x0=0.5, width=0.05, clip=(300.0, 3500.0)) -> States:
    """Flame-like states on a cubic grid of hexahedral elements with (order+1)^3 GLL points each.

    Point index = element * (order+1)^3 + lexicographic GLL index; elements are ordered
    x-fastest on an m x m x m grid (m^3 = n_elements).  T follows
    T_u + dT (1 + tanh((x - x0)/width)) along x in [0, 1] (300..2200 K by default), times
    (1 + noise N(0,1)), clipped; p constant; Y ~ Dirichlet(alpha) per point.
    """
    m = int(round(n_elements ** (1.0 / 3.0)))
    if m ** 3 != n_elements:
        raise ValueError("n_elements must be a perfect cube")
    q = order + 1
    xi = gll_nodes(order)
    e = np.arange(n_elements)
    ex = e % m
    ix = np.arange(q ** 3) % q
    x = (ex[:, None] + xi[ix][None, :]) / m
    rng = np.random.Generator(np.random.PCG64(seed))
    T = T_u + dT * (1.0 + np.tanh((x.ravel() - x0) / width))
    T = T * (1.0 + noise * rng.standard_normal(T.shape[0]))
    T = np.clip(T, clip[0], clip[1])
    n = T.shape[0]
    Y = _dirichlet(rng, alpha, K, n)
    return States(T=T, p=np.full(n, float(p)), Y=np.ascontiguousarray(Y))


def normal(shape, seed):
    """Seeded N(0,1) array (directions v and cotangents w for the derivative workloads)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape)


# --------------------------------------------------------------------------------------
# named workloads (the paper's shapes: p = 7, 512 GLL points per element)
# --------------------------------------------------------------------------------------
MECHS = {
    "h2_9sp_21rx": dict(K=9, R=21, n_tb=3, n_troe=1, elements=("H", "O", "N"), seed=1009),
    "ch4_53sp_325rx": dict(K=53, R=325, n_tb=20, n_troe=25, elements=("C", "H", "O", "N"), seed=1053),
    "big_120sp_700rx": dict(K=120, R=700, n_tb=40, n_troe=60, elements=("C", "H", "O", "N"), seed=1120),
}

_MECH_CACHE = {}


def mechanism(name) -> Mechanism:
    if name not in _MECH_CACHE:
        _MECH_CACHE[name] = make_mechanism(**MECHS[name])
    return _MECH_CACHE[name]


def workload_states(name, K, n_points=None, n_elements=None):
    """States of a named workload; ``n_points`` takes the first points (whole elements first).
    ``n_elements`` (a cube) shrinks the flame field to that many elements, same profile."""
    if name == "uniform_64el":        # 64 elements x 512 = 32,768 points
        st = states_uniform(K, 64 * 512, seed=2009, alpha=0.5)
    elif name == "flame_4096el":      # 16^3 elements x 512 = 2,097,152 points
        st = states_flame(K, n_elements or 4096, seed=2053 if K == 53 else 2120)
    elif name == "flame_32768el":     # 32^3 elements x 512 = 16,777,216 points (implicit stage)
        st = states_flame(K, n_elements or 32768, seed=2053)
    else:
        raise KeyError(name)
    if n_points is not None:
        st = States(T=st.T[:n_points].copy(), p=st.p[:n_points].copy(),
                    Y=np.ascontiguousarray(st.Y[:, :n_points]))
    return st
