"""Pins for the oracle's kinetics: omega_k, heat release (definition steps 3-8).

The paper names the species production rates and the heat release sum_k h_k omega_k
(Eq. 1a-b, Sec. 3.3) but prints no kinetics; the oracle follows the Chemkin/Cantera
mass-action convention.  These tests pin it to what the definitions force, without
retyping them:
  * conservation of mass and of every element (sum_k W_k omega_k = 0, sum_k a_ek omega_k = 0),
    also with negative mass fractions, whose concentrations enter as plain integer powers;
  * zero net rates at equilibrium states built from element potentials and the
    (separately pinned) Gibbs energies, at p = 1 atm and away from it;
  * the de Donder relation rev_r/fwd_r = exp(sum_k nu_kr mu_k/RT) at arbitrary states;
  * Arrhenius special values (k = A, k = A T, k = A/10 at Ea = R T ln 10);
  * third-body [M] = p/(RT) for unit efficiencies, plus the (eps-1) C_k correction;
  * Troe: Lindemann limit, the centre point F = F_cent, the T2 term, one interior point;
  * element-wise enthalpy-shift invariance of omega and the heat release;
  * invariance under relabelling the species.
"""
import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import logsumexp

import oracle
from paper_2409_06404_gb300 import synth
from conftest import R_GAS, P_ATM, nu_matrix


def _states(mech, n, seed, T=(300.0, 3000.0), alpha=0.5):
    st = synth.states_uniform(mech.K, n, seed=seed, T_lo=T[0], T_hi=T[1], alpha=alpha)
    return st.T, st.p, st.Y


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx", "big_120sp_700rx"])
def test_mass_and_element_conservation(name):
    m = synth.mechanism(name)
    T, p, Y = _states(m, 300, seed=21)
    w, h, ws, hs = oracle.rates(m, T, p, Y, scales=True)
    mass = np.abs(m.W @ w)
    assert np.all(mass <= 1e-13 * (m.W @ ws))
    for e in range(m.atoms.shape[1]):
        a = m.atoms[:, e].astype(float)
        assert np.all(np.abs(a @ w) <= 1e-13 * (a @ ws + 1e-300)), e


def equilibrium_state(mech, T, p, rng, spread=0.5):
    """Mole fractions X_k = exp(-g_k/RT - ln(p/p0) + sum_e lambda_e a_ek), normalised by a
    uniform shift of the element potentials; Gibbs energies from the oracle's thermo."""
    K = mech.K
    g = oracle.thermo(mech, [T], p, np.full((K, 1), 1.0 / K))["g_k"][:, 0]
    gRT = g / (R_GAS * T)
    a = mech.atoms.astype(float)
    # element potentials that flatten -g/RT as far as possible, then a random perturbation
    A = np.hstack([a, np.ones((K, 1))])
    lam = np.linalg.lstsq(A, gRT, rcond=None)[0][:-1] + spread * rng.standard_normal(a.shape[1])
    base = -gRT - np.log(p / P_ATM) + a @ lam
    na = a.sum(axis=1)
    t = brentq(lambda t: logsumexp(base + t * na), -1e4, 1e4, xtol=1e-15, rtol=1e-15)
    X = np.exp(base + t * na)
    Y = X * mech.W / np.sum(X * mech.W)
    return Y


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
@pytest.mark.parametrize("T,p", [(2500.0, P_ATM), (1400.0, P_ATM), (2000.0, 5 * P_ATM), (3200.0, 0.3 * P_ATM)])
def test_zero_net_rates_at_equilibrium(name, T, p):
    m = synth.mechanism(name)
    rng = np.random.default_rng(7)
    Y = equilibrium_state(m, T, p, rng)[:, None]
    fwd, rev = oracle.rates_of_progress(m, [T], p, Y)
    fwd, rev = fwd[:, 0], rev[:, 0]
    ok = (fwd > 1e-250) & (rev > 1e-250)
    assert ok.mean() > 0.5, "equilibrium state too sparse to test"
    assert np.all(np.abs(fwd[ok] - rev[ok]) <= 1e-10 * (fwd[ok] + rev[ok]))
    # and the net production rates vanish on the same scale
    w, h, ws, hs = oracle.rates(m, [T], p, Y, scales=True)
    assert np.all(np.abs(w[:, 0]) <= 1e-9 * ws[:, 0] + 1e-280)


def test_nonequilibrium_state_has_nonzero_rates(mech9):
    # guard against a vacuous equilibrium test: perturbing the state breaks the balance
    rng = np.random.default_rng(8)
    Y = equilibrium_state(mech9, 2500.0, P_ATM, rng)
    Y2 = Y.copy()
    Y2[0] *= 1.5
    fwd, rev = oracle.rates_of_progress(mech9, [2500.0], P_ATM, Y2[:, None])
    rel = np.abs(fwd - rev) / (fwd + rev)
    assert np.max(rel) > 1e-3


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
def test_de_donder_relation(name):
    """rev_r/fwd_r = exp(sum_k nu_kr mu_k/RT), mu_k/RT = g_k/RT + ln(C_k R T/p0)."""
    m = synth.mechanism(name)
    T, p, Y = _states(m, 40, seed=31, T=(300.0, 3400.0))
    p = p * np.linspace(0.2, 8.0, len(T))
    th = oracle.thermo(m, T, p, Y)
    C = th["rho"][None, :] * Y / m.W[:, None]
    muRT = th["g_k"] / (R_GAS * T) + np.log(C * R_GAS * T / P_ATM)
    nu = nu_matrix(m)
    fwd, rev = oracle.rates_of_progress(m, T, p, Y)
    lhs = np.log(rev) - np.log(fwd)
    rhs = nu.T @ muRT
    ok = np.isfinite(lhs) & np.isfinite(rhs)
    assert ok.mean() > 0.9
    assert np.max(np.abs(lhs[ok] - rhs[ok]) / (1.0 + np.abs(rhs[ok]))) < 1e-12


def _one_reaction(reac, prod, W, rtype=0, lnA=np.log(1e10), beta=0.0, Ea=0.0, eff=None, troe=None,
                  lnA0=0.0, beta0=0.0, Ea0=0.0, a6=None):
    K = len(W)
    nasa = np.zeros((K, 7))
    nasa[:, 0] = 3.5
    nasa[:, 6] = 5.0
    if a6 is not None:
        nasa[:, 5] = a6
    rs, rn = zip(*reac)
    ps, pn = zip(*prod)
    kw = dict(K=K, R=1, W=np.array(W), nasa_lo=nasa, nasa_hi=nasa, reac_ptr=[0, len(rs)], reac_sp=rs,
              reac_nu=rn, prod_ptr=[0, len(ps)], prod_sp=ps, prod_nu=pn, rtype=[rtype], lnA=[lnA],
              beta=[beta], Ea=[Ea], lnA0=[lnA0], beta0=[beta0], Ea0=[Ea0])
    if eff is not None:
        kw["eff"] = np.array(eff, dtype=float)[None, :]
    if troe is not None:
        kw["troe"] = np.array(troe, dtype=float)[None, :]
    return synth.mechanism_from_arrays(**kw)


def _conc(mech, T, p, Y):
    rho = oracle.thermo(mech, T, p, Y)["rho"]
    return rho[None, :] * Y / mech.W[:, None]


def test_arrhenius_special_values():
    W = [0.03, 0.03]
    T = np.array([400.0, 1000.0, 2000.0])
    Y = np.array([[0.7, 0.7, 0.7], [0.3, 0.3, 0.3]])
    cases = [
        (dict(beta=0.0, Ea=0.0), lambda T: 1e10 * np.ones_like(T)),
        (dict(beta=1.0, Ea=0.0), lambda T: 1e10 * T),
        (dict(beta=-1.5, Ea=0.0), lambda T: 1e10 * T ** -1.5),
        (dict(beta=0.0, Ea=R_GAS * 1000.0 * np.log(10.0)), lambda T: 1e10 * 10.0 ** (-1000.0 / T)),
    ]
    for kw, kf in cases:
        m = _one_reaction([(0, 1)], [(1, 1)], W, **kw)
        fwd, _ = oracle.rates_of_progress(m, T, P_ATM, Y)
        C = _conc(m, T, P_ATM, Y)
        assert np.allclose(fwd[0] / C[0], kf(T), rtol=1e-13), kw
    # A <=> B with identical thermodynamics: K_c = 1, omega_B = k (C_A - C_B)
    m = _one_reaction([(0, 1)], [(1, 1)], W)
    w, h = oracle.rates(m, T, P_ATM, Y)
    C = _conc(m, T, P_ATM, Y)
    assert np.allclose(w[1], 1e10 * (C[0] - C[1]), rtol=1e-13)
    assert np.allclose(w[0], -w[1], rtol=1e-15)
    assert np.allclose(h, 0.0, atol=1e-3)       # equal enthalpies: no heat release


def test_third_body_concentration():
    W = [0.002, 0.032, 0.034]
    T = np.array([800.0, 1800.0])
    p = np.array([P_ATM, 3 * P_ATM])
    Y = np.array([[0.2, 0.1], [0.5, 0.6], [0.3, 0.3]])
    m = _one_reaction([(0, 1), (1, 1)], [(2, 1)], W, rtype=1, eff=[1.0, 1.0, 1.0])
    fwd, _ = oracle.rates_of_progress(m, T, p, Y)
    C = _conc(m, T, p, Y)
    assert np.allclose(fwd[0], 1e10 * C[0] * C[1] * p / (R_GAS * T), rtol=1e-13)
    m5 = _one_reaction([(0, 1), (1, 1)], [(2, 1)], W, rtype=1, eff=[5.0, 1.0, 1.0])
    fwd5, _ = oracle.rates_of_progress(m5, T, p, Y)
    assert np.allclose(fwd5[0], 1e10 * C[0] * C[1] * (p / (R_GAS * T) + 4.0 * C[0]), rtol=1e-13)


def test_negative_concentrations_enter_as_plain_powers():
    """Mass action with a negative concentration (a negative mass fraction): the products are
    plain integer powers, so a squared negative concentration gives a positive term and a single
    one a negative term, and [M] takes the signed C_k."""
    W = [0.002, 0.032, 0.034]
    T = np.array([900.0, 1700.0])
    p = np.array([P_ATM, 2 * P_ATM])
    Y = np.array([[-0.01, -1e-4], [0.6, 0.7], [0.41, 0.3001]])
    sq = _one_reaction([(0, 2)], [(2, 1)], W)                       # 2 A -> C
    fwd, rev = oracle.rates_of_progress(sq, T, p, Y)
    C = _conc(sq, T, p, Y)
    assert np.all(C[0] < 0) and np.all(fwd[0] > 0) and np.all(rev[0] > 0)
    assert np.allclose(fwd[0], 1e10 * C[0] * C[0], rtol=1e-13)
    ab = _one_reaction([(0, 1), (1, 1)], [(2, 1)], W)               # A + B -> C
    fwd, _ = oracle.rates_of_progress(ab, T, p, Y)
    assert np.all(fwd[0] < 0) and np.allclose(fwd[0], 1e10 * C[0] * C[1], rtol=1e-13)
    tb = _one_reaction([(0, 1), (1, 1)], [(2, 1)], W, rtype=1, eff=[5.0, 1.0, 1.0])
    fwd, _ = oracle.rates_of_progress(tb, T, p, Y)
    assert np.allclose(fwd[0], 1e10 * C[0] * C[1] * (p / (R_GAS * T) + 4.0 * C[0]), rtol=1e-13)


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
def test_conservation_with_negative_fractions(name):
    """Mass and elements are conserved whatever the signs of the concentrations."""
    m = synth.mechanism(name)
    T, p, Y = _states(m, 200, seed=23)
    rng = np.random.default_rng(24)
    Y = Y - 1e-3 * rng.random(Y.shape) * (rng.random(Y.shape) < 0.2)   # some fractions negative
    assert np.any(Y < 0)
    w, h, ws, hs = oracle.rates(m, T, p, Y, scales=True)
    assert np.all(np.isfinite(w))
    assert np.all(np.abs(m.W @ w) <= 1e-13 * (m.W @ ws))
    for e in range(m.atoms.shape[1]):
        a = m.atoms[:, e].astype(float)
        assert np.all(np.abs(a @ w) <= 1e-13 * (a @ ws + 1e-300)), e


def _troe_k(troe, p, T=1500.0, A0=1e12, Ainf=1e8):
    W = [0.016, 0.017, 0.033]
    Y = np.tile(np.array([[0.3], [0.3], [0.4]]), (1, len(p)))
    Tv = np.full(len(p), T)
    m = _one_reaction([(0, 1), (1, 1)], [(2, 1)], W, rtype=2, lnA=np.log(Ainf), lnA0=np.log(A0),
                      troe=troe)
    fwd, _ = oracle.rates_of_progress(m, Tv, p, Y)
    C = _conc(m, Tv, p, Y)
    k = fwd[0] / (C[0] * C[1])
    M = p / (R_GAS * T)
    return k, A0 * M / Ainf


def test_troe_lindemann_limit():
    p = P_ATM * np.logspace(-4, 4, 9)
    k, Pr = _troe_k([0.0, 1e30, 1.0, 0.0], p)    # F_cent = 1 -> F = 1
    assert np.allclose(k, 1e8 * Pr / (1 + Pr), rtol=1e-12)


def test_troe_centre_and_limits():
    T = 1500.0
    troe = [1.0, 1e30, T / np.log(2.0), 0.0]     # F_cent = exp(-ln 2) = 1/2
    c = -0.4 - 0.67 * np.log10(0.5)
    Pr_c = 10.0 ** (-c)                            # log10 Pr + c = 0 -> F = F_cent
    p = np.array([Pr_c * 1e8 / 1e12 * R_GAS * T])
    k, Pr = _troe_k(troe, p, T=T)
    assert np.allclose(Pr, Pr_c, rtol=1e-14)
    assert np.allclose(k, 1e8 * Pr / (1 + Pr) * 0.5, rtol=1e-12)
    # F_cent < 1 broadens the falloff curve below Lindemann everywhere
    for Pr_t in (1e-6, 1e-2, 1e2, 1e6):
        p = np.array([Pr_t * 1e8 / 1e12 * R_GAS * T])
        k, Pr = _troe_k(troe, p, T=T)
        F = k / (1e8 * Pr / (1 + Pr))
        assert 0.5 < F[0] < 1.0
    # an interior point, evaluated by hand from the standard Troe constants:
    # log10 Pr + c = 1 -> n = 0.75 + 1.27*log10(2) = 1.1323063..., f1 = 1/(n - 0.14),
    # log10 F = -log10(2)/(1 + f1^2)
    n = 0.75 + 1.27 * 0.30102999566398120
    f1 = 1.0 / (n - 0.14)
    F_expect = 10.0 ** (-0.30102999566398120 / (1.0 + f1 * f1))
    p = np.array([10.0 ** (1.0 - c) * 1e8 / 1e12 * R_GAS * T])
    k, Pr = _troe_k(troe, p, T=T)
    assert np.allclose(k / (1e8 * Pr / (1 + Pr)), F_expect, rtol=1e-12)
    # T2 term: a = 0 and T3 -> inf give F_cent = 1 + exp(-T2/T)
    troe2 = [0.0, 1e30, 1.0, T * np.log(4.0)]     # F_cent = 1 + 1/4
    p = np.array([10.0 ** (0.4 + 0.67 * np.log10(1.25)) * 1e8 / 1e12 * R_GAS * T])
    k, Pr = _troe_k(troe2, p, T=T)
    assert np.allclose(k / (1e8 * Pr / (1 + Pr)), 1.25, rtol=1e-12)


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
def test_enthalpy_shift_invariance(name):
    m = synth.mechanism(name)
    T, p, Y = _states(m, 50, seed=41)
    w0, h0, ws, hs = oracle.rates(m, T, p, Y, scales=True)
    rng = np.random.default_rng(5)
    delta = rng.uniform(-5000.0, 5000.0, m.atoms.shape[1])   # kelvin, per element
    m2 = m.copy()
    shift = m.atoms @ delta
    m2.nasa_lo[:, 5] += shift
    m2.nasa_hi[:, 5] += shift
    w1, h1 = oracle.rates(m2, T, p, Y)
    assert np.all(np.abs(w1 - w0) <= 1e-11 * ws)
    assert np.all(np.abs(h1 - h0) <= 1e-11 * hs)
    # the shift is not a no-op for the enthalpies themselves
    assert not np.allclose(oracle.thermo(m2, T, p, Y)["h_k"], oracle.thermo(m, T, p, Y)["h_k"])


def test_heat_release_is_minus_sum_h_omega(mech53):
    T, p, Y = _states(mech53, 60, seed=51)
    w, h, ws, hs = oracle.rates(mech53, T, p, Y, scales=True)
    hk = oracle.thermo(mech53, T, p, Y)["h_k"]
    assert np.all(np.abs(h + np.sum(hk * w, axis=0)) <= 1e-12 * hs)


def permute_species(m, perm):
    """Mechanism with species k renamed perm[k]."""
    K = m.K
    inv = np.argsort(perm)
    m2 = m.copy()
    for f in ("W", "T_mid", "T_lo", "T_hi"):
        setattr(m2, f, getattr(m, f)[inv].copy())
    for f in ("atoms", "nasa_lo", "nasa_hi", "mu_fit", "lam_fit"):
        setattr(m2, f, getattr(m, f)[inv].copy())
    m2.reac_sp = perm[m.reac_sp].astype(np.int32)
    m2.prod_sp = perm[m.prod_sp].astype(np.int32)
    m2.eff = m.eff[:, inv].copy()
    D = np.zeros_like(m.D_fit)
    for j in range(K):
        for k in range(j + 1, K):
            a, b = sorted((perm[j], perm[k]))
            D[a * K - a * (a + 1) // 2 + (b - a - 1)] = m.D_fit[j * K - j * (j + 1) // 2 + (k - j - 1)]
    m2.D_fit = D
    return m2


def test_species_relabelling(mech53):
    rng = np.random.default_rng(3)
    perm = rng.permutation(mech53.K)
    m2 = permute_species(mech53, perm)
    T, p, Y = _states(mech53, 30, seed=61)
    Y2 = np.empty_like(Y)
    Y2[perm] = Y
    w, h, ws, hs = oracle.rates(mech53, T, p, Y, scales=True)
    w2, h2 = oracle.rates(m2, T, p, Y2)
    assert np.all(np.abs(w2[perm] - w) <= 1e-12 * ws)
    assert np.all(np.abs(h2 - h) <= 1e-12 * hs)
    mu, lam, D = oracle.transport(mech53, T, p, Y)
    mu2, lam2, D2 = oracle.transport(m2, T, p, Y2)
    assert np.allclose(mu2, mu, rtol=1e-13) and np.allclose(lam2, lam, rtol=1e-13)
    assert np.allclose(D2[perm], D, rtol=1e-13)
