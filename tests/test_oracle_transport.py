"""Pins for the oracle's mixture-averaged transport (definition step 9).

The paper uses mixture-averaged transport without Soret/Dufour effects (Eq. 2, Sec. 2)
and the mixture viscosity (Eq. 4) and conductivity (Eq. 1b); it prints no mixture rule.
The oracle takes Wilke's rule, the Mathur-Saxena average and the Hirschfelder-Curtiss
mixture-averaged diffusion coefficients.  Pinned here by: pure-species limits, power-law
fits, hand-derived binary mixtures, the 1/p scaling of D, and the textbook form
(1 - Y_k)/sum_{j!=k} X_j/D_jk with binary coefficients extracted from trace limits.
"""
import numpy as np

import oracle
from paper_2409_06404_gb300 import synth
from conftest import P_ATM


def _mech(W, mu_fit, lam_fit, D_fit):
    K = len(W)
    nasa = np.zeros((K, 7))
    nasa[:, 0] = 3.5
    return synth.mechanism_from_arrays(
        K=K, R=1, W=np.array(W, float), nasa_lo=nasa, nasa_hi=nasa, reac_ptr=[0, 1], reac_sp=[0],
        reac_nu=[1], prod_ptr=[0, 1], prod_sp=[1 % K], prod_nu=[1], lnA=[0.0], beta=[0.0], Ea=[0.0],
        mu_fit=np.array(mu_fit, float), lam_fit=np.array(lam_fit, float), D_fit=np.array(D_fit, float))


def test_power_law_fits_and_pure_species_limits():
    # ln v = a0 + a1 ln T: v = exp(a0) T^a1
    W = [0.002, 0.028, 0.044]
    mu_fit = [[np.log(1e-7), 0.7, 0, 0], [np.log(2e-7), 0.65, 0, 0], [np.log(3e-7), 0.6, 0, 0]]
    lam_fit = [[np.log(1e-3), 0.8, 0, 0], [np.log(3e-4), 0.75, 0, 0], [np.log(2e-4), 0.85, 0, 0]]
    D_fit = [[np.log(1e-9), 1.7, 0, 0], [np.log(2e-9), 1.75, 0, 0], [np.log(3e-9), 1.65, 0, 0]]
    m = _mech(W, mu_fit, lam_fit, D_fit)
    T = np.array([500.0, 1500.0, 2500.0])
    for k in range(3):
        Y = np.zeros((3, 3))
        Y[k] = 1.0
        p = np.array([P_ATM, 2 * P_ATM, 0.5 * P_ATM])
        mu, lam, D = oracle.transport(m, T, p, Y)
        assert np.allclose(mu, np.exp(mu_fit[k][0]) * T ** mu_fit[k][1], rtol=1e-13)
        assert np.allclose(lam, np.exp(lam_fit[k][0]) * T ** lam_fit[k][1], rtol=1e-13)
        # trace species j in pure k: D_jm = D_jk; the pure species itself gets 0
        for j in range(3):
            if j == k:
                assert np.all(D[j] == 0.0)
                continue
            a, b = sorted((j, k))
            pi = a * 3 - a * (a + 1) // 2 + (b - a - 1)
            Djk = np.exp(D_fit[pi][0]) * T ** D_fit[pi][1] * P_ATM / p
            assert np.allclose(D[j], Djk, rtol=1e-13)


def test_wilke_binary_hand_values():
    # equal molar masses, mu_2 = 4 mu_1: Phi_12 = (1/4)(1 + 1/2)^2, Phi_21 = (1/4)(1 + 2)^2
    T = np.array([1000.0])
    m = _mech([0.03, 0.03], [[np.log(1e-5), 0, 0, 0], [np.log(4e-5), 0, 0, 0]],
              [[0, 0, 0, 0], [0, 0, 0, 0]], [[np.log(1e-5), 0, 0, 0]])
    Y = np.array([[0.5], [0.5]])
    mu, _, _ = oracle.transport(m, T, P_ATM, Y)
    phi12, phi21 = 0.25 * 1.5 ** 2, 0.25 * 3.0 ** 2
    expect = 1e-5 * (0.5 / (0.5 + 0.5 * phi12) + 0.5 * 4 / (0.5 + 0.5 * phi21))
    assert np.isclose(mu[0], expect, rtol=1e-14)
    # identical gases: the mixture viscosity is the species viscosity at any composition
    m = _mech([0.03, 0.03], [[np.log(2e-5), 0, 0, 0]] * 2, [[0, 0, 0, 0]] * 2, [[np.log(1e-5), 0, 0, 0]])
    for y in (0.1, 0.5, 0.9):
        mu, _, _ = oracle.transport(m, T, P_ATM, np.array([[y], [1 - y]]))
        assert np.isclose(mu[0], 2e-5, rtol=1e-14)
    # equal viscosities, W_2 = 16 W_1 (mole fractions 1/2 each):
    # Phi_12 = 8^-1/2 (17/16)^-1/2 (1 + 16^1/4)^2 = 18/sqrt(34),
    # Phi_21 = 8^-1/2 17^-1/2 (1 + 16^-1/4)^2 = 2.25/sqrt(136)
    m = _mech([0.002, 0.032], [[np.log(2e-5), 0, 0, 0]] * 2, [[0, 0, 0, 0]] * 2, [[np.log(1e-5), 0, 0, 0]])
    Wb = 2.0 / (1 / 0.002 + 1 / 0.032)        # X = (1/2, 1/2)
    Y = np.array([[0.5 * 0.002 / Wb], [0.5 * 0.032 / Wb]])
    mu, _, _ = oracle.transport(m, T, P_ATM, Y)
    phi12, phi21 = 18.0 / np.sqrt(34.0), 2.25 / np.sqrt(136.0)
    expect = 2e-5 * (0.5 / (0.5 + 0.5 * phi12) + 0.5 / (0.5 + 0.5 * phi21))
    assert np.isclose(mu[0], expect, rtol=1e-13)


def test_mathur_binary_hand_value():
    # lambda_2 = 4 lambda_1, X = (1/2, 1/2): 1/2 (2.5 + 1/0.625) lambda_1 = 2.05 lambda_1
    m = _mech([0.03, 0.03], [[np.log(1e-5), 0, 0, 0]] * 2, [[np.log(0.01), 0, 0, 0], [np.log(0.04), 0, 0, 0]],
              [[np.log(1e-5), 0, 0, 0]])
    _, lam, _ = oracle.transport(m, np.array([900.0]), P_ATM, np.array([[0.5], [0.5]]))
    assert np.isclose(lam[0], 2.05 * 0.01, rtol=1e-14)


def test_diffusion_pressure_scaling(mech53):
    st = synth.states_uniform(mech53.K, 40, seed=71)
    _, _, D1 = oracle.transport(mech53, st.T, P_ATM, st.Y)
    _, _, D2 = oracle.transport(mech53, st.T, 2 * P_ATM, st.Y)
    assert np.allclose(D2, D1 / 2, rtol=1e-14)


def test_hirschfelder_curtiss_textbook_form(mech9):
    """For sum Y = 1, D_km = (1 - Y_k) / sum_{j!=k} X_j/D_jk, with D_jk taken from trace limits."""
    m = mech9
    K = m.K
    T0 = 1700.0
    # binary coefficients from the pure-species limits of the oracle itself
    Dbin = np.zeros((K, K))
    for k in range(K):
        Y = np.zeros((K, 1))
        Y[k] = 1.0
        _, _, D = oracle.transport(m, [T0], P_ATM, Y)
        Dbin[:, k] = D[:, 0]
    assert np.allclose(Dbin, Dbin.T, rtol=1e-14)           # D_jk = D_kj
    st = synth.states_uniform(K, 20, seed=72)
    Y = st.Y
    _, _, D = oracle.transport(m, np.full(20, T0), P_ATM, Y)
    X = (Y / m.W[:, None]) / np.sum(Y / m.W[:, None], axis=0)
    for k in range(K):
        s = sum(X[j] / Dbin[j, k] for j in range(K) if j != k)
        assert np.allclose(D[k], (1 - Y[k]) / s, rtol=1e-12)


def test_mixture_values_within_species_bounds(mech53):
    st = synth.states_uniform(mech53.K, 50, seed=73)
    mu, lam, D = oracle.transport(mech53, st.T, st.p, st.Y)
    L = np.log(st.T)
    V = np.stack([np.ones_like(L), L, L ** 2, L ** 3])
    lam_k = np.exp(mech53.lam_fit @ V)
    X = (st.Y / mech53.W[:, None]) / np.sum(st.Y / mech53.W[:, None], axis=0)
    # the Mathur average lies between the harmonic and arithmetic means
    assert np.all(lam <= np.sum(X * lam_k, axis=0) * (1 + 1e-14))
    assert np.all(lam >= 1 / np.sum(X / lam_k, axis=0) * (1 - 1e-14))
    assert np.all(mu > 0) and np.all(D > 0)
