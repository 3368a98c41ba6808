"""Pins of the oracle's implicit-stage chemistry sources (Eq. 1a-b at fixed p):
fY_k = W_k omega_k / rho, fT = hrr / (rho c_p), and of their complex-step JVP.

Independent of the oracle's own formula: mass conservation (sum_k fY_k = 0), conservation of
the mixture enthalpy in an adiabatic constant-pressure reactor (sum_k h_k/W_k fY_k + c_p fT =
0), the density factor against the separately pinned rho and omega, the pressure scaling of
unimolecular and bimolecular chemistry, the sign of the temperature source of an exothermic
reaction, and the JVP against central differences and the linearised conservation laws.
"""
import numpy as np
import pytest

import oracle
from paper_2409_06404_gb300 import synth
from conftest import R_GAS, P_ATM

MECHS = ["h2_9sp_21rx", "ch4_53sp_325rx"]


def _states(mech, n, seed=3):
    st = synth.states_flame(mech.K, 1, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


@pytest.mark.parametrize("name", MECHS)
def test_mass_conservation(name):
    mech = synth.mechanism(name)
    T, p, Y = _states(mech, 64)
    fT, fY, sT, sY = oracle.rhs(mech, T, p, Y, scales=True)
    assert np.all(np.abs(fY.sum(0)) <= 1e-12 * sY.sum(0))


@pytest.mark.parametrize("name", MECHS)
def test_enthalpy_conservation_at_constant_pressure(name):
    """d/dt of h = sum_k Y_k h_k(T)/W_k vanishes: sum_k h_k/W_k dY_k/dt + c_p dT/dt = 0."""
    mech = synth.mechanism(name)
    T, p, Y = _states(mech, 64)
    fT, fY, sT, sY = oracle.rhs(mech, T, p, Y, scales=True)
    th = oracle.thermo(mech, T, p, Y)
    hk = th["h_k"] / mech.W[:, None]                       # J/kg
    resid = (hk * fY).sum(0) + th["cp_mix"] * fT
    scale = (np.abs(hk) * sY).sum(0) + th["cp_mix"] * sT
    assert np.all(np.abs(resid) <= 1e-12 * scale)


@pytest.mark.parametrize("name", MECHS)
def test_density_factor(name):
    mech = synth.mechanism(name)
    T, p, Y = _states(mech, 32)
    fT, fY, sT, sY = oracle.rhs(mech, T, p, Y, scales=True)
    w, h, ws, hs = oracle.rates(mech, T, p, Y, scales=True)
    rho = oracle.thermo(mech, T, p, Y)["rho"]
    assert np.all(np.abs(fY * rho / mech.W[:, None] - w) <= 1e-13 * ws)
    cp = oracle.thermo(mech, T, p, Y)["cp_mix"]
    assert np.all(np.abs(fT * rho * cp - h) <= 1e-13 * hs)


def _isomers_and_exchange():
    """A <-> B, B <-> C (isomers, W = 0.03) and A + D <-> C + E with W_A + W_D = W_C + W_E."""
    W = np.array([0.03, 0.03, 0.03, 0.02, 0.02])
    nasa = np.zeros((5, 7))
    nasa[:, 0] = [3.5, 3.6, 3.7, 3.3, 3.4]
    nasa[:, 5] = [-1000.0, -3000.0, 500.0, -200.0, -800.0]
    nasa[:, 6] = [4.0, 5.0, 6.0, 3.0, 4.5]
    kw = dict(K=5, R=3, W=W, nasa_lo=nasa, nasa_hi=nasa,
              reac_ptr=[0, 1, 2, 4], reac_sp=[0, 1, 0, 3], reac_nu=[1, 1, 1, 1],
              prod_ptr=[0, 1, 2, 4], prod_sp=[1, 2, 2, 4], prod_nu=[1, 1, 1, 1],
              rtype=[0, 0, 0], lnA=np.log([1e6, 3e5, 2e7]), beta=[0.5, -0.3, 0.0], Ea=[4e4, 2e4, 3e4])
    return synth.mechanism_from_arrays(**kw)


def test_pressure_scaling():
    """At fixed T and Y, C_k and rho scale with p: unimolecular reactions give sources
    independent of p, a bimolecular reaction with no change of mole number scales them by p."""
    base = _isomers_and_exchange()
    uni = synth.mechanism_from_arrays(**{**base.__dict__, "R": 2, "reac_ptr": [0, 1, 2], "reac_sp": [0, 1],
                                         "reac_nu": [1, 1], "prod_ptr": [0, 1, 2], "prod_sp": [1, 2],
                                         "prod_nu": [1, 1], "rtype": [0, 0], "lnA": base.lnA[:2],
                                         "beta": base.beta[:2], "Ea": base.Ea[:2], "lnA0": np.zeros(2),
                                         "beta0": np.zeros(2), "Ea0": np.zeros(2), "troe": np.zeros((2, 4)),
                                         "eff": np.ones((2, 5))})
    bi = synth.mechanism_from_arrays(**{**base.__dict__, "R": 1, "reac_ptr": [0, 2], "reac_sp": [0, 3],
                                        "reac_nu": [1, 1], "prod_ptr": [0, 2], "prod_sp": [2, 4],
                                        "prod_nu": [1, 1], "rtype": [0], "lnA": base.lnA[2:],
                                        "beta": base.beta[2:], "Ea": base.Ea[2:], "lnA0": np.zeros(1),
                                        "beta0": np.zeros(1), "Ea0": np.zeros(1), "troe": np.zeros((1, 4)),
                                        "eff": np.ones((1, 5))})
    rng = np.random.default_rng(4)
    n = 16
    T = rng.uniform(600, 2400, n)
    Y = rng.dirichlet(np.ones(5), n).T.copy()
    for lam in (0.1, 7.0):
        p1, p2 = np.full(n, P_ATM), np.full(n, lam * P_ATM)
        a_T, a_Y = oracle.rhs(uni, T, p1, Y)
        b_T, b_Y = oracle.rhs(uni, T, p2, Y)
        assert np.allclose(b_Y, a_Y, rtol=1e-12, atol=0) and np.allclose(b_T, a_T, rtol=1e-12, atol=0)
        a_T, a_Y = oracle.rhs(bi, T, p1, Y)
        b_T, b_Y = oracle.rhs(bi, T, p2, Y)
        assert np.allclose(b_Y, lam * a_Y, rtol=1e-12, atol=0) and np.allclose(b_T, lam * a_T, rtol=1e-12, atol=0)


def test_exothermic_reaction_heats():
    """A -> B releasing heat (h_f(B) < h_f(A)), started with no B: the temperature rises,
    Y_A falls and Y_B rises by the same mass."""
    W = np.array([0.03, 0.03])
    nasa = np.zeros((2, 7))
    nasa[:, 0] = 3.5
    nasa[:, 5] = [0.0, -2.0e4]                            # h_f(B) - h_f(A) = -R 2e4 K
    nasa[:, 6] = [5.0, 5.0]
    mech = synth.mechanism_from_arrays(K=2, R=1, W=W, nasa_lo=nasa, nasa_hi=nasa, reac_ptr=[0, 1], reac_sp=[0],
                                       reac_nu=[1], prod_ptr=[0, 1], prod_sp=[1], prod_nu=[1], rtype=[0],
                                       lnA=[np.log(1e5)], beta=[0.0], Ea=[0.0])
    T = np.array([800.0, 1500.0])
    p = np.full(2, P_ATM)
    Y = np.array([[1.0, 1.0], [0.0, 0.0]])
    fT, fY = oracle.rhs(mech, T, p, Y)
    assert np.all(fT > 0) and np.all(fY[0] < 0) and np.allclose(fY[1], -fY[0], rtol=1e-14)
    # pure A at rate k: dY_A/dt = -k exactly (W_A omega_A / rho = -k C_A W_A / rho = -k Y_A)
    assert np.allclose(fY[0], -1e5, rtol=1e-13)
    # dT/dt = k (h_A - h_B)/c_p with c_p = 3.5 R / W
    assert np.allclose(fT, 1e5 * R_GAS * 2.0e4 / (3.5 * R_GAS), rtol=1e-12)


@pytest.mark.parametrize("name", MECHS)
def test_jvp_vs_central_differences(name):
    mech = synth.mechanism(name)
    n = 24
    T, p, Y = _states(mech, n, seed=8)
    vT = synth.normal(n, 11)
    vY = synth.normal((mech.K, n), 12) * Y                # relative: keeps tiny Y_k away from 0
    dfT, dfY, sT, sY = oracle.rhs_jvp(mech, T, p, Y, vT, vY, scales=True)
    h = 1e-5
    aT, aY = oracle.rhs(mech, T + h * vT, p, Y + h * vY)
    bT, bY = oracle.rhs(mech, T - h * vT, p, Y - h * vY)
    _, _, s0T, s0Y = oracle.rhs(mech, T, p, Y, scales=True)
    # central differences carry O(h^2) truncation and eps/h rounding against the value scale
    tolT = 1e-6 * sT + 1e-9 * s0T
    tolY = 1e-6 * sY + 1e-9 * s0Y
    assert np.all(np.abs((aT - bT) / (2 * h) - dfT) <= tolT)
    assert np.all(np.abs((aY - bY) / (2 * h) - dfY) <= tolY)


@pytest.mark.parametrize("name", MECHS)
def test_jvp_conservation_laws(name):
    """Both conservation laws hold for every state, so their derivatives along any direction
    vanish: sum_k dfY_k = 0 and sum_k (c_p,k vT fY_k + h_k dfY_k)/W_k + dc_p fT + c_p dfT = 0."""
    mech = synth.mechanism(name)
    n = 32
    T, p, Y = _states(mech, n, seed=9)
    vT = synth.normal(n, 13)
    vY = synth.normal((mech.K, n), 14)
    dfT, dfY, sT, sY = oracle.rhs_jvp(mech, T, p, Y, vT, vY, scales=True)
    assert np.all(np.abs(dfY.sum(0)) <= 1e-12 * sY.sum(0))
    fT, fY, s0T, s0Y = oracle.rhs(mech, T, p, Y, scales=True)
    th = oracle.thermo(mech, T, p, Y)
    W = mech.W[:, None]
    # d c_p along v: c_p is linear in Y and a quartic in T; central difference with a small step
    e = 1e-4
    cpa = oracle.thermo(mech, T + e * vT, p, Y + e * vY)["cp_mix"]
    cpb = oracle.thermo(mech, T - e * vT, p, Y - e * vY)["cp_mix"]
    dcp = (cpa - cpb) / (2 * e)
    resid = (th["cp_k"] * vT / W * fY).sum(0) + (th["h_k"] / W * dfY).sum(0) + dcp * fT + th["cp_mix"] * dfT
    scale = ((np.abs(th["cp_k"] * vT) / W * s0Y).sum(0) + (np.abs(th["h_k"]) / W * sY).sum(0)
             + np.abs(dcp) * s0T + th["cp_mix"] * sT)
    assert np.all(np.abs(resid) <= 1e-9 * scale)
