"""Pins of the oracle's dense Jacobian of the implicit-stage sources (rows fT, fY_k; columns T,
Y_j; complex step per column).

Independent of the complex-step driver: central differences of the separately pinned sources;
the derivatives of identities the sources satisfy at every state (sum_k fY_k = 0, the element
mass balance sum_k a_ek/W_k fY_k = 0, and the enthalpy balance of an adiabatic
constant-pressure reactor, sum_k h_k/W_k fY_k + c_p fT = 0, whose derivative ties the
temperature row to the species rows); the closed form of an isothermal isomerisation A <-> B.
"""
import numpy as np
import pytest

import oracle
from paper_2409_06404_gb300 import synth
from conftest import R_GAS

MECHS = ["h2_9sp_21rx", "ch4_53sp_325rx"]


def _states(mech, n, seed=3):
    st = synth.states_flame(mech.K, 1, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


@pytest.mark.parametrize("name", MECHS)
def test_columns_match_central_differences(name):
    mech = synth.mechanism(name)
    T, p, Y = _states(mech, 3, seed=5)
    J = oracle.rhs_jacobian(mech, T, p, Y)
    K = mech.K
    for j in range(K + 1):
        step = 1e-6 * (T if j == 0 else np.maximum(Y[j - 1], 1e-3))
        Tp, Tm, Yp, Ym = T.copy(), T.copy(), Y.copy(), Y.copy()
        if j == 0:
            Tp += step
            Tm -= step
        else:
            Yp[j - 1] += step
            Ym[j - 1] -= step
        fTp, fYp, sTp, sYp = oracle.rhs(mech, Tp, p, Yp, scales=True)
        fTm, fYm = oracle.rhs(mech, Tm, p, Ym)
        # the error of a central difference is relative to the magnitudes behind the sources
        assert np.all(np.abs(J[:, 0, j] - (fTp - fTm) / (2 * step)) <= 1e-6 * sTp / step), j
        assert np.all(np.abs(J[:, 1:, j].T - (fYp - fYm) / (2 * step)) <= 1e-6 * sYp / step), j


@pytest.mark.parametrize("name", MECHS)
def test_conservation_rows(name):
    mech = synth.mechanism(name)
    T, p, Y = _states(mech, 24, seed=6)
    J, Js = oracle.rhs_jacobian(mech, T, p, Y, scales=True)
    JY, SY = J[:, 1:, :], Js[:, 1:, :]
    assert np.all(np.abs(JY.sum(axis=1)) <= 1e-11 * SY.sum(axis=1))
    a = mech.atoms.astype(float) / mech.W[:, None]              # [K, elements]
    for e in range(a.shape[1]):
        bal = np.einsum("k,nkj->nj", a[:, e], JY)
        assert np.all(np.abs(bal) <= 1e-11 * np.einsum("k,nkj->nj", a[:, e], SY) + 1e-300)


@pytest.mark.parametrize("name", MECHS)
def test_enthalpy_balance_ties_the_temperature_row(name):
    """d/dx_j of sum_k h_k/W_k fY_k + c_p fT = 0: for Y_j, sum_k h_k/W_k J[Y_k, Y_j] +
    c_p J[T, Y_j] + (c_p,j/W_j) fT = 0; for T, sum_k (c_p,k/W_k fY_k + h_k/W_k J[Y_k, T]) +
    (dc_p/dT) fT + c_p J[T, T] = 0."""
    mech = synth.mechanism(name)
    T, p, Y = _states(mech, 24, seed=7)
    J, Js = oracle.rhs_jacobian(mech, T, p, Y, scales=True)
    fT, fY = oracle.rhs(mech, T, p, Y)
    th = oracle.thermo(mech, T, p, Y)
    hk = th["h_k"] / mech.W[:, None]                            # [K, n] J/kg
    cpk = th["cp_k"] / mech.W[:, None]
    cp = th["cp_mix"]
    # dc_p/dT by central differences of the separately pinned thermo
    dT = 1e-3 * T
    dcp = (oracle.thermo(mech, T + dT, p, Y)["cp_mix"] - oracle.thermo(mech, T - dT, p, Y)["cp_mix"]) / (2 * dT)
    JY, JT = J[:, 1:, :], J[:, 0, :]
    SY, ST = Js[:, 1:, :], Js[:, 0, :]
    resY = np.einsum("kn,nkj->nj", hk, JY[:, :, 1:]) + cp[:, None] * JT[:, 1:] + (cpk * fT[None]).T
    scY = np.einsum("kn,nkj->nj", np.abs(hk), SY[:, :, 1:]) + cp[:, None] * ST[:, 1:] + np.abs(cpk * fT[None]).T
    assert np.all(np.abs(resY) <= 1e-11 * scY)
    resT = (cpk * fY).sum(0) + np.einsum("kn,nk->n", hk, JY[:, :, 0]) + dcp * fT + cp * JT[:, 0]
    scT = (np.abs(cpk * fY)).sum(0) + np.einsum("kn,nk->n", np.abs(hk), SY[:, :, 0]) + np.abs(dcp * fT) + cp * ST[:, 0]
    assert np.all(np.abs(resT) <= 1e-7 * scT)                   # (dc_p/dT by differences)


def test_isomerization_closed_form():
    """A <-> B with identical thermochemistry and equal W: fY_A = k (Y_B - Y_A) = -fY_B with
    k = A exp(-Ea/(R T)), fT = 0 at every state."""
    W = np.array([0.03, 0.03])
    nasa = np.zeros((2, 7))
    nasa[:, 0] = 3.5
    nasa[:, 6] = 4.0
    A, Ea = 1e7, 5e4
    mech = synth.mechanism_from_arrays(K=2, R=1, W=W, nasa_lo=nasa, nasa_hi=nasa, reac_ptr=[0, 1], reac_sp=[0],
                                       reac_nu=[1], prod_ptr=[0, 1], prod_sp=[1], prod_nu=[1], rtype=[0],
                                       lnA=[np.log(A)], beta=[0.0], Ea=[Ea])
    T = np.array([900.0, 1500.0, 2200.0])
    p = np.full(3, 101325.0)
    YA = np.array([0.9, 0.2, 0.55])
    Y = np.vstack([YA, 1.0 - YA])
    J = oracle.rhs_jacobian(mech, T, p, Y)
    k = A * np.exp(-Ea / (R_GAS * T))
    dk = k * Ea / (R_GAS * T ** 2)
    expect = np.zeros((3, 3, 3))
    expect[:, 1, 1] = -k
    expect[:, 1, 2] = k
    expect[:, 2, 1] = k
    expect[:, 2, 2] = -k
    expect[:, 1, 0] = dk * (Y[1] - Y[0])
    expect[:, 2, 0] = -dk * (Y[1] - Y[0])
    assert np.allclose(J, expect, rtol=1e-12, atol=1e-12 * k.max())
    assert np.all(J[:, 0, :] == 0.0)
