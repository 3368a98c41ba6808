"""Pins of the oracle's mixture-averaged diffusion fluxes (Eq. 2 and its correction velocity):
the fluxes sum to zero (the correction velocity's purpose), the binary mixture reduces to
Fick's law in mass fractions, a trace species diffuses by its own gradient alone, a uniform
composition has no flux, the fluxes are linear in the gradients, and the enthalpy-flux factor
is sum_k c_p,k j_k with the separately pinned heat capacities."""
import numpy as np
import pytest

import oracle
from paper_2409_06404_gb300 import synth
from conftest import P_ATM


def _case(mech, n, seed):
    rng = np.random.default_rng(seed)
    st = synth.states_flame(mech.K, 1, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    D = np.exp(rng.uniform(np.log(5e-6), np.log(8e-5), (mech.K, n)))
    G = rng.standard_normal((3, mech.K, n)) * 50.0
    return T, p, Y, D, G


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
def test_fluxes_sum_to_zero(name):
    mech = synth.mechanism(name)
    T, p, Y, D, G = _case(mech, 48, 3)
    j, Vc, hf = oracle.diffusion(mech, T, p, Y, D, G)
    scale = np.abs(j).sum(axis=1)
    resid = np.abs(j.sum(axis=1))
    # sum_k Y_k = 1 up to the generator's rounding
    assert np.all(resid <= 1e-13 * scale + np.abs(Y.sum(0) - 1.0) * scale)


def _binary():
    W = np.array([0.002, 0.032])
    nasa = np.zeros((2, 7))
    nasa[:, 0] = [3.5, 3.6]
    return synth.mechanism_from_arrays(K=2, R=1, W=W, nasa_lo=nasa, nasa_hi=nasa, reac_ptr=[0, 1], reac_sp=[0],
                                       reac_nu=[1], prod_ptr=[0, 1], prod_sp=[1], prod_nu=[1], rtype=[0],
                                       lnA=[0.0], beta=[0.0], Ea=[0.0])


def test_binary_reduces_to_fick_in_mass_fractions():
    """Binary mixture: the mixture-averaged coefficients are D_1 = (W_2/Wbar) D_12 and
    D_2 = (W_1/Wbar) D_12; with grad X_2 = -grad X_1 the correction vanishes and
    j_1 = -rho D_12 grad Y_1, grad Y_1 = (W_1 W_2/Wbar^2) grad X_1."""
    mech = _binary()
    n = 8
    rng = np.random.default_rng(1)
    T = rng.uniform(300, 2500, n)
    p = np.full(n, P_ATM)
    Y1 = rng.uniform(0.05, 0.95, n)
    Y = np.vstack([Y1, 1.0 - Y1])
    W1, W2 = mech.W
    Wbar = 1.0 / (Y[0] / W1 + Y[1] / W2)
    D12 = rng.uniform(1e-5, 1e-4, n)
    D = np.vstack([W2 / Wbar * D12, W1 / Wbar * D12])
    g = rng.standard_normal((3, n)) * 30.0
    G = np.stack([g, -g], axis=1)
    j, Vc, hf = oracle.diffusion(mech, T, p, Y, D, G)
    rho = oracle.thermo(mech, T, p, Y)["rho"]
    expect = -rho * D12 * (W1 * W2 / Wbar ** 2) * g
    assert np.allclose(j[:, 0], expect, rtol=1e-13, atol=0)
    assert np.allclose(j[:, 1], -expect, rtol=1e-13, atol=0)
    assert np.all(np.abs(Vc) <= 1e-15 * np.abs(expect / rho[None, :]))


def test_trace_species_and_uniform_composition():
    mech = synth.mechanism("h2_9sp_21rx")
    T, p, Y, D, G = _case(mech, 16, 5)
    Y = Y.copy()
    Y[2] = 1e-14 * Y[2]
    Y /= Y.sum(0)
    j, Vc, hf = oracle.diffusion(mech, T, p, Y, D, G)
    th = oracle.thermo(mech, T, p, Y)
    rho, Wbar = th["rho"], th["Wbar"]
    own = -rho * (mech.W[2] / Wbar) * D[2] * G[:, 2]
    assert np.allclose(j[:, 2], own, rtol=1e-10, atol=0)
    # no gradient, no flux
    j0, Vc0, hf0 = oracle.diffusion(mech, T, p, Y, D, np.zeros_like(G))
    assert np.all(j0 == 0.0) and np.all(Vc0 == 0.0) and np.all(hf0 == 0.0)


def test_linear_in_gradients_and_enthalpy_factor():
    mech = synth.mechanism("ch4_53sp_325rx")
    T, p, Y, D, G = _case(mech, 16, 7)
    G2 = synth.normal(G.shape, 8) * 10.0
    a, b = 0.7, -2.5
    j1, V1, h1 = oracle.diffusion(mech, T, p, Y, D, G)
    j2, V2, h2 = oracle.diffusion(mech, T, p, Y, D, G2)
    j3, V3, h3 = oracle.diffusion(mech, T, p, Y, D, a * G + b * G2)
    sc = np.abs(a * j1) + np.abs(b * j2)
    assert np.all(np.abs(j3 - (a * j1 + b * j2)) <= 1e-13 * sc.max(axis=1, keepdims=True))
    cpk = oracle.thermo(mech, T, p, Y)["cp_k"] / mech.W[:, None]        # J/kg/K
    hsc = (np.abs(cpk[None] * j1)).sum(axis=1)
    assert np.all(np.abs(h1 - (cpk[None] * j1).sum(axis=1)) <= 1e-13 * hsc)
