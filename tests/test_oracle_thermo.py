"""Pins for the oracle's mixture state and NASA-7 thermodynamics (definition steps 1-2).

The paper names c_p,k, h_k and the mixture c_p (Eq. 1b, Sec. 2) and the ideal-gas state
(Eq. 1d) without formulas; these tests tie the oracle to what thermodynamics fixes:
c_p = dh/dT, c_p/T = ds/dT, continuity at T_mid, the constant-c_p ideal gas, W-bar and
rho of pure species and binary mixtures.
"""
import numpy as np

import oracle
from paper_2409_06404_gb300 import synth
from conftest import R_GAS, P_ATM


def test_cp_is_dh_dT_and_ds_dT_is_cp_over_T(mech53):
    T = np.concatenate([np.linspace(300, 999, 40), np.linspace(1001, 3500, 60)])
    for k in range(0, mech53.K, 5):
        o = oracle.nasa7_cs(mech53, k, T)
        assert np.max(np.abs(o["dh_dT"] - o["cp"]) / np.abs(o["cp"])) < 1e-12
        assert np.max(np.abs(o["ds_dT"] - o["cp"] / T) / np.abs(o["cp"] / T)) < 1e-12


def test_continuity_at_T_mid(mech53, mech9):
    for m in (mech53, mech9):
        for k in range(m.K):
            tm = m.T_mid[k]
            lo = oracle.nasa7_cs(m, k, [tm])                     # T <= T_mid: low range
            hi = oracle.nasa7_cs(m, k, [np.nextafter(tm, 4000.0)])  # high range
            for q in ("cp", "h", "s"):
                scale = max(abs(lo[q][0]), R_GAS * tm)
                assert abs(lo[q][0] - hi[q][0]) <= 1e-9 * scale, (k, q)


def _constant_cp_mech(a1, a6, a7):
    K = 2
    nasa = np.zeros((K, 7))
    nasa[:, 0] = a1
    nasa[:, 5] = a6
    nasa[:, 6] = a7
    return synth.mechanism_from_arrays(
        K=K, R=1, W=np.array([0.028, 0.032]), nasa_lo=nasa, nasa_hi=nasa,
        reac_ptr=[0, 1], reac_sp=[0], reac_nu=[1], prod_ptr=[0, 1], prod_sp=[1], prod_nu=[1],
        lnA=[0.0], beta=[0.0], Ea=[0.0])


def test_constant_cp_ideal_gas():
    # a2..a5 = 0: c_p = a1 R, h = R (a1 T + a6), s = R (a1 ln T + a7)
    m = _constant_cp_mech(3.5, -1000.0, 7.0)
    T = np.array([300.0, 777.0, 1000.0, 2500.0])
    o = oracle.nasa7_cs(m, 0, T)
    assert np.allclose(o["cp"], 3.5 * R_GAS, rtol=1e-15)
    assert np.allclose(o["h"], R_GAS * (3.5 * T - 1000.0), rtol=1e-14)
    assert np.allclose(o["s"], R_GAS * (3.5 * np.log(T) + 7.0), rtol=1e-14)


def test_pure_species_and_binary_mixture_state(mech9):
    K = mech9.K
    T = np.full(K, 1234.0)
    Y = np.eye(K)
    th = oracle.thermo(mech9, T, P_ATM, Y)
    assert np.allclose(th["Wbar"], mech9.W, rtol=1e-15)
    # ideal gas: rho = p W / (R T)
    assert np.allclose(th["rho"], P_ATM * mech9.W / (R_GAS * 1234.0), rtol=1e-14)
    # pure species: mass c_p and h are the molar values over W_k
    for k in range(K):
        assert np.isclose(th["cp_mix"][k], th["cp_k"][k, k] / mech9.W[k], rtol=1e-14)
        assert np.isclose(th["h_mix"][k], th["h_k"][k, k] / mech9.W[k], rtol=1e-13)
    # binary mixture: 1/Wbar = Y1/W1 + Y2/W2
    Y2 = np.zeros((K, 1))
    Y2[0, 0], Y2[3, 0] = 0.25, 0.75
    th2 = oracle.thermo(mech9, [900.0], 2 * P_ATM, Y2)
    assert np.isclose(1.0 / th2["Wbar"][0], 0.25 / mech9.W[0] + 0.75 / mech9.W[3], rtol=1e-15)


def test_mixture_properties_are_mass_weighted(mech53):
    st = synth.states_uniform(mech53.K, 64, seed=11)
    th = oracle.thermo(mech53, st.T, st.p, st.Y)
    # linear in Y: the mass-based mixture value is the Y-weighted mass-based pure value
    cp_pure_mass = th["cp_k"] / mech53.W[:, None]
    assert np.allclose(th["cp_mix"], np.sum(st.Y * cp_pure_mass, axis=0), rtol=1e-13)
    # g = h - T s consistency with the complex-step s of one species
    o = oracle.nasa7_cs(mech53, 7, st.T)
    assert np.allclose(th["g_k"][7], o["h"] - st.T * o["s"], rtol=1e-12, atol=1e-9 * R_GAS * st.T.max())


def test_heat_capacity_stays_on_the_fitted_curve(mech53, mech120):
    """c_p/R of every species stays within the range of the smooth curve it was fitted to
    (c0 in [2.5, 4.5], rise up to 1.5 per atom): evaluating the wrong NASA range, or a
    coefficient in the wrong slot, leaves this band."""
    T = np.linspace(300.0, 3500.0, 161)
    for m in (mech53, mech120):
        for k in range(m.K):
            cp = oracle.nasa7_cs(m, k, T)["cp"] / R_GAS
            top = 4.5 + 1.5 * m.atoms[k].sum()
            assert np.all(cp > 2.3) and np.all(cp < top + 0.3), k
