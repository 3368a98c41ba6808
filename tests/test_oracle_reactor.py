"""Pins of the oracle's implicit Euler reactor step (x1 - x0 - dt f(x1) = 0 per point, dense
Newton): the defining residual through the separate source evaluation, the linear invariants
every backward Euler step keeps (sum_k Y_k and the element mass fractions, since
sum_k dY_k/dt and sum_k a_ek/W_k dY_k/dt vanish), the closed-form step of an isothermal
isomerisation, and equilibrium as a fixed point."""
import numpy as np
import pytest

import oracle
from paper_2409_06404_gb300 import synth
from conftest import P_ATM
from test_oracle_rates import equilibrium_state


def _near_equilibrium(mech, n, seed, pert=1e-3):
    rng = np.random.default_rng(seed)
    T = rng.uniform(1300.0, 2600.0, n)
    p = np.full(n, P_ATM)
    Y = np.stack([equilibrium_state(mech, T[i], p[i], rng) for i in range(n)], axis=1)
    Y = Y * (1.0 + pert * rng.standard_normal(Y.shape))
    Y /= Y.sum(0)
    return T + pert * 1e3 * rng.standard_normal(n), p, np.ascontiguousarray(Y)


@pytest.mark.parametrize("dt", [1e-9, 1e-6])
def test_residual_and_invariants(dt):
    mech = synth.mechanism("h2_9sp_21rx")
    T, p, Y = _near_equilibrium(mech, 12, 1)
    T1, Y1, it = oracle.reactor_step(mech, T, p, Y, dt)
    assert np.all(it > 0)
    fT, fY, sT, sY = oracle.rhs(mech, T1, p, Y1, scales=True)
    # the residual is at the rounding level of the terms it is made of, plus the Newton
    # tolerance's absolute part (1e-14 of atol_Y = 1e-16, amplified by I - dt J)
    assert np.all(np.abs(T1 - T - dt * fT) <= 1e-12 * (np.abs(T1) + dt * sT))
    assert np.all(np.abs(Y1 - Y - dt * fY) <= 1e-12 * (np.abs(Y1) + np.abs(Y) + dt * sY) + 1e-20)
    assert np.allclose(Y1.sum(0), Y.sum(0), rtol=0, atol=1e-14)
    a = mech.atoms.astype(float) / mech.W[:, None]          # element moles per kg
    assert np.allclose(a.T @ Y1, a.T @ Y, rtol=1e-12, atol=1e-14)


def test_isomerization_closed_form():
    """A <-> B with identical thermochemistry (K_c = 1, k_r = k_f = k, no heat release, equal
    W): dY_A/dt = -k Y_A + k Y_B, so with Y_A + Y_B = 1 the backward Euler step is
    Y_A1 = (Y_A0 + dt k) / (1 + 2 dt k), and T does not change."""
    W = np.array([0.03, 0.03])
    nasa = np.zeros((2, 7))
    nasa[:, 0] = 3.5
    nasa[:, 6] = 4.0
    A, Ea = 1e7, 5e4
    mech = synth.mechanism_from_arrays(K=2, R=1, W=W, nasa_lo=nasa, nasa_hi=nasa, reac_ptr=[0, 1], reac_sp=[0],
                                       reac_nu=[1], prod_ptr=[0, 1], prod_sp=[1], prod_nu=[1], rtype=[0],
                                       lnA=[np.log(A)], beta=[0.0], Ea=[Ea])
    T = np.array([900.0, 1500.0, 2200.0])
    p = np.full(3, P_ATM)
    YA = np.array([0.9, 0.2, 0.55])
    Y = np.vstack([YA, 1.0 - YA])
    k = A * np.exp(-Ea / (8.314462618 * T))
    for dt in (1e-9, 1e-5, 1e-2):
        T1, Y1, it = oracle.reactor_step(mech, T, p, Y, dt)
        assert np.all(it > 0)
        assert np.allclose(Y1[0], (YA + dt * k) / (1.0 + 2.0 * dt * k), rtol=1e-12, atol=0)
        assert np.allclose(Y1.sum(0), 1.0, rtol=0, atol=1e-15)
        assert np.allclose(T1, T, rtol=1e-14, atol=0)


def test_equilibrium_is_a_fixed_point():
    mech = synth.mechanism("h2_9sp_21rx")
    T, p, Y = _near_equilibrium(mech, 6, 3, pert=0.0)
    for dt in (1e-8, 1e-3):
        T1, Y1, it = oracle.reactor_step(mech, T, p, Y, dt)
        assert np.all(it > 0)
        assert np.allclose(T1, T, rtol=1e-12, atol=0)
        assert np.allclose(Y1, Y, rtol=1e-9, atol=1e-20)
