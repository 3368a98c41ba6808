"""Implicit Euler step of the homogeneous reactor (nk_reactor_step: Newton with one GMRES solve
over all points per iteration, exact JVPs, single-precision Krylov basis) against the oracle's
dense per-point Newton solution of the same nonlinear system.

States: chemical equilibria from element potentials (as in the rates pins) at flame-like
temperatures, perturbed by 1e-3 in the mass fractions and by ~1 K, so that the step relaxes a
stiff perturbation; dt from 1e-9 s (a few Krylov iterations) to 1e-5 s (stiffer)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, P_ATM
from test_oracle_rates import equilibrium_state

pytestmark = pytest.mark.gpu


def _near_equilibrium(mech, n, seed):
    rng = np.random.default_rng(seed)
    T = rng.uniform(1300.0, 2600.0, n)
    p = np.full(n, P_ATM)
    Y = np.stack([equilibrium_state(mech, T[i], p[i], rng) for i in range(n)], axis=1)
    Y = Y * (1.0 + 1e-3 * rng.standard_normal(Y.shape))
    Y /= Y.sum(0)
    T = T + rng.standard_normal(n)
    return T, p, np.ascontiguousarray(Y)


def _step(m, T, p, Y, dt, **kw):
    o = nk.reactor_opts(**kw)
    T1, Y1 = T.clone(), Y.clone()
    st = nk.reactor_step(m, T1, p, Y1, dt, o)
    return T1, Y1, st


# Without a preconditioner the global Krylov solve must resolve every point's stiff modes at
# once; these steps stay in the regime where it converges within a few cycles (the paper's
# small DNS steps, Sec. 2).
@pytest.mark.parametrize("name,n,dt", [("h2_9sp_21rx", 600, 1e-11), ("h2_9sp_21rx", 600, 1e-9),
                                       ("h2_9sp_21rx", 600, 1e-7), ("ch4_53sp_325rx", 160, 1e-9),
                                       ("ch4_53sp_325rx", 160, 1e-7), ("ch4_53sp_325rx", 160, 1e-5)])
def test_reactor_step_vs_dense_newton(cuda, name, n, dt):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _near_equilibrium(mech, n, seed=17)
    rtol, atolT, atolY = 1e-6, 1e-6, 1e-12
    T1, Y1, st = _step(m, *to_dev(T, p, Y), dt, rtol=rtol, atol_T=atolT, atol_Y=atolY, newton_tol=1e-4,
                       lin_tol=1e-6, max_newton=50, krylov_dim=30)
    assert st["converged"] == 1, st
    T_o, Y_o, it = oracle.reactor_step(mech, T, p, Y, dt, atol_T=atolT, atol_Y=atolY)
    assert np.all(it > 0)
    # weighted RMS difference with the step's own weights (rtol |x0| + atol)
    wT = 1.0 / (rtol * np.abs(T) + atolT)
    wY = 1.0 / (rtol * np.abs(Y) + atolY)
    d = np.concatenate([((host(T1) - T_o) * wT)[None], (host(Y1) - Y_o) * wY])
    wrms = np.sqrt(np.mean(d ** 2))
    print(f"\n{name} dt={dt:g}: newton {st['newton_iters']}, krylov {st['krylov_iters']}, wrms diff {wrms:.2e}")
    assert wrms <= 1e-3                                    # 1e-3 of the weights: ~1e-9 relative


def test_reactor_step_moving_states_53sp(cuda):
    """53 species on states where chemistry moves: the synthetic mechanism's equilibria hold most
    species near 1e-157 (net rates ~1e-25/s, a frozen step), so they are blended with 1e-20 of a
    Dirichlet(0.3) composition (those species at ~1e-22).  The block-Jacobi step at dt = 1e-10 s
    then needs several Newton and Krylov iterations; its result against the oracle's dense Newton
    solution."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y = _near_equilibrium(mech, 96, seed=23)
    rng = np.random.default_rng(24)
    Y = (1.0 - 1e-20) * Y + 1e-20 * rng.dirichlet(np.full(mech.K, 0.3), size=96).T
    Y = np.ascontiguousarray(Y / Y.sum(0))
    rtol, atolT, atolY, dt = 1e-6, 1e-6, 1e-12, 1e-10
    T1, Y1, st = _step(m, *to_dev(T, p, Y), dt, rtol=rtol, atol_T=atolT, atol_Y=atolY, newton_tol=1e-4,
                       lin_tol=1e-6, max_newton=20, krylov_dim=30, precond=1)
    assert st["converged"] == 1, st
    assert st["krylov_iters"] > 1 and st["newton_iters"] > 1, st
    T_o, Y_o, it = oracle.reactor_step(mech, T, p, Y, dt, atol_T=atolT, atol_Y=atolY)
    assert np.all(it > 0)
    wT = 1.0 / (rtol * np.abs(T) + atolT)
    wY = 1.0 / (rtol * np.abs(Y) + atolY)
    d = np.concatenate([((host(T1) - T_o) * wT)[None], (host(Y1) - Y_o) * wY])
    assert np.sqrt(np.mean(d ** 2)) <= 1e-3
    # the step moved the state (the oracle's own change, in the same weights)
    moved = np.concatenate([((T_o - T) * wT)[None], (Y_o - Y) * wY])
    print(f"\n53 species moving: newton {st['newton_iters']}, krylov {st['krylov_iters']}, "
          f"oracle change {np.sqrt(np.mean(moved ** 2)):.2e}")
    assert np.max(np.abs(moved)) > 0.0


def test_reactor_step_edge_cases(cuda):
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    T, p, Y = _near_equilibrium(mech, 64, seed=3)
    Tt, pt, Yt = to_dev(T, p, Y)
    # dt = 0: the state is the solution
    T1, Y1, st = _step(m, Tt, pt, Yt, 0.0)
    assert st["converged"] == 1 and torch.equal(T1, Tt) and torch.equal(Y1, Yt)
    # bad options are argument errors
    with pytest.raises(nk.NkError):
        _step(m, Tt, pt, Yt, 1e-9, krylov_dim=0)
    with pytest.raises(nk.NkError):
        _step(m, Tt, pt, Yt, -1.0)
    # workspace size grows with the Krylov dimension
    assert nk.reactor_workspace(m, 64, 30) > nk.reactor_workspace(m, 64, 5) > 0


def _perturbed_equilibrium(mech, n, seed, pert=0.3):
    """Equilibria with log-normal perturbations of pert in the mass fractions and 30 pert K in
    T: with the 9-species mechanism the step then relaxes active chemistry (the weighted change
    over 1e-3 s is O(0.1))."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(1300.0, 2600.0, n)
    p = np.full(n, P_ATM)
    Y = np.stack([equilibrium_state(mech, T[i], p[i], rng) for i in range(n)], axis=1)
    Y = Y * np.exp(pert * rng.standard_normal(Y.shape))
    Y /= Y.sum(0)
    T = T + 30.0 * pert * rng.standard_normal(n)
    return T, p, np.ascontiguousarray(Y)


# With the per-point block-Jacobi preconditioner the Krylov solve no longer has to resolve the
# stiff modes itself: large steps converge within a few iterations per Newton iteration.
@pytest.mark.parametrize("name,n,dt", [("h2_9sp_21rx", 600, 1e-9), ("h2_9sp_21rx", 600, 1e-6),
                                       ("h2_9sp_21rx", 600, 1e-4), ("h2_9sp_21rx", 600, 1e-3),
                                       ("ch4_53sp_325rx", 160, 1e-5), ("ch4_53sp_325rx", 160, 1e-3),
                                       ("big_120sp_700rx", 40, 1e-5)])
def test_preconditioned_step_vs_dense_newton(cuda, name, n, dt):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _perturbed_equilibrium(mech, n, seed=29)
    rtol, atolT, atolY = 1e-6, 1e-6, 1e-12
    T1, Y1, st = _step(m, *to_dev(T, p, Y), dt, rtol=rtol, atol_T=atolT, atol_Y=atolY, newton_tol=1e-4,
                       lin_tol=1e-6, max_newton=30, krylov_dim=10, precond=1)
    assert st["converged"] == 1, st
    T_o, Y_o, it = oracle.reactor_step(mech, T, p, Y, dt, atol_T=atolT, atol_Y=atolY)
    assert np.all(it > 0)
    wT = 1.0 / (rtol * np.abs(T) + atolT)
    wY = 1.0 / (rtol * np.abs(Y) + atolY)
    d = np.concatenate([((host(T1) - T_o) * wT)[None], (host(Y1) - Y_o) * wY])
    wrms = np.sqrt(np.mean(d ** 2))
    change = np.sqrt(np.mean(np.concatenate([((T_o - T) * wT)[None], (Y_o - Y) * wY]) ** 2))
    print(f"\n{name} dt={dt:g}: newton {st['newton_iters']}, krylov {st['krylov_iters']}, "
          f"step change {change:.2e}, wrms diff {wrms:.2e}")
    assert wrms <= 1e-3
    assert st["krylov_iters"] <= 10 * st["newton_iters"]


@pytest.mark.parametrize("name,n,dt,precond,linearized", [
    ("h2_9sp_21rx", 600, 1e-9, 0, 1), ("ch4_53sp_325rx", 160, 1e-7, 0, 1), ("h2_9sp_21rx", 600, 1e-4, 1, 1),
    ("h2_9sp_21rx", 600, 1e-9, 0, 2), ("ch4_53sp_325rx", 160, 1e-7, 0, 2), ("big_120sp_700rx", 64, 1e-8, 0, 2)])
def test_linearized_products_vs_dense_newton(cuda, name, n, dt, precond, linearized):
    """GMRES products from a stored linearization refreshed per Newton iteration, in double
    (linearized 1) or rounded to float with single-precision products (2): the same solution
    as the oracle's dense Newton (the residual, and so the converged state, is double in both)."""
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _perturbed_equilibrium(mech, n, seed=41) if precond else _near_equilibrium(mech, n, seed=41)
    rtol, atolT, atolY = 1e-6, 1e-6, 1e-12
    T1, Y1, st = _step(m, *to_dev(T, p, Y), dt, rtol=rtol, atol_T=atolT, atol_Y=atolY, newton_tol=1e-4,
                       lin_tol=1e-6, max_newton=30, krylov_dim=30, precond=precond, linearized=linearized)
    assert st["converged"] == 1, st
    T_o, Y_o, it = oracle.reactor_step(mech, T, p, Y, dt, atol_T=atolT, atol_Y=atolY)
    assert np.all(it > 0)
    wT = 1.0 / (rtol * np.abs(T) + atolT)
    wY = 1.0 / (rtol * np.abs(Y) + atolY)
    d = np.concatenate([((host(T1) - T_o) * wT)[None], (host(Y1) - Y_o) * wY])
    assert np.sqrt(np.mean(d ** 2)) <= 1e-3


def test_preconditioned_and_plain_solves_agree(cuda):
    """Where both converge (small steps) the two solves reach the same solution."""
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    T, p, Y = _perturbed_equilibrium(mech, 300, seed=31)
    kw = dict(rtol=1e-6, atol_T=1e-6, atol_Y=1e-12, newton_tol=1e-5, lin_tol=1e-7, max_newton=30, krylov_dim=30)
    Ta, Ya, sa = _step(m, *to_dev(T, p, Y), 1e-9, **kw)
    Tb, Yb, sb = _step(m, *to_dev(T, p, Y), 1e-9, precond=1, **kw)
    assert sa["converged"] == 1 and sb["converged"] == 1
    wY = 1.0 / (1e-6 * np.abs(Y) + 1e-12)
    assert np.sqrt(np.mean(((host(Ya) - host(Yb)) * wY) ** 2)) <= 1e-3
    assert np.sqrt(np.mean(((host(Ta) - host(Tb)) / (1e-6 * T + 1e-6)) ** 2)) <= 1e-3


def test_preconditioned_workspace_and_limits(cuda):
    m = gpu_mechanism("h2_9sp_21rx")
    assert nk.reactor_workspace(m, 64, 10, 1) > nk.reactor_workspace(m, 64, 10, 0)
    with pytest.raises(nk.NkError):
        nk.reactor_workspace(m, 64, 10, 3)
    assert nk.reactor_workspace(m, 64, 10, 0, 1) > nk.reactor_workspace(m, 64, 10, 0, 2) > \
        nk.reactor_workspace(m, 64, 10, 0, 0)
    with pytest.raises(nk.NkError):
        nk.reactor_workspace(m, 64, 10, 0, 3)
    with pytest.raises(nk.NkError):                    # single-precision products, no preconditioner
        nk.reactor_workspace(m, 64, 10, 1, 2)


def test_reused_factors(cuda):
    """precond = 2 keeps the factors of the previous call: a second step from the same states
    reaches the same solution without the set-up."""
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    T, p, Y = _perturbed_equilibrium(mech, 400, seed=37)
    kw = dict(rtol=1e-6, atol_T=1e-6, atol_Y=1e-12, newton_tol=1e-4, lin_tol=1e-6, max_newton=30, krylov_dim=10)
    Tt, pt, Yt = to_dev(T, p, Y)
    ws = torch.empty(nk.reactor_workspace(m, 400, 10, 1), dtype=torch.uint8, device="cuda")
    Ta, Ya = Tt.clone(), Yt.clone()
    sa = nk.reactor_step(m, Ta, pt, Ya, 1e-5, nk.reactor_opts(precond=1, **kw), workspace=ws)
    Tb, Yb = Tt.clone(), Yt.clone()
    sb = nk.reactor_step(m, Tb, pt, Yb, 1e-5, nk.reactor_opts(precond=2, **kw), workspace=ws)
    assert sa["converged"] == 1 and sb["converged"] == 1
    wY = 1.0 / (1e-6 * np.abs(Y) + 1e-12)
    assert np.sqrt(np.mean(((host(Ya) - host(Yb)) * wY) ** 2)) <= 1e-3
