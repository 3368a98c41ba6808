"""Hand-written JVP / VJP kernels vs the oracle's complex-step derivatives.

Tolerance 1e-10, cancellation-aware: relative to sum_r |nu_kr| (|d fwd_r| + |d rev_r|)
along the direction (JVP) or, per Jacobian entry, to the same magnitudes weighted by the
cotangent (VJP).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, scaled_err, nu_matrix

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _flame(mech, n, seed=3):
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 4096), ("h2_9sp_21rx", 2000), ("big_120sp_700rx", 600)])
def test_jvp_vs_complex_step(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n)
    vT = synth.normal(n, 4053)
    vY = synth.normal((mech.K, n), 4054)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    dw, dh, w, h = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt, primal=True)
    dw_o, dh_o, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, scales=True)
    assert scaled_err(host(dw), dw_o, dws) <= TOL
    assert scaled_err(host(dh), dh_o, dhs) <= TOL
    w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, scales=True)
    assert scaled_err(host(w), w_o, ws) <= TOL and scaled_err(host(h), h_o, hs) <= TOL


def test_vjp_vs_dense_jacobian(cuda):
    """53 species: (gT, gY) = J^T (bar_omega, bar_hrr) against the oracle's dense 54 x 54
    complex-step Jacobian at 512 points."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    n = 512
    T, p, Y = _flame(mech, n, seed=5)
    wbar = synth.normal((mech.K, n), 3053)
    hbar = synth.normal(n, 3054) * 1e-5
    Tt, pt, Yt, wt, ht = to_dev(T, p, Y, wbar, hbar)
    gT, gY, g = nk.rates_vjp(m, Tt, pt, Yt, wt, ht)
    J, Js = oracle.jacobian(mech, T, p, Y, scales=True)
    u = np.vstack([wbar, hbar[None, :]])                   # [K+1, n] cotangent over outputs
    JTu = np.einsum("nij,in->jn", J, u)                   # [K+1 inputs, n]
    scale = np.einsum("nij,in->jn", Js, np.abs(u))
    assert scaled_err(host(gT), JTu[0], scale[0]) <= TOL
    assert scaled_err(host(gY), JTu[1:], scale[1:]) <= TOL


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "big_120sp_700rx"])
def test_vjp_vs_dense_jacobian_other_mechanisms(cuda, name):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    n = 128
    T, p, Y = _flame(mech, n, seed=6)
    wbar = synth.normal((mech.K, n), 1)
    hbar = synth.normal(n, 2) * 1e-5
    Tt, pt, Yt, wt, ht = to_dev(T, p, Y, wbar, hbar)
    gT, gY, g = nk.rates_vjp(m, Tt, pt, Yt, wt, ht)
    J, Js = oracle.jacobian(mech, T, p, Y, scales=True)
    u = np.vstack([wbar, hbar[None, :]])
    JTu = np.einsum("nij,in->jn", J, u)
    scale = np.einsum("nij,in->jn", Js, np.abs(u))
    assert scaled_err(host(gT), JTu[0], scale[0]) <= TOL
    assert scaled_err(host(gY), JTu[1:], scale[1:]) <= TOL


def test_grad_lnA_vs_oracle_and_deterministic(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    n = 4096
    T, p, Y = _flame(mech, n, seed=8)
    wbar = synth.normal((mech.K, n), 3053)
    Tt, pt, Yt, wt = to_dev(T, p, Y, wbar)
    _, _, g1 = nk.rates_vjp(m, Tt, pt, Yt, wt)
    _, _, g2 = nk.rates_vjp(m, Tt, pt, Yt, wt)
    assert torch.equal(g1, g2)                              # fixed-order reduction
    g_o = oracle.grad_lnA(mech, T, p, Y, wbar)
    fwd, rev = oracle.rates_of_progress(mech, T, p, Y)
    qbar = nu_matrix(mech).T @ wbar
    scale = np.sum(np.abs(qbar) * (fwd + rev), axis=1)
    assert scaled_err(host(g1), g_o, scale) <= TOL


def test_adjoint_identity_full_size_sampled(cuda):
    """<u, J v> = <J^T u, v> point by point on the 2,097,152-point flame workload."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    n = st.n
    T, p, Y = to_dev(st.T, st.p, st.Y)
    g = torch.Generator(device="cuda").manual_seed(4053)
    vT = torch.randn(n, generator=g, dtype=torch.float64, device="cuda")
    vY = torch.randn((mech.K, n), generator=g, dtype=torch.float64, device="cuda")
    uw = torch.randn((mech.K, n), generator=g, dtype=torch.float64, device="cuda")
    uh = torch.randn(n, generator=g, dtype=torch.float64, device="cuda") * 1e-5
    dw, dh = nk.rates_jvp(m, T, p, Y, vT, vY)
    gT, gY, gl = nk.rates_vjp(m, T, p, Y, uw, uh)
    lhs = host((uw * dw).sum(0) + uh * dh)
    rhs = host(gT * vT + (gY * vY).sum(0))
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(n, 400, replace=False))
    _, _, dws, dhs = oracle.jvp(mech, st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx]),
                                host(vT)[idx], np.ascontiguousarray(host(vY)[:, idx]), scales=True)
    scale = np.sum(np.abs(host(uw)[:, idx]) * dws, axis=0) + np.abs(host(uh)[idx]) * dhs
    assert scaled_err(lhs[idx], rhs[idx], scale) <= TOL
    assert np.all(np.isfinite(lhs)) and np.all(np.isfinite(rhs)) and torch.isfinite(gl).all()


def test_autograd_function(cuda):
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    n = 64
    T, p, Y = _flame(mech, n, seed=9)
    Tt, pt, Yt = to_dev(T, p, Y)
    Tt.requires_grad_(True)
    Yt.requires_grad_(True)
    dlnA = torch.zeros(mech.R, dtype=torch.float64, device="cuda", requires_grad=True)
    w, h = nk.rates(m, Tt, pt, Yt, dlnA)
    wbar = torch.from_numpy(synth.normal((mech.K, n), 5)).cuda()
    hbar = torch.from_numpy(synth.normal(n, 6)).cuda() * 1e-5
    loss = (w * wbar).sum() + (h * hbar).sum()
    loss.backward()
    gT, gY, gA = nk.rates_vjp(m, Tt.detach(), pt, Yt.detach(), wbar, hbar)
    assert torch.equal(Tt.grad, gT) and torch.equal(Yt.grad, gY) and torch.equal(dlnA.grad, gA)
    # forward mode through the hand-written JVP
    import torch.autograd.forward_ad as fwAD
    vT = torch.from_numpy(synth.normal(n, 7)).cuda()
    vY = torch.from_numpy(synth.normal((mech.K, n), 8)).cuda()
    with fwAD.dual_level():
        w2, h2 = nk.rates(m, fwAD.make_dual(Tt.detach(), vT), pt, fwAD.make_dual(Yt.detach(), vY))
        dw = fwAD.unpack_dual(w2).tangent
        dh = fwAD.unpack_dual(h2).tangent
    dw_ref, dh_ref = nk.rates_jvp(m, Tt.detach(), pt, Yt.detach(), vT, vY)
    assert torch.equal(dw, dw_ref) and torch.equal(dh, dh_ref)
