"""Diffusion fluxes (nk_diffusion_fluxes) against the oracle, 1e-10 relative to the magnitudes
behind each output: |a_k grad X_k| + Y_k sum_j |a_j grad X_j| for j_k (a_k = -rho (W_k/Wbar) D_k,
the uncorrected flux factor), sum_j |a_j grad X_j| / rho for V_c, sum_k c_p,k times the flux
scales for the enthalpy-flux factor."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, scaled_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _scales(mech, T, p, Y, D, G):
    th = oracle.thermo(mech, T, p, Y)
    a = -th["rho"][None, :] * (mech.W[:, None] / th["Wbar"][None, :]) * D
    u = np.abs(a[None] * G)                                   # [3, K, n]
    tot = u.sum(axis=1)                                       # [3, n]
    sj = u + Y[None] * tot[:, None, :]
    cpk = th["cp_k"] / mech.W[:, None]
    return sj, tot / th["rho"][None, :], (cpk[None] * sj).sum(axis=1)


def _inputs(mech, n, seed):
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    rng = np.random.default_rng(seed)
    D = np.exp(rng.uniform(np.log(5e-6), np.log(8e-5), (mech.K, n)))
    G = rng.standard_normal((3, mech.K, n)) * 50.0
    return T, p, Y, D, G


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 4096 + 77), ("h2_9sp_21rx", 1000), ("big_120sp_700rx", 500)])
def test_fluxes_vs_oracle(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y, D, G = _inputs(mech, n, 21)
    Y = Y.copy()
    Y[:, 0] = 0.0
    Y[1, 0] = 1.0                                             # a pure point: X_k = 0 elsewhere
    Y[2, 1] = 0.0
    Y[:, 1] /= Y[:, 1].sum()                                  # an absent species
    j, Vc, hf = nk.diffusion_fluxes(m, *to_dev(T, p, Y, D, G))
    j_o, Vc_o, hf_o = oracle.diffusion(mech, T, p, Y, D, G)
    sj, sv, sh = _scales(mech, T, p, Y, D, G)
    assert scaled_err(host(j), j_o, sj) <= TOL
    assert scaled_err(host(Vc), Vc_o, sv) <= TOL
    assert scaled_err(host(hf), hf_o, sh) <= TOL
    # the fluxes of each point sum to zero
    assert np.all(np.abs(host(j).sum(axis=1)) <= 1e-12 * sj.sum(axis=1))
    # optional outputs
    j2, none_v, none_h = nk.diffusion_fluxes(m, *to_dev(T, p, Y, D, G), want_vc=False, want_hf=False)
    assert none_v is None and none_h is None and torch.equal(j2, j)


def test_fluxes_with_transport_coefficients(cuda):
    """End to end: D_k from nk_transport_eval (FP64), then the fluxes, against the oracle's
    transport and diffusion."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y, _, G = _inputs(mech, 2000, 22)
    Tt, pt, Yt, Gt = to_dev(T, p, Y, G)
    _, _, Dt = nk.transport_eval(m, Tt, pt, Yt)
    j, Vc, hf = nk.diffusion_fluxes(m, Tt, pt, Yt, Dt, Gt)
    _, _, D_o = oracle.transport(mech, T, p, Y)
    j_o, Vc_o, hf_o = oracle.diffusion(mech, T, p, Y, D_o, G)
    sj, sv, sh = _scales(mech, T, p, Y, D_o, G)
    assert scaled_err(host(j), j_o, sj) <= TOL
    assert scaled_err(host(Vc), Vc_o, sv) <= TOL
    assert scaled_err(host(hf), hf_o, sh) <= TOL


def test_fluxes_full_size_sampled(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    n = st.n
    T, p, Y = to_dev(st.T, st.p, st.Y)
    _, _, D = nk.transport_eval(m, T, p, Y)
    g = torch.Generator(device="cuda").manual_seed(4453)
    G = torch.randn((3, mech.K, n), generator=g, dtype=torch.float64, device="cuda") * 50.0
    j, Vc, hf = nk.diffusion_fluxes(m, T, p, Y, D, G)
    rng = np.random.default_rng(13)
    idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 800, replace=False)]))
    sub = torch.from_numpy(idx).cuda()
    Ts, ps, Ys = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    Ds, Gs = np.ascontiguousarray(host(D[:, sub])), np.ascontiguousarray(host(G[:, :, sub]))
    j_o, Vc_o, hf_o = oracle.diffusion(mech, Ts, ps, Ys, Ds, Gs)
    sj, sv, sh = _scales(mech, Ts, ps, Ys, Ds, Gs)
    assert scaled_err(host(j[:, :, sub]), j_o, sj) <= TOL
    assert scaled_err(host(Vc[:, sub]), Vc_o, sv) <= TOL
    assert scaled_err(host(hf[:, sub]), hf_o, sh) <= TOL
