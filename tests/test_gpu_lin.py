"""Stored linearization (nk_rates_linearize + nk_rates_jvp_linearized) against the oracle's
complex-step JVP (1e-10, cancellation-aware) and against the recomputing JVP kernel."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, scaled_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _flame(mech, n, seed=3):
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 4096 + 77), ("h2_9sp_21rx", 2000), ("big_120sp_700rx", 600)])
def test_linearized_jvp_vs_complex_step(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=5)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize(m, Tt, pt, Yt)
    assert lin.shape[0] == nk.linearization_slots(m)
    for d in range(3):                                   # several directions, one linearization
        vT = synth.normal(n, 4300 + 2 * d)
        vY = synth.normal((mech.K, n), 4301 + 2 * d)
        vTt, vYt = to_dev(vT, vY)
        dw, dh = nk.rates_jvp_linearized(m, Tt, pt, Yt, lin, vTt, vYt)
        dw_o, dh_o, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, scales=True)
        assert scaled_err(host(dw), dw_o, dws) <= TOL
        assert scaled_err(host(dh), dh_o, dhs) <= TOL
        dw2, dh2 = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt)
        assert scaled_err(host(dw), host(dw2), dws) <= TOL and scaled_err(host(dh), host(dh2), dhs) <= TOL


def test_linearized_jvp_edge_states(cuda):
    """Zero and negative mass fractions, nearly pure mixtures, T at the range ends: the stored
    concentration derivatives are exclusive products, exact at C = 0 (the recomputing JVP's
    dual products likewise)."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y = _flame(mech, 64, seed=7)
    Y = Y.copy()
    Y[:, 0] = 0.0
    Y[3, 0] = 1.0                                        # pure species
    Y[5:20, 1] = 0.0                                     # absent species
    Y[7, 2] = -1e-3                                      # a negative Y
    Y[:, 3] = 1e-12
    Y[11, 3] = 1.0 - 52e-12                              # nearly pure
    T = T.copy()
    T[4], T[5], T[6] = 300.0, 3500.0, 1000.0
    p = p.copy()
    p[8] = 0.05 * 101325.0
    vT = synth.normal(64, 9)
    vY = synth.normal((mech.K, 64), 10)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    lin = nk.rates_linearize(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized(m, Tt, pt, Yt, lin, vTt, vYt)
    dw_o, dh_o, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, scales=True)
    # Entries whose exact derivative vanishes at a pure mixture keep the complex step's h^2
    # remainder (~1e-119 here, with an equal scale); a floor of 1e-60 of the point's largest
    # derivative scale admits that remainder and nothing a double could resolve.
    dws = dws + 1e-60 * dws.max(axis=0, keepdims=True)
    assert scaled_err(host(dw), dw_o, dws) <= TOL
    assert scaled_err(host(dh), dh_o, dhs) <= TOL
    # the recomputing JVP at the same states
    dw2, dh2 = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt)
    assert scaled_err(host(dw2), dw_o, dws) <= TOL
    assert scaled_err(host(dh2), dh_o, dhs) <= TOL


def test_linearized_strided_and_padded(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y = _flame(mech, 300, seed=8)
    vT, vY = synth.normal(300, 3), synth.normal((mech.K, 300), 4)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    lin = nk.rates_linearize(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized(m, Tt, pt, Yt, lin, vTt, vYt)
    # a chunk of a wider field, its linearization in a wider buffer: same bits
    a, b = 37, 200
    big = torch.full((nk.linearization_slots(m), 500), float("nan"), dtype=torch.float64, device="cuda")
    lin2 = nk.rates_linearize(m, Tt[a:b], pt[a:b], Yt[:, a:b], lin=big)
    dw2, dh2 = nk.rates_jvp_linearized(m, Tt[a:b], pt[a:b], Yt[:, a:b], lin2, vTt[a:b], vYt[:, a:b])
    assert torch.equal(dw2, dw[:, a:b]) and torch.equal(dh2, dh[a:b])
    one = nk.rates_linearize(m, Tt[5:6], pt[5:6], Yt[:, 5:6])
    dw3, dh3 = nk.rates_jvp_linearized(m, Tt[5:6], pt[5:6], Yt[:, 5:6], one, vTt[5:6], vYt[:, 5:6])
    assert torch.equal(dw3, dw[:, 5:6]) and torch.equal(dh3, dh[5:6])


def test_linearized_full_size_sampled(cuda):
    """2,097,152 points (the stored data are ~31 GB at 53 species): sampled against the oracle."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    n = st.n
    T, p, Y = to_dev(st.T, st.p, st.Y)
    lin = nk.rates_linearize(m, T, p, Y)
    g = torch.Generator(device="cuda").manual_seed(4353)
    vT = torch.randn(n, generator=g, dtype=torch.float64, device="cuda")
    vY = torch.randn((mech.K, n), generator=g, dtype=torch.float64, device="cuda")
    dw, dh = nk.rates_jvp_linearized(m, T, p, Y, lin, vT, vY)
    rng = np.random.default_rng(12)
    idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 800, replace=False)]))
    sub = torch.from_numpy(idx).cuda()
    dw_o, dh_o, dws, dhs = oracle.jvp(mech, st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx]),
                                      host(vT[sub]), np.ascontiguousarray(host(vY[:, sub])), scales=True)
    assert scaled_err(host(dw[:, sub]), dw_o, dws) <= TOL
    assert scaled_err(host(dh[sub]), dh_o, dhs) <= TOL
    assert torch.isfinite(dh).all()
    del lin


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 2000 + 33), ("h2_9sp_21rx", 1000), ("big_120sp_700rx", 300)])
def test_sources_jvp_from_linearization(cuda, name, n):
    """nk_rhs_jvp_linearized against the oracle's complex-step JVP of the sources (1e-10 of the
    derivative magnitudes) and against the recomputing nk_rhs_jvp."""
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=8)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize(m, Tt, pt, Yt)
    fT, fY = nk.rhs_eval(m, Tt, pt, Yt)
    for d in range(2):
        vT = synth.normal(n, 4400 + 2 * d) * 30.0
        vY = synth.normal((mech.K, n), 4401 + 2 * d) * (Y + 1e-12)
        vTt, vYt = to_dev(vT, vY)
        dfT, dfY = nk.rhs_jvp_linearized(m, Tt, pt, Yt, lin, fT, fY, vTt, vYt)
        dT_o, dY_o, sT, sY = oracle.rhs_jvp(mech, T, p, Y, vT, vY, scales=True)
        assert scaled_err(host(dfT), dT_o, sT) <= TOL
        assert scaled_err(host(dfY), dY_o, sY) <= TOL
        dfT2, dfY2 = nk.rhs_jvp(m, Tt, pt, Yt, vTt, vYt)
        assert scaled_err(host(dfT), host(dfT2), sT) <= TOL and scaled_err(host(dfY), host(dfY2), sY) <= TOL
