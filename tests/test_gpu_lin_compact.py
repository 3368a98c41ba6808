"""Per-reaction (compact) stored linearization (nk_rates_linearize_compact + the products from it)
against the oracle's complex-step JVP (1e-10, cancellation-aware), against the recomputing JVP
kernel, and its forward output against the oracle's rates."""
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


def test_compact_is_smaller_than_per_entry(cuda):
    m = gpu_mechanism("ch4_53sp_325rx")
    mech = synth.mechanism("ch4_53sp_325rx")
    R_el = int(np.sum(mech.rtype == 0))
    # A, forward and reverse terms per reaction, L per third-body/Troe reaction, S1, and
    # h_k/RT, 1/Y_k, C_k per species
    assert nk.linearization_slots_compact(m) == 3 * mech.R + (mech.R - R_el) + 1 + 3 * mech.K
    assert nk.linearization_slots_compact(m) < 0.6 * nk.linearization_slots(m)


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 4096 + 77), ("h2_9sp_21rx", 2000), ("big_120sp_700rx", 600)])
def test_compact_jvp_vs_complex_step(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=5)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize_compact(m, Tt, pt, Yt)
    assert lin.shape[0] == nk.linearization_slots_compact(m)
    for d in range(3):                                   # several directions, one linearization
        vT = synth.normal(n, 4300 + 2 * d)
        vY = synth.normal((mech.K, n), 4301 + 2 * d)
        vTt, vYt = to_dev(vT, vY)
        dw, dh = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin, vTt, vYt)
        dw_o, dh_o, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, scales=True)
        assert scaled_err(host(dw), dw_o, dws) <= TOL
        assert scaled_err(host(dh), dh_o, dhs) <= TOL
        dw2, dh2 = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt)
        assert scaled_err(host(dw), host(dw2), dws) <= TOL and scaled_err(host(dh), host(dh2), dhs) <= TOL


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 1000 + 13), ("big_120sp_700rx", 300)])
def test_compact_primal_outputs(cuda, name, n):
    """The linearization pass's omega and heat release against the oracle (1e-10), and the same
    stored data with and without them."""
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=6)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin, w, h = nk.rates_linearize_compact(m, Tt, pt, Yt, primal=True)
    w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, scales=True)
    assert scaled_err(host(w), w_o, ws) <= TOL
    assert scaled_err(host(h), h_o, hs) <= TOL
    # the pass without the outputs stores the same data; only S1, a sum over the reactions that
    # each kernel variant splits over its own number of warps per point, may round differently
    lin2 = nk.rates_linearize_compact(m, Tt, pt, Yt)
    R_el = int(np.sum(mech.rtype == 0))
    s1 = 3 * mech.R + (mech.R - R_el)
    keep = torch.ones(lin.shape[0], dtype=torch.bool, device="cuda")
    keep[s1] = False
    assert torch.equal(lin[keep, :n], lin2[keep, :n])
    vT, vY = synth.normal(n, 80), synth.normal((mech.K, n), 81)
    vTt, vYt = to_dev(vT, vY)
    _, _, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, scales=True)
    dw1, dh1 = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin, vTt, vYt)
    dw2, dh2 = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin2, vTt, vYt)
    assert torch.equal(dw1, dw2) and scaled_err(host(dh1), host(dh2), dhs) <= 1e-13
    # with an ln A shift, against the oracle at the same shift, and the JVP from that linearization
    dlnA = synth.normal(mech.R, 77) * 0.3
    dlnAt = torch.from_numpy(dlnA).cuda()
    lin3, w3, h3 = nk.rates_linearize_compact(m, Tt, pt, Yt, dlnA=dlnAt, primal=True)
    w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, dlnA=dlnA, scales=True)
    assert scaled_err(host(w3), w_o, ws) <= TOL and scaled_err(host(h3), h_o, hs) <= TOL
    vT, vY = synth.normal(n, 78), synth.normal((mech.K, n), 79)
    vTt, vYt = to_dev(vT, vY)
    dw, dh = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin3, vTt, vYt)
    dw_o, dh_o, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, dlnA=dlnA, scales=True)
    assert scaled_err(host(dw), dw_o, dws) <= TOL and scaled_err(host(dh), dh_o, dhs) <= TOL


def test_compact_edge_states(cuda):
    """Zero, tiny, subnormal and negative mass fractions, pure and nearly pure mixtures, T at the
    range ends: sides with a mass fraction below 2^-200 take the exclusive-product form."""
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
    Y[5:20, 9] = 1e-100                                  # tiny, not zero
    Y[21:30, 10] = 5e-320                                # subnormal
    Y[31:40, 10] = 1e-59                                 # just above the tiny threshold (2^-200)
    Y[4, 11] = 0.0                                       # one absent species
    T = T.copy()
    T[4], T[5], T[6] = 300.0, 3500.0, 1000.0
    p = p.copy()
    p[8] = 0.05 * 101325.0
    vT = synth.normal(64, 9)
    vY = synth.normal((mech.K, 64), 10)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    lin = nk.rates_linearize_compact(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin, vTt, vYt)
    dw_o, dh_o, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, scales=True)
    # the complex step's h^2 remainder at pure mixtures (see test_gpu_lin.py)
    dws = dws + 1e-60 * dws.max(axis=0, keepdims=True)
    assert scaled_err(host(dw), dw_o, dws) <= TOL
    assert scaled_err(host(dh), dh_o, dhs) <= TOL
    dw2, dh2 = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt)
    assert scaled_err(host(dw), host(dw2), dws) <= TOL


def test_compact_nonfinite_point_stays_local(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y = _flame(mech, 96, seed=11)
    Y = Y.copy()
    Y[2, 40] = np.nan
    vT, vY = synth.normal(96, 12), synth.normal((mech.K, 96), 13)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    lin = nk.rates_linearize_compact(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin, vTt, vYt)
    ok = np.ones(96, bool)
    ok[40] = False
    assert np.all(np.isfinite(host(dw)[:, ok])) and np.all(np.isfinite(host(dh)[ok]))
    assert not np.all(np.isfinite(host(dh)[40:41]))
    dw2, dh2 = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt)
    _, _, dws, dhs = oracle.jvp(mech, T[ok], p[ok], np.ascontiguousarray(Y[:, ok]), vT[ok],
                                np.ascontiguousarray(vY[:, ok]), scales=True)
    assert scaled_err(host(dw)[:, ok], host(dw2)[:, ok], dws) <= TOL


def test_compact_strided_and_padded(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y = _flame(mech, 300, seed=8)
    vT, vY = synth.normal(300, 3), synth.normal((mech.K, 300), 4)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    lin = nk.rates_linearize_compact(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin, vTt, vYt)
    # a chunk of a wider field, its linearization in a wider buffer: same bits
    a, b = 37, 200
    big = torch.full((nk.linearization_slots_compact(m), 500), float("nan"), dtype=torch.float64, device="cuda")
    lin2 = nk.rates_linearize_compact(m, Tt[a:b], pt[a:b], Yt[:, a:b], lin=big)
    dw2, dh2 = nk.rates_jvp_linearized_compact(m, Tt[a:b], pt[a:b], Yt[:, a:b], lin2, vTt[a:b], vYt[:, a:b])
    assert torch.equal(dw2, dw[:, a:b]) and torch.equal(dh2, dh[a:b])
    one = nk.rates_linearize_compact(m, Tt[5:6], pt[5:6], Yt[:, 5:6])
    dw3, dh3 = nk.rates_jvp_linearized_compact(m, Tt[5:6], pt[5:6], Yt[:, 5:6], one, vTt[5:6], vYt[:, 5:6])
    assert torch.equal(dw3, dw[:, 5:6]) and torch.equal(dh3, dh[5:6])
    # n = 0 enqueues nothing and succeeds
    e = nk.rates_linearize_compact(m, Tt[:0], pt[:0], Yt[:, :0])
    assert e.shape[0] == nk.linearization_slots_compact(m)


def test_compact_argument_errors(cuda):
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    T, p, Y = _flame(mech, 40, seed=2)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize_compact(m, Tt, pt, Yt)
    L = nk.lib()
    w = torch.empty((mech.K, 40), dtype=torch.float64, device="cuda")
    st = L.nk_rates_linearize_compact(m.handle, 40, 40, nk._ptr(Tt), nk._ptr(pt), nk._ptr(Yt), None,
                                      nk._ptr(lin), lin.stride(0), nk._ptr(w), None, None)
    assert st == 1 and b"both" in L.nk_last_error()
    st = L.nk_rates_linearize_compact(m.handle, 40, 40, nk._ptr(Tt), nk._ptr(pt), nk._ptr(Yt), None,
                                      nk._ptr(lin), 39, None, None, None)
    assert st == 1
    with pytest.raises(ValueError):
        nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, lin[:-1], Tt, Yt)


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 2000 + 33), ("h2_9sp_21rx", 1000), ("big_120sp_700rx", 300)])
def test_compact_sources_jvp(cuda, name, n):
    """nk_rhs_jvp_linearized_compact against the oracle's complex-step JVP of the sources and
    against the recomputing nk_rhs_jvp."""
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=8)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize_compact(m, Tt, pt, Yt)
    fT, fY = nk.rhs_eval(m, Tt, pt, Yt)
    for d in range(2):
        vT = synth.normal(n, 4400 + 2 * d) * 30.0
        vY = synth.normal((mech.K, n), 4401 + 2 * d) * (Y + 1e-12)
        vTt, vYt = to_dev(vT, vY)
        dfT, dfY = nk.rhs_jvp_linearized_compact(m, Tt, pt, Yt, lin, fT, fY, vTt, vYt)
        dT_o, dY_o, sT, sY = oracle.rhs_jvp(mech, T, p, Y, vT, vY, scales=True)
        assert scaled_err(host(dfT), dT_o, sT) <= TOL
        assert scaled_err(host(dfY), dY_o, sY) <= TOL
        dfT2, dfY2 = nk.rhs_jvp(m, Tt, pt, Yt, vTt, vYt)
        assert scaled_err(host(dfT), host(dfT2), sT) <= TOL and scaled_err(host(dfY), host(dfY2), sY) <= TOL


def test_compact_full_size_sampled(cuda):
    """2,097,152 points, the benchmark's launch configuration: sampled against the oracle, and
    every point against the recomputing JVP (the same 1e-10 bar on the oracle's scales is not
    available for all points; the two kernels' difference is bounded by 1e-10 of the larger of
    their results' magnitudes per species row)."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    n = st.n
    T, p, Y = to_dev(st.T, st.p, st.Y)
    lin, w, h = nk.rates_linearize_compact(m, T, p, Y, primal=True)
    g = torch.Generator(device="cuda").manual_seed(4353)
    vT = torch.randn(n, generator=g, dtype=torch.float64, device="cuda")
    vY = torch.randn((mech.K, n), generator=g, dtype=torch.float64, device="cuda")
    dw, dh = nk.rates_jvp_linearized_compact(m, T, p, Y, lin, vT, vY)
    rng = np.random.default_rng(12)
    idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 800, replace=False)]))
    sub = torch.from_numpy(idx).cuda()
    Ts, ps, Ys = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    dw_o, dh_o, dws, dhs = oracle.jvp(mech, Ts, ps, Ys, host(vT[sub]), np.ascontiguousarray(host(vY[:, sub])),
                                      scales=True)
    assert scaled_err(host(dw[:, sub]), dw_o, dws) <= TOL
    assert scaled_err(host(dh[sub]), dh_o, dhs) <= TOL
    w_o, h_o, ws, hs = oracle.rates(mech, Ts, ps, Ys, scales=True)
    assert scaled_err(host(w[:, sub]), w_o, ws) <= TOL
    assert scaled_err(host(h[sub]), h_o, hs) <= TOL
    assert torch.isfinite(dh).all() and torch.isfinite(dw).all()
    del lin
