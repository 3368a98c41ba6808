"""CUDA path vs the CPU oracle, element by element: thermo, rates and transport, FP64 and mixed.

FP64 bar: 1e-10, cancellation-aware for omega and the heat release (relative to
sum_r |nu_kr| (|fwd_r| + |rev_r|) and sum_k |h_k| times that), relative for c_p, mu,
lambda, D_k.  Mixed bar: 1e-5 on the same norms.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import R_GAS, P_ATM, gpu_mechanism, to_dev, host, scaled_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOLMIX = 1e-5


def _rates_err(mech, m, T, p, Y, precision="fp64", dlnA=None):
    Tt, pt, Yt = to_dev(T, p, Y)
    dA = None if dlnA is None else to_dev(dlnA)[0]
    w, h = nk.rates_eval(m, Tt, pt, Yt, dlnA=dA, precision=precision)
    w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, dlnA=dlnA, scales=True)
    return scaled_err(host(w), w_o, ws), scaled_err(host(h), h_o, hs)


def _transport_err(mech, m, T, p, Y, precision="fp64"):
    Tt, pt, Yt = to_dev(T, p, Y)
    mu, lam, D = nk.transport_eval(m, Tt, pt, Yt, precision=precision)
    mu_o, lam_o, D_o = oracle.transport(mech, T, p, Y)
    return (scaled_err(host(mu), mu_o, np.abs(mu_o)), scaled_err(host(lam), lam_o, np.abs(lam_o)),
            scaled_err(host(D), D_o, np.abs(D_o)))


def _thermo_err(mech, m, T, p, Y):
    Tt, pt, Yt = to_dev(T, p, Y)
    out = nk.thermo_eval(m, Tt, pt, Yt)
    o = oracle.thermo(mech, T, p, Y)
    RT = R_GAS * T
    hscale = np.sum(np.abs(Y * o["h_k"]) / mech.W[:, None], axis=0)
    return {
        "cp_mix": scaled_err(host(out["cp_mix"]), o["cp_mix"], np.abs(o["cp_mix"])),
        "h_mix": scaled_err(host(out["h_mix"]), o["h_mix"], hscale),
        "Wbar": scaled_err(host(out["Wbar"]), o["Wbar"], np.abs(o["Wbar"])),
        "rho": scaled_err(host(out["rho"]), o["rho"], np.abs(o["rho"])),
        "cp_k": scaled_err(host(out["cp_k"]), o["cp_k"], np.abs(o["cp_k"])),
        "h_k": scaled_err(host(out["h_k"]), o["h_k"], np.maximum(np.abs(o["h_k"]), RT)),
        "g_k": scaled_err(host(out["g_k"]), o["g_k"], np.maximum(np.abs(o["g_k"]), RT)),
    }


FP64_FORMS = ["fp64", "fp64_native"]


@pytest.mark.parametrize("form", FP64_FORMS)
def test_h2_9sp_full_workload_fp64(cuda, form):
    """9 species / 21 reactions, 64 elements x 512 GLL points (all 32,768 points)."""
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    st = synth.workload_states("uniform_64el", mech.K)
    ew, eh = _rates_err(mech, m, st.T, st.p, st.Y, precision=form)
    assert ew <= TOL64 and eh <= TOL64, (ew, eh)
    et = _transport_err(mech, m, st.T, st.p, st.Y, precision=form)
    print(f"\n{form}: omega {ew:.1e} hrr {eh:.1e} mu/lambda/D {et[0]:.1e} {et[1]:.1e} {et[2]:.1e}")
    assert max(et) <= TOL64
    e = _thermo_err(mech, m, st.T, st.p, st.Y)
    assert max(e.values()) <= TOL64, e


@pytest.mark.parametrize("form", FP64_FORMS)
@pytest.mark.parametrize("n", [1, 31, 129, 4096 + 77])
def test_53sp_tiles_and_ragged_tail_fp64(cuda, n, form):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.states_flame(mech.K, 27, seed=99)          # 3^3 elements: every T regime
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    ew, eh = _rates_err(mech, m, T, p, Y, precision=form)
    assert ew <= TOL64 and eh <= TOL64, (ew, eh)
    assert max(_transport_err(mech, m, T, p, Y, precision=form)) <= TOL64
    assert max(_thermo_err(mech, m, T, p, Y).values()) <= TOL64


@pytest.mark.parametrize("form", FP64_FORMS)
def test_120sp_fp64(cuda, form):
    mech = synth.mechanism("big_120sp_700rx")
    m = gpu_mechanism("big_120sp_700rx")
    st = synth.states_uniform(mech.K, 2048 + 13, seed=120, T_lo=300, T_hi=3400, alpha=0.3)
    ew, eh = _rates_err(mech, m, st.T, st.p, st.Y, precision=form)
    assert ew <= TOL64 and eh <= TOL64, (ew, eh)
    assert max(_transport_err(mech, m, st.T, st.p, st.Y, precision=form)) <= TOL64


def test_lnA_shift(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.states_uniform(mech.K, 500, seed=5, alpha=0.3)
    dlnA = synth.normal(mech.R, 11) * 0.5
    ew, eh = _rates_err(mech, m, st.T, st.p, st.Y, dlnA=dlnA)
    assert ew <= TOL64 and eh <= TOL64


@pytest.mark.parametrize("form", FP64_FORMS)
def test_edge_states(cuda, form):
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    K = mech.K
    cols, Ts, ps = [], [], []
    for k in range(K):                                      # pure species
        y = np.zeros(K)
        y[k] = 1.0
        cols.append(y)
        Ts.append(1200.0)
        ps.append(P_ATM)
    y = np.full(K, 1.0 / K)
    for T in (300.0, 1000.0, np.nextafter(1000.0, 2000.0), 3500.0):   # range ends and T_mid
        cols.append(y)
        Ts.append(T)
        ps.append(P_ATM)
    for pr in (0.05, 20.0):                                 # far from 1 atm
        cols.append(y)
        Ts.append(1500.0)
        ps.append(pr * P_ATM)
    y = np.zeros(K)
    y[[1, 4, 6]] = (0.2, 0.5, 0.3)                          # most species absent
    cols.append(y)
    Ts.append(1800.0)
    ps.append(P_ATM)
    y = np.full(K, 0.12)
    y[2] = -0.02                                            # a negative mass fraction
    cols.append(y)
    Ts.append(1400.0)
    ps.append(P_ATM)
    y = np.full(K, 1e-12)
    y[0] = 1 - 8e-12                                        # nearly pure
    cols.append(y)
    Ts.append(900.0)
    ps.append(P_ATM)
    Y = np.stack(cols, axis=1)
    T = np.array(Ts)
    p = np.array(ps)
    ew, eh = _rates_err(mech, m, T, p, Y, precision=form)
    assert ew <= TOL64 and eh <= TOL64, (ew, eh)
    assert max(_transport_err(mech, m, T, p, Y, precision=form)) <= TOL64
    assert max(_thermo_err(mech, m, T, p, Y).values()) <= TOL64


def test_strided_chunk_matches_contiguous(cuda):
    """A column chunk of a larger field (ld > n, offset base) gives the same bits as a copy."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.states_uniform(mech.K, 3000, seed=6)
    T, p, Y = to_dev(st.T, st.p, st.Y)
    a, b = 1000, 2237
    Yc = Y[:, a:b]                                          # row stride 3000
    w1, h1 = nk.rates_eval(m, T[a:b], p[a:b], Yc)
    w2, h2 = nk.rates_eval(m, T[a:b].contiguous(), p[a:b].contiguous(), Yc.contiguous())
    assert w1.stride(0) == 3000
    assert torch.equal(w1, w2) and torch.equal(h1, h2)
    mu1, l1, D1 = nk.transport_eval(m, T[a:b], p[a:b], Yc)
    mu2, l2, D2 = nk.transport_eval(m, T[a:b].contiguous(), p[a:b].contiguous(), Yc.contiguous())
    assert torch.equal(mu1, mu2) and torch.equal(D1, D2)


def test_empty_input_is_a_no_op(cuda):
    m = gpu_mechanism("h2_9sp_21rx")
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    Y = torch.empty((m.K, 0), dtype=torch.float64, device="cuda")
    w, h = nk.rates_eval(m, z, z, Y)
    assert w.shape == (m.K, 0) and h.shape == (0,)
    mu, lam, D = nk.transport_eval(m, z, z, Y)
    gT, gY, g = nk.rates_vjp(m, z, z, Y, Y)
    torch.cuda.synchronize()
    assert torch.all(g == 0)


def test_argument_errors(cuda):
    m = gpu_mechanism("h2_9sp_21rx")
    L = nk.lib()
    T, p = to_dev(np.full(64, 1000.0), np.full(64, P_ATM))
    Y = torch.full((m.K, 64), 1.0 / m.K, dtype=torch.float64, device="cuda")
    w = torch.empty_like(Y)
    h = torch.empty_like(T)
    P = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)
    assert L.nk_rates_eval(m.handle, 64, 63, P(T), P(p), P(Y), None, P(w), P(h), 0, None) == 1   # ld < n
    assert L.nk_rates_eval(m.handle, -1, 64, P(T), P(p), P(Y), None, P(w), P(h), 0, None) == 1
    assert L.nk_rates_eval(m.handle, 32, 64, P(T, 4), P(p), P(Y), None, P(w), P(h), 0, None) == 2  # align
    assert L.nk_rates_eval(m.handle, 64, 64, P(T), P(p), P(Y), None, P(w), P(h), 7, None) == 1    # precision
    assert L.nk_rates_eval(m.handle, 64, 64, P(T), P(p), None, None, P(w), P(h), 0, None) == 1    # NULL Y
    with pytest.raises(nk.NkError):
        nk.rates_vjp_workspace(m, -5)


def test_nonfinite_inputs_stay_local(cuda):
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    st = synth.states_uniform(mech.K, 64, seed=9)
    T = st.T.copy()
    T[5] = np.nan
    T[9] = -100.0
    T[11] = 0.0
    Tt, pt, Yt = to_dev(T, st.p, st.Y)
    w, h = nk.rates_eval(m, Tt, pt, Yt)
    w, h = host(w), host(h)
    good = np.ones(64, bool)
    good[[5, 9, 11]] = False
    assert not np.isfinite(h[5])
    assert np.all(np.isfinite(w[:, good])) and np.all(np.isfinite(h[good]))
    w_o, h_o, ws, hs = oracle.rates(mech, st.T[good], st.p[good], st.Y[:, good], scales=True)
    assert scaled_err(w[:, good], w_o, ws) <= TOL64


def test_full_size_flame_workload_sampled(cuda):
    """53 species on 4,096 elements x 512 points (2,097,152 points) in the benchmark's launch
    configuration; the oracle checks 1,500 sampled points plus the first and last."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    T, p, Y = to_dev(st.T, st.p, st.Y)
    w, h = nk.rates_eval(m, T, p, Y)
    mu, lam, D = nk.transport_eval(m, T, p, Y)
    mu2, lam2, D2 = nk.transport_eval(m, T, p, Y, precision="fp64_native")
    # the two FP64 transport forms agree everywhere, not only on the sample
    assert scaled_err(host(mu), host(mu2), host(mu2)) <= TOL64
    assert scaled_err(host(lam), host(lam2), host(lam2)) <= TOL64
    assert scaled_err(host(D), host(D2), host(D2)) <= TOL64
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, st.n - 1], rng.choice(st.n, 1500, replace=False)]))
    Ys = np.ascontiguousarray(st.Y[:, idx])
    w_o, h_o, ws, hs = oracle.rates(mech, st.T[idx], st.p[idx], Ys, scales=True)
    assert scaled_err(host(w)[:, idx], w_o, ws) <= TOL64
    assert scaled_err(host(h)[idx], h_o, hs) <= TOL64
    mu_o, lam_o, D_o = oracle.transport(mech, st.T[idx], st.p[idx], Ys)
    assert scaled_err(host(mu)[idx], mu_o, mu_o) <= TOL64
    assert scaled_err(host(lam)[idx], lam_o, lam_o) <= TOL64
    assert scaled_err(host(D)[:, idx], D_o, D_o) <= TOL64
    assert np.all(np.isfinite(host(h))) and np.all(np.isfinite(host(mu)))


def test_full_size_all_points_cross_forms(cuda):
    """Every point of the 2,097,152-point field, between independent code paths (the oracle checks a
    sample above): the FP64 rates (logarithmic products in double-float pairs) against the
    all-double form (products in double, the library's double exp/log); the JVP (logarithmic
    tangents) against the per-entry stored linearization's product (exclusive products in double).
    Without the oracle's cancellation scales at every point, each point's differences are measured
    against its largest |omega_k| (|d omega_k|) and the heat release against sum_k |h_k omega_k|
    (sum_k |h_k d omega_k|); the flame-field states are far from equilibrium, where these are of the
    order of the scales."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    T, p, Y = to_dev(st.T, st.p, st.Y)
    hk = nk.thermo_eval(m, T, p, Y)["h_k"]
    w, h = nk.rates_eval(m, T, p, Y)
    w2, h2 = nk.rates_eval(m, T, p, Y, precision="fp64_native")
    sw = w2.abs().amax(0)
    assert float(((w - w2).abs().amax(0) / sw).max()) <= TOL64
    assert float(((h - h2).abs() / (hk * w2).abs().sum(0)).max()) <= TOL64
    del w, w2, h, h2
    g = torch.Generator(device="cuda").manual_seed(77)
    vT = torch.randn(st.n, generator=g, dtype=torch.float64, device="cuda")
    vY = torch.randn((mech.K, st.n), generator=g, dtype=torch.float64, device="cuda")
    dw, dh = nk.rates_jvp(m, T, p, Y, vT, vY)
    lin = nk.rates_linearize(m, T, p, Y)
    dw2, dh2 = nk.rates_jvp_linearized(m, T, p, Y, lin, vT, vY)
    del lin
    assert float(((dw - dw2).abs().amax(0) / dw2.abs().amax(0)).max()) <= TOL64
    assert float(((dh - dh2).abs() / (hk * dw2).abs().sum(0)).max()) <= TOL64
    assert torch.isfinite(dh).all()


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 4096), ("big_120sp_700rx", 2048), ("h2_9sp_21rx", 4096)])
def test_mixed_form_per_output_errors(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    st = synth.states_flame(mech.K, 27, seed=31)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    ew, eh = _rates_err(mech, m, T, p, Y, precision="mixed")
    emu, elam, eD = _transport_err(mech, m, T, p, Y, precision="mixed")
    print(f"\n{name} mixed: omega {ew:.2e}  hrr {eh:.2e}  mu {emu:.2e}  lambda {elam:.2e}  D {eD:.2e}")
    assert ew <= TOLMIX and eh <= TOLMIX
    assert emu <= TOLMIX and elam <= TOLMIX and eD <= TOLMIX
