"""Negative mass fractions (the states a difference quotient or a transport step produces) in the
rates kernels: the concentration products enter through ln |C_k| with the concentrations' signs
beside them (a side's product is negative when an odd power of a negative concentration is in
it, [M] takes the signed C_j).  Checked against the oracle, whose products are plain powers, at
the FP64 and mixed bars, on perturbed flame states where many points hold a negative mass
fraction, and for independence of a point's result from the other points of its block."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, scaled_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOLMIX = 1e-5


def _perturbed(mech, n, seed, size=1e-6):
    """Flame states moved along a seeded N(0, 1) direction by about ten difference-quotient steps
    (the NITSOL step of a state of norm ~2000 is ~1e-7 per unit direction): the smallest mass
    fractions turn negative, in nearly every block of 32 points."""
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    v = synth.normal((mech.K, n), seed + 100)
    return T, p, Y + size * v


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 700 + 19), ("h2_9sp_21rx", 1000), ("big_120sp_700rx", 200)])
@pytest.mark.parametrize("form,tol", [("fp64", TOL64), ("mixed", TOLMIX)])
def test_perturbed_states(cuda, name, n, form, tol):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _perturbed(mech, n, seed=61)
    assert np.mean(np.any(Y < 0, axis=0)) > 0.05                      # many points hold one
    Tt, pt, Yt = to_dev(T, p, Y)
    w, h = nk.rates_eval(m, Tt, pt, Yt, precision=form)
    w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, scales=True)
    assert scaled_err(host(w), w_o, ws) <= tol
    assert scaled_err(host(h), h_o, hs) <= tol


@pytest.mark.parametrize("form,tol", [("fp64", TOL64), ("mixed", TOLMIX)])
def test_large_negative_fractions(cuda, form, tol):
    """Negative mass fractions far above rounding, on reactants, products and third-body
    species alike (each species of the 53 negative at some point, squared ones included), small
    enough that [M] and rho stay positive (the oracle's falloff needs ln [M])."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    K, n = mech.K, 3 * mech.K
    st = synth.states_flame(K, 27, seed=62)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.array(st.Y[:, idx])
    for j in range(n):
        Y[j % K, j] = -(10.0 ** -(4 + j % 5))                        # -1e-4 ... -1e-8
    Tt, pt, Yt = to_dev(T, p, Y)
    w, h = nk.rates_eval(m, Tt, pt, Yt, precision=form)
    w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, scales=True)
    assert scaled_err(host(w), w_o, ws) <= tol
    assert scaled_err(host(h), h_o, hs) <= tol


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_result_independent_of_block_neighbours(cuda, form):
    """A point without a negative mass fraction gets the same rates, to the last bits, whether or
    not another point of its block holds one (the two passes take the same steps for a positive
    concentration)."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    n = 4096
    st = synth.states_flame(mech.K, 27, seed=63)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    Yn = Y.copy()
    hit = np.arange(5, n, 37)                                          # one or two per block of 32
    Yn[3, hit] = -1e-6
    Tt, pt, Yt, Ynt = to_dev(T, p, Y, Yn)
    w, h = nk.rates_eval(m, Tt, pt, Yt, precision=form)
    wn, hn = nk.rates_eval(m, Tt, pt, Ynt, precision=form)
    keep = np.setdiff1d(np.arange(n), hit)
    w, h, wn, hn = host(w)[:, keep], host(h)[keep], host(wn)[:, keep], host(hn)[keep]
    _, _, ws, hs = oracle.rates(mech, T[keep[:64]], p[keep[:64]], Y[:, keep[:64]], scales=True)
    assert np.all(np.isfinite(wn)) and np.all(np.isfinite(hn))
    # the same arithmetic on the same operands (a compiler may still contract an operation
    # differently in the two passes' code: a few units of the last place of the scale)
    assert scaled_err(wn[:, :64], w[:, :64], ws) <= 1e-14
    assert scaled_err(hn[:64], h[:64], hs) <= 1e-14


def test_fd_quotient_matches_exact_jvp(cuda):
    """A forward difference of the FP64 rates along a direction, at the NITSOL step (which drives
    small mass fractions negative), agrees with the exact JVP to the difference quotient's
    truncation and rounding (checked in the scale of the exact JVP)."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    n = 2048
    st = synth.states_flame(mech.K, 27, seed=64)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    T, p, Y = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    vT = synth.normal(n, 6401)
    vY = synth.normal((mech.K, n), 6402)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    eps = np.finfo(np.float64).eps
    xnorm = torch.sqrt(Tt * Tt + torch.linalg.vector_norm(Yt, dim=0) ** 2)
    sig = torch.sqrt((1.0 + xnorm) * eps) / torch.sqrt(vTt * vTt + torch.linalg.vector_norm(vYt, dim=0) ** 2)
    Yp = Yt + sig * vYt
    assert float((Yp < 0).any(0).double().mean()) > 0.1
    w0, _ = nk.rates_eval(m, Tt, pt, Yt)
    w1, _ = nk.rates_eval(m, Tt + sig * vTt, pt, Yp)
    fd = (w1 - w0) / sig
    dw, _ = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt)
    rel = ((fd - dw).abs().amax(0) / dw.abs().amax(0)).cpu().numpy()
    assert np.median(rel) < 1e-4
