"""Pins for the oracle's derivatives (definition step 10).

The complex-step Jacobian, JVP and ln A gradient are checked against central finite
differences of the forward oracle, against each other, against the closed form
d q_r / d ln A_r = q_r (a shift of ln A_r scales forward and reverse rates alike), and
against the derivatives of the conservation laws.
"""
import numpy as np
import pytest

import oracle
from paper_2409_06404_gb300 import synth
from conftest import nu_matrix


def _pts(m, n, seed):
    st = synth.states_uniform(m.K, n, seed=seed, T_lo=400.0, T_hi=2800.0, alpha=0.8)
    return st.T, st.p, st.Y


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
def test_jacobian_matches_central_differences(name):
    m = synth.mechanism(name)
    T, p, Y = _pts(m, 3, seed=81)
    J = oracle.jacobian(m, T, p, Y)
    w0, h0, ws, hs = oracle.rates(m, T, p, Y, scales=True)
    K = m.K
    for j in range(K + 1):
        step = 1e-6 * (T if j == 0 else np.maximum(Y[j - 1], 1e-3))
        Tp, Tm, Yp, Ym = T.copy(), T.copy(), Y.copy(), Y.copy()
        if j == 0:
            Tp += step
            Tm -= step
        else:
            Yp[j - 1] += step
            Ym[j - 1] -= step
        wp, hp = oracle.rates(m, Tp, p, Yp)
        wm, hm = oracle.rates(m, Tm, p, Ym)
        fd_w = (wp - wm) / (2 * step)
        fd_h = (hp - hm) / (2 * step)
        # scale-aware: the error of a central difference is relative to the rate magnitudes
        tol_w = 1e-6 * ws / step
        tol_h = 1e-6 * hs / step
        assert np.all(np.abs(J[:, :K, j].T - fd_w) <= tol_w), j
        assert np.all(np.abs(J[:, K, j] - fd_h) <= tol_h), j


def test_jvp_equals_jacobian_times_v(mech53):
    T, p, Y = _pts(mech53, 4, seed=82)
    J = oracle.jacobian(mech53, T, p, Y)
    rng = np.random.default_rng(1)
    vT = rng.standard_normal(4)
    vY = rng.standard_normal((mech53.K, 4))
    dw, dh, dws, dhs = oracle.jvp(mech53, T, p, Y, vT, vY, scales=True)
    v = np.vstack([vT[None], vY])                      # [K+1, n]
    Jv = np.einsum("nij,jn->in", J, v)
    # cancellation-aware: relative to the magnitudes of the per-reaction derivative terms
    scale = np.einsum("nij,jn->in", np.abs(J), np.abs(v))
    assert np.all(np.abs(Jv[:-1] - dw) <= 1e-13 * (dws + scale[:-1]))
    assert np.all(np.abs(Jv[-1] - dh) <= 1e-13 * (dhs + scale[-1]))
    assert np.all(dws >= np.abs(dw) * (1 - 1e-12))


def test_jacobian_respects_conservation(mech53):
    T, p, Y = _pts(mech53, 3, seed=83)
    J = oracle.jacobian(mech53, T, p, Y)
    K = mech53.K
    absJ = np.abs(J[:, :K, :])
    assert np.all(np.abs(np.einsum("k,nkj->nj", mech53.W, J[:, :K, :])) <=
                  1e-11 * np.einsum("k,nkj->nj", mech53.W, absJ))
    for e in range(mech53.atoms.shape[1]):
        a = mech53.atoms[:, e].astype(float)
        assert np.all(np.abs(np.einsum("k,nkj->nj", a, J[:, :K, :])) <=
                      1e-11 * np.einsum("k,nkj->nj", a, absJ) + 1e-300)


@pytest.mark.parametrize("name", ["h2_9sp_21rx", "ch4_53sp_325rx"])
def test_grad_lnA_closed_form_and_fd(name):
    m = synth.mechanism(name)
    n = 16
    T, p, Y = _pts(m, n, seed=84)
    rng = np.random.default_rng(2)
    wbar = rng.standard_normal((m.K, n))
    hbar = rng.standard_normal(n) * 1e-6
    g = oracle.grad_lnA(m, T, p, Y, wbar, hbar)
    # closed form: dq_r/dlnA_r = q_r; dL/dq_r = sum_k nu_kr (wbar_k - hbar h_k)
    fwd, rev = oracle.rates_of_progress(m, T, p, Y)
    q = fwd - rev
    hk = oracle.thermo(m, T, p, Y)["h_k"]
    nu = nu_matrix(m)
    qbar = nu.T @ (wbar - hbar[None, :] * hk)
    g_cf = np.sum(qbar * q, axis=1)
    scale = np.sum(np.abs(qbar) * (fwd + rev), axis=1)
    assert np.all(np.abs(g - g_cf) <= 1e-12 * scale)
    # central differences in ln A for a few reactions; the rounding floor of a difference of
    # omega values is eps * omega_scale / step, weighted by |wbar|
    _, _, ws, hs = oracle.rates(m, T, p, Y, scales=True)
    step = 1e-4
    floor = 1e-15 * (np.sum(np.abs(wbar) * ws) + np.sum(np.abs(hbar) * hs)) / step
    for r in (0, m.R // 2, m.R - 1):
        d = np.zeros(m.R)
        d[r] = step
        wp, hp = oracle.rates(m, T, p, Y, dlnA=d)
        wm, hm = oracle.rates(m, T, p, Y, dlnA=-d)
        fd = (np.sum(wbar * (wp - wm)) + np.sum(hbar * (hp - hm))) / (2 * step)
        assert abs(fd - g[r]) <= 1e-8 * scale[r] + floor
