"""Implicit-stage chemistry sources (nk_rhs_eval) and their exact JVP (nk_rhs_jvp) against the
oracle: 1e-10 cancellation-aware for the FP64 forms and the JVP, 1e-5 for the mixed form."""
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


def _flame(mech, n, seed=3):
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 4096 + 77), ("h2_9sp_21rx", 2000), ("big_120sp_700rx", 700)])
@pytest.mark.parametrize("form,tol", [("fp64", TOL64), ("fp64_native", TOL64), ("mixed", TOLMIX)])
def test_rhs_eval(cuda, name, n, form, tol):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n)
    fT, fY = nk.rhs_eval(m, *to_dev(T, p, Y), precision=form)
    fT_o, fY_o, sT, sY = oracle.rhs(mech, T, p, Y, scales=True)
    assert scaled_err(host(fT), fT_o, sT) <= tol
    assert scaled_err(host(fY), fY_o, sY) <= tol
    # mass conservation of the device result itself
    assert np.all(np.abs(host(fY).sum(0)) <= 10 * tol * sY.sum(0))


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 4096 + 77), ("h2_9sp_21rx", 2000), ("big_120sp_700rx", 600)])
def test_rhs_jvp_vs_complex_step(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=4)
    vT = synth.normal(n, 4153)
    vY = synth.normal((mech.K, n), 4154)
    dfT, dfY, fT, fY = nk.rhs_jvp(m, *to_dev(T, p, Y, vT, vY), primal=True)
    dfT_o, dfY_o, dsT, dsY = oracle.rhs_jvp(mech, T, p, Y, vT, vY, scales=True)
    assert scaled_err(host(dfT), dfT_o, dsT) <= TOL64
    assert scaled_err(host(dfY), dfY_o, dsY) <= TOL64
    fT_o, fY_o, sT, sY = oracle.rhs(mech, T, p, Y, scales=True)
    assert scaled_err(host(fT), fT_o, sT) <= TOL64
    assert scaled_err(host(fY), fY_o, sY) <= TOL64
    assert np.all(np.abs(host(dfY).sum(0)) <= 10 * TOL64 * dsY.sum(0))
    # without the primal sources (a kernel variant that keeps no omega_k rows)
    dfT2, dfY2 = nk.rhs_jvp(m, *to_dev(T, p, Y, vT, vY))
    assert scaled_err(host(dfT2), dfT_o, dsT) <= TOL64
    assert scaled_err(host(dfY2), dfY_o, dsY) <= TOL64


def test_rhs_small_and_strided(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y = _flame(mech, 300, seed=6)
    vT, vY = synth.normal(300, 1), synth.normal((mech.K, 300), 2)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    fT, fY = nk.rhs_eval(m, Tt, pt, Yt)
    dfT, dfY = nk.rhs_jvp(m, Tt, pt, Yt, vTt, vYt)
    # n = 1 and a strided chunk of a wider field give the same bits as the contiguous run
    for a, b in ((0, 1), (37, 200)):
        gT, gY = nk.rhs_eval(m, Tt[a:b], pt[a:b], Yt[:, a:b])
        assert torch.equal(gT, fT[a:b]) and torch.equal(gY, fY[:, a:b])
        hT, hY = nk.rhs_jvp(m, Tt[a:b], pt[a:b], Yt[:, a:b], vTt[a:b], vYt[:, a:b])
        assert torch.equal(hT, dfT[a:b]) and torch.equal(hY, dfY[:, a:b])


def test_rhs_full_size_sampled(cuda):
    """The 2,097,152-point flame field: sources and their JVP on 1,000 sampled points."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    n = st.n
    T, p, Y = to_dev(st.T, st.p, st.Y)
    g = torch.Generator(device="cuda").manual_seed(4253)
    vT = torch.randn(n, generator=g, dtype=torch.float64, device="cuda")
    vY = torch.randn((mech.K, n), generator=g, dtype=torch.float64, device="cuda")
    fT, fY = nk.rhs_eval(m, T, p, Y)
    dfT, dfY = nk.rhs_jvp(m, T, p, Y, vT, vY)
    rng = np.random.default_rng(11)
    idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 1000, replace=False)]))
    Ts, ps, Ys = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    fT_o, fY_o, sT, sY = oracle.rhs(mech, Ts, ps, Ys, scales=True)
    assert scaled_err(host(fT)[idx], fT_o, sT) <= TOL64
    assert scaled_err(host(fY)[:, idx], fY_o, sY) <= TOL64
    sub = torch.from_numpy(idx).cuda()
    dfT_o, dfY_o, dsT, dsY = oracle.rhs_jvp(mech, Ts, ps, Ys, host(vT[sub]), np.ascontiguousarray(host(vY[:, sub])),
                                            scales=True)
    assert scaled_err(host(dfT[sub]), dfT_o, dsT) <= TOL64
    assert scaled_err(host(dfY[:, sub]), dfY_o, dsY) <= TOL64
    assert torch.isfinite(fT).all() and torch.isfinite(dfT).all()
