"""The Troe falloff chain of the FP64 kernels runs in double-float pairs; a falloff centre F_cent
below the pairs' float range (every term of (1 - a) exp(-T/T3) + a exp(-T/T1) + exp(-T2/T) under
2^-100) takes a double path out of line.  These cases drive every Troe reaction of the
53-species mechanism there (T3 = T1 = 3.8 K: F_cent from ~1e-35 down to ~1e-298 over the flame
field, below the float range and above the double one's subnormals) and compare the rates, the
JVP, the VJP and the stored linearizations with the oracle at the FP64 bar."""
import numpy as np
import pytest

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, scaled_err

pytestmark = pytest.mark.gpu
TOL = 1e-10
T3T1 = 3.8


def _tiny_centre_mechanism():
    mech = synth.mechanism("ch4_53sp_325rx").copy()
    troe = np.nonzero(mech.rtype == 2)[0]
    assert troe.size > 0
    mech.troe[troe, 1] = T3T1          # T3 [K]
    mech.troe[troe, 2] = T3T1          # T1 [K]
    mech.troe[troe, 3] = 0.0           # no T2 term
    return mech


def _flame(mech, n, seed=41):
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


@pytest.fixture(scope="module")
def tiny():
    mech = _tiny_centre_mechanism()
    m = gpu_mechanism(mech)
    yield mech, m
    m.close()


def test_centre_is_below_the_float_range(tiny):
    mech, _ = tiny
    T, _, _ = _flame(mech, 700)
    Fc = np.exp(-T / T3T1)                                   # (1 - a) + a = 1
    assert np.all(Fc < 2.0 ** -100) and np.all(Fc > 2.0 ** -1000)


def test_rates_fp64(cuda, tiny):
    mech, m = tiny
    T, p, Y = _flame(mech, 700)
    Tt, pt, Yt = to_dev(T, p, Y)
    w, h = nk.rates_eval(m, Tt, pt, Yt, precision="fp64")
    w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, scales=True)
    assert scaled_err(host(w), w_o, ws) <= TOL
    assert scaled_err(host(h), h_o, hs) <= TOL


def test_jvp_and_linearizations(cuda, tiny):
    mech, m = tiny
    n = 700
    T, p, Y = _flame(mech, n)
    vT = synth.normal(n, 4101)
    vY = synth.normal((mech.K, n), 4102)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    dw_o, dh_o, dws, dhs = oracle.jvp(mech, T, p, Y, vT, vY, scales=True)
    dw, dh = nk.rates_jvp(m, Tt, pt, Yt, vTt, vYt)
    assert scaled_err(host(dw), dw_o, dws) <= TOL and scaled_err(host(dh), dh_o, dhs) <= TOL
    lin = nk.rates_linearize(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized(m, Tt, pt, Yt, lin, vTt, vYt)
    assert scaled_err(host(dw), dw_o, dws) <= TOL and scaled_err(host(dh), dh_o, dhs) <= TOL
    linc = nk.rates_linearize_compact(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized_compact(m, Tt, pt, Yt, linc, vTt, vYt)
    assert scaled_err(host(dw), dw_o, dws) <= TOL and scaled_err(host(dh), dh_o, dhs) <= TOL


def test_vjp(cuda, tiny):
    mech, m = tiny
    n = 256
    T, p, Y = _flame(mech, n, seed=43)
    wbar = synth.normal((mech.K, n), 4103)
    hbar = synth.normal(n, 4104) * 1e-5
    Tt, pt, Yt, wt, ht = to_dev(T, p, Y, wbar, hbar)
    gT, gY, _ = nk.rates_vjp(m, Tt, pt, Yt, wt, ht)
    J, Js = oracle.jacobian(mech, T, p, Y, scales=True)
    u = np.vstack([wbar, hbar[None, :]])
    JTu = np.einsum("nij,in->jn", J, u)
    scale = np.einsum("nij,in->jn", Js, np.abs(u))
    assert scaled_err(host(gT), JTu[0], scale[0]) <= TOL
    assert scaled_err(host(gY), JTu[1:], scale[1:]) <= TOL
