"""The mechanism-specialised rates kernel (nk_rates_eval with NK_JIT, compiled with NVRTC at
first use) against the oracle (1e-10, cancellation-aware, as the table-driven FP64 forms) and
against the table-driven all-double kernel whose arithmetic it repeats."""
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


@pytest.mark.parametrize("name,n", [("h2_9sp_21rx", 1000 + 13), ("ch4_53sp_325rx", 4096 + 77),
                                    ("big_120sp_700rx", 600)])
def test_jit_rates_vs_oracle(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    nk.mechanism_jit(m)
    T, p, Y = _flame(mech, n, seed=21)
    Y = Y.copy()
    Y[:, 0] = 0.0
    Y[1, 0] = 1.0                                             # a pure species
    Y[2, 1] = 0.0
    Y[:, 1] /= Y[:, 1].sum()                                  # an absent species
    T = T.copy()
    T[2], T[3] = 300.0, 3500.0
    dlnA = synth.normal(mech.R, 91) * 0.3
    Tt, pt, Yt, dt = to_dev(T, p, Y, dlnA)
    for shift, sh in ((None, None), (dt, dlnA)):
        w, h = nk.rates_eval(m, Tt, pt, Yt, dlnA=shift, precision="jit")
        w_o, h_o, ws, hs = oracle.rates(mech, T, p, Y, dlnA=sh, scales=True)
        assert scaled_err(host(w), w_o, ws) <= TOL
        assert scaled_err(host(h), h_o, hs) <= TOL
        w2, h2 = nk.rates_eval(m, Tt, pt, Yt, dlnA=shift, precision="fp64_native")
        assert scaled_err(host(w), host(w2), ws) <= 1e-12 and scaled_err(host(h), host(h2), hs) <= 1e-12


def test_jit_full_size_sampled(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_4096el", mech.K)
    T, p, Y = to_dev(st.T, st.p, st.Y)
    w, h = nk.rates_eval(m, T, p, Y, precision="jit")
    rng = np.random.default_rng(19)
    idx = np.unique(np.concatenate([[0, st.n - 1], rng.choice(st.n, 600, replace=False)]))
    sub = torch.from_numpy(idx).cuda()
    w_o, h_o, ws, hs = oracle.rates(mech, st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx]), scales=True)
    assert scaled_err(host(w[:, sub]), w_o, ws) <= TOL
    assert scaled_err(host(h[sub]), h_o, hs) <= TOL


def test_jit_is_rates_only(cuda):
    m = gpu_mechanism("h2_9sp_21rx")
    mech = synth.mechanism("h2_9sp_21rx")
    T, p, Y = to_dev(*_flame(mech, 16))
    with pytest.raises(nk.NkError):
        nk.rhs_eval(m, T, p, Y, precision="jit")
    w, h = nk.rates_eval(m, T[:0], p[:0], Y[:, :0].contiguous(), precision="jit")     # n = 0
