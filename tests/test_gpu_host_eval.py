"""Host-resident evaluation (nk_host_eval: chunks cycling over streams, 2-D copies of the
species rows) gives the device entry points' results bit for bit: every point's arithmetic is
independent of the chunking."""
import numpy as np
import pytest
import torch

import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev

pytestmark = pytest.mark.gpu


def _states(mech, n, seed=5):
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


@pytest.mark.parametrize("precision,pinned,chunk", [("fp64", True, 1024), ("mixed", True, 4096),
                                                    ("fp64_native", False, 3000), ("fp64", False, 1 << 20)])
def test_host_eval_matches_device(cuda, precision, pinned, chunk):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    n = 10000 + 7
    T, p, Y = _states(mech, n)
    hT, hp, hY = (torch.from_numpy(a) for a in (T, p, Y))
    if pinned:
        hT, hp, hY = hT.pin_memory(), hp.pin_memory(), hY.pin_memory()
    w, h, mu, lam, D = nk.host_eval(m, hT, hp, hY, precision=precision, chunk=chunk)
    torch.cuda.synchronize()
    Tt, pt, Yt = to_dev(T, p, Y)
    w_d, h_d = nk.rates_eval(m, Tt, pt, Yt, precision=precision)
    mu_d, lam_d, D_d = nk.transport_eval(m, Tt, pt, Yt, precision=precision)
    for a, b in ((w, w_d), (h, h_d), (mu, mu_d), (lam, lam_d), (D, D_d)):
        assert torch.equal(a, b.cpu())


def test_host_eval_partial_outputs_and_errors(cuda):
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    n = 777
    T, p, Y = _states(mech, n)
    hT, hp, hY = (torch.from_numpy(a).pin_memory() for a in (T, p, Y))
    w = torch.full((mech.K, n), -1.0, dtype=torch.float64).pin_memory()
    mu = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
    nk.host_eval(m, hT, hp, hY, chunk=100, outputs=(w, None, mu, None, None))
    Tt, pt, Yt = to_dev(T, p, Y)
    assert torch.equal(w, nk.rates_eval(m, Tt, pt, Yt)[0].cpu())
    assert torch.equal(mu, nk.transport_eval(m, Tt, pt, Yt)[0].cpu())
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(nk.NkError):
        nk.host_eval(m, hT, hp, hY, chunk=100, workspace=ws)     # too small
    with pytest.raises(nk.NkError):
        nk.host_eval(m, hT, hp, hY, precision="jit")             # not a host-evaluation form
