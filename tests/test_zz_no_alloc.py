"""nk_rates_vjp_noalloc: the vector-Jacobian product for callers that cannot allocate device
memory or pass a workspace (a solver callback with a fixed signature, or code under a
memory pool that owns the device).  Its ln A partial sums live in a fixed scratch array
inside the library instead.  Checked through the C ABI against nk_rates_vjp on the same
inputs, on two calls in a row with different cotangents (the scratch keeps whatever the
previous call left in it, so stale contents would show up in the second call)."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_vjp_matches_workspace_vjp():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    mech = synth.mechanism("ch4_53sp_325rx")
    m = nk.mechanism_load(mech)
    L = nk.lib()
    st = synth.states_flame(mech.K, 27, seed=12)          # 13,824 points, several blocks
    n = st.n
    T, p, Y = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (st.T, st.p, st.Y))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        wbar = torch.from_numpy(synth.normal((mech.K, n), 100 + call)).cuda()
        hbar = torch.from_numpy(synth.normal(n, 200 + call) * 1e-5).cuda()
        gT_ref, gY_ref, g_ref = nk.rates_vjp(m, T, p, Y, wbar, hbar)
        gT = torch.empty_like(T)
        gY = torch.empty_like(Y)
        g = torch.full((mech.R,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        status = L.nk_rates_vjp_noalloc(m.handle, n, n, _ptr(T), _ptr(p), _ptr(Y), None, _ptr(wbar), _ptr(hbar),
                                        _ptr(gT), _ptr(gY), _ptr(g), stream)
        assert status == 0, L.nk_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0      # nothing allocated by the call
        for a, b in ((gT, gT_ref), (gY, gY_ref), (g, g_ref)):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.allclose(a, b, rtol=TOL, atol=TOL * np.max(np.abs(b)))
    m.close()


def test_noalloc_vjp_rejects_oversized_reduction_and_handles_empty():
    torch.cuda.set_device(0)
    # R large enough that one R-vector per resident block (at least one block per SM) exceeds
    # the 8 MiB scratch
    big = synth.make_mechanism(K=40, R=8000, n_tb=4, n_troe=4, seed=77)
    m = nk.mechanism_load(big)
    L = nk.lib()
    n = 1 << 16
    T = torch.full((n,), 1500.0, dtype=torch.float64, device="cuda")
    p = torch.full((n,), 101325.0, dtype=torch.float64, device="cuda")
    Y = torch.full((big.K, n), 1.0 / big.K, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(Y)
    gT, gY = torch.empty_like(T), torch.empty_like(Y)
    g = torch.empty(big.R, dtype=torch.float64, device="cuda")
    assert nk.rates_vjp_workspace(m, n) > 8 * 2 ** 20
    status = L.nk_rates_vjp_noalloc(m.handle, n, n, _ptr(T), _ptr(p), _ptr(Y), None, _ptr(w), None, _ptr(gT),
                                    _ptr(gY), _ptr(g), None)
    assert status == 5 and b"scratch" in L.nk_last_error()
    # without the ln A gradient no scratch is needed at all
    status = L.nk_rates_vjp_noalloc(m.handle, n, n, _ptr(T), _ptr(p), _ptr(Y), None, _ptr(w), None, _ptr(gT),
                                    _ptr(gY), None, None)
    assert status == 0
    # an empty point set gives a zero gradient
    g.fill_(1.0)
    status = L.nk_rates_vjp_noalloc(m.handle, 0, 0, None, None, None, None, None, None, None, None, _ptr(g), None)
    assert status == 0
    torch.cuda.synchronize()
    assert torch.all(g == 0)
    m.close()
