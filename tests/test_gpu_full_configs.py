"""Full-size workloads in the benchmark's launch configuration, checked on sampled points
against the oracle:

* 120 species / 700 reactions on the 2,097,152-point flame field, FP64 and mixed forms, with
  the mixed form's error per output (maximum and 99.9th percentile);
* the implicit-stage workload: 53 species on 32^3 elements x 512 points = 16,777,216 points,
  one mixed forward (thermo, rates, transport) and ten JVPs along seeded N(0, 1) directions,
  as a Newton-Krylov stage issues them, rates of progress recomputed for each;
* the reactor step on 2,097,152 near-equilibrium points, unpreconditioned, block-Jacobi and with
  single-precision products from the float linearization.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, scaled_err, P_ATM

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL64 = 1e-10
TOLMIX = 1e-5


def _per_point_err(actual, expect, scale):
    """max over species (rows) of |actual - expect| / scale per point (columns)."""
    a, e, s = (np.atleast_2d(x) for x in (actual, expect, scale))
    return np.max(np.abs(a - e) / np.maximum(s, 1e-300), axis=0)


def test_120sp_full_size_sampled_fp64_and_mixed(cuda):
    mech = synth.mechanism("big_120sp_700rx")
    m = gpu_mechanism("big_120sp_700rx")
    st = synth.workload_states("flame_4096el", mech.K)
    assert st.n == 2_097_152
    T, p, Y = to_dev(st.T, st.p, st.Y)
    w, h = nk.rates_eval(m, T, p, Y)
    mu, lam, D = nk.transport_eval(m, T, p, Y)
    wm, hm = nk.rates_eval(m, T, p, Y, precision="mixed")
    mum, lamm, Dm = nk.transport_eval(m, T, p, Y, precision="mixed")
    rng = np.random.default_rng(120)
    idx = np.unique(np.concatenate([[0, st.n - 1], rng.choice(st.n, 1200, replace=False)]))
    Ts, ps, Ys = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    w_o, h_o, ws, hs = oracle.rates(mech, Ts, ps, Ys, scales=True)
    mu_o, lam_o, D_o = oracle.transport(mech, Ts, ps, Ys)
    # FP64 form
    assert scaled_err(host(w)[:, idx], w_o, ws) <= TOL64
    assert scaled_err(host(h)[idx], h_o, hs) <= TOL64
    assert scaled_err(host(mu)[idx], mu_o, mu_o) <= TOL64
    assert scaled_err(host(lam)[idx], lam_o, lam_o) <= TOL64
    assert scaled_err(host(D)[:, idx], D_o, D_o) <= TOL64
    # mixed form, per output
    errs = {
        "omega": _per_point_err(host(wm)[:, idx], w_o, ws),
        "hrr": _per_point_err(host(hm)[idx], h_o, hs),
        "mu": _per_point_err(host(mum)[idx], mu_o, mu_o),
        "lambda": _per_point_err(host(lamm)[idx], lam_o, lam_o),
        "D": _per_point_err(host(Dm)[:, idx], D_o, D_o),
    }
    print("\n120 species, 2,097,152 points, mixed form vs oracle (sampled):")
    for k, e in errs.items():
        print(f"  {k:7s} max {e.max():.2e}  p99.9 {np.quantile(e, 0.999):.2e}")
        assert e.max() <= TOLMIX, k
    for t in (h, mu, lam, hm, mum, lamm):
        assert torch.isfinite(t).all()


def test_implicit_stage_16M_points_sampled(cuda):
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_32768el", mech.K)
    n, K = st.n, mech.K
    assert n == 16_777_216
    T, p, Y = to_dev(st.T, st.p, st.Y)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 800, replace=False)]))
    Ts, ps, Ys = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    del st

    # one mixed forward: thermo (FP64), rates and transport (mixed)
    th = nk.thermo_eval(m, T, p, Y)
    wm, hm = nk.rates_eval(m, T, p, Y, precision="mixed")
    mum, lamm, Dm = nk.transport_eval(m, T, p, Y, precision="mixed")
    o = oracle.thermo(mech, Ts, ps, Ys)
    assert scaled_err(host(th["cp_mix"])[idx], o["cp_mix"], np.abs(o["cp_mix"])) <= TOL64
    hscale = np.sum(np.abs(Ys * o["h_k"]) / mech.W[:, None], axis=0)
    assert scaled_err(host(th["h_mix"])[idx], o["h_mix"], hscale) <= TOL64
    w_o, h_o, ws, hs = oracle.rates(mech, Ts, ps, Ys, scales=True)
    assert scaled_err(host(wm)[:, idx], w_o, ws) <= TOLMIX
    assert scaled_err(host(hm)[idx], h_o, hs) <= TOLMIX
    mu_o, lam_o, D_o = oracle.transport(mech, Ts, ps, Ys)
    assert scaled_err(host(mum)[idx], mu_o, mu_o) <= TOLMIX
    assert scaled_err(host(lamm)[idx], lam_o, lam_o) <= TOLMIX
    assert scaled_err(host(Dm)[:, idx], D_o, D_o) <= TOLMIX
    del wm, mum, lamm, Dm, th

    # ten JVPs along seeded directions, one buffer set reused (rates recomputed each time)
    vT = torch.empty(n, dtype=torch.float64, device="cuda")
    vY = torch.empty((K, n), dtype=torch.float64, device="cuda")
    sub = torch.from_numpy(idx).cuda()
    for d in range(10):
        g = torch.Generator(device="cuda").manual_seed(5000 + d)
        torch.randn(n, generator=g, out=vT)
        torch.randn((K, n), generator=g, out=vY)
        dw, dh = nk.rates_jvp(m, T, p, Y, vT, vY)
        if d in (0, 4, 9):
            vTs, vYs = host(vT[sub]), np.ascontiguousarray(host(vY[:, sub]))
            dw_o, dh_o, dws, dhs = oracle.jvp(mech, Ts, ps, Ys, vTs, vYs, scales=True)
            assert scaled_err(host(dw[:, sub]), dw_o, dws) <= TOL64, d
            assert scaled_err(host(dh[sub]), dh_o, dhs) <= TOL64, d
        assert torch.isfinite(dh).all()
        del dw, dh


def test_implicit_stage_16M_points_compact_sampled(cuda):
    """The implicit-stage workload with the per-reaction stored linearization (158 GB at
    16,777,216 points, beside the 7.4 GB state): one pass giving the rates at the state and the
    stored data, then ten JVPs along the same seeded directions as the recomputing sweep, three
    of them sampled against the oracle (1e-10)."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    st = synth.workload_states("flame_32768el", mech.K)
    n, K = st.n, mech.K
    assert n == 16_777_216
    T, p, Y = to_dev(st.T, st.p, st.Y)
    rng = np.random.default_rng(55)
    idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 800, replace=False)]))
    Ts, ps, Ys = st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])
    del st
    sub = torch.from_numpy(idx).cuda()
    lin, w, h = nk.rates_linearize_compact(m, T, p, Y, primal=True)
    w_o, h_o, ws, hs = oracle.rates(mech, Ts, ps, Ys, scales=True)
    assert scaled_err(host(w[:, sub]), w_o, ws) <= TOL64
    assert scaled_err(host(h[sub]), h_o, hs) <= TOL64
    assert torch.isfinite(h).all()
    del w, h
    vT = torch.empty(n, dtype=torch.float64, device="cuda")
    vY = torch.empty((K, n), dtype=torch.float64, device="cuda")
    for d in range(10):
        g = torch.Generator(device="cuda").manual_seed(5000 + d)
        torch.randn(n, generator=g, out=vT)
        torch.randn((K, n), generator=g, out=vY)
        dw, dh = nk.rates_jvp_linearized_compact(m, T, p, Y, lin, vT, vY)
        if d in (0, 4, 9):
            vTs, vYs = host(vT[sub]), np.ascontiguousarray(host(vY[:, sub]))
            dw_o, dh_o, dws, dhs = oracle.jvp(mech, Ts, ps, Ys, vTs, vYs, scales=True)
            assert scaled_err(host(dw[:, sub]), dw_o, dws) <= TOL64, d
            assert scaled_err(host(dh[sub]), dh_o, dhs) <= TOL64, d
        assert torch.isfinite(dh).all()
        del dw, dh
    del lin
    torch.cuda.empty_cache()


def test_reactor_step_full_size_sampled(cuda):
    """The reactor step at the benchmark's size (2,097,152 points, 53 species), unpreconditioned,
    block-Jacobi and with single-precision products (linearized 2), on near-equilibrium states built as the benchmark builds them (512
    equilibria from element potentials, here with the oracle's Gibbs energies, tiled over the
    points and perturbed by 1e-3 in Y and ~1 K in T); 100 sampled points against the oracle's
    dense Newton solution (weighted RMS difference within 1e-3 of the tolerance weights)."""
    from test_oracle_rates import equilibrium_state
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    n, nu = 2097152, 512
    rng = np.random.default_rng(6053)
    Tu = np.linspace(1300.0, 2600.0, nu)
    Yu = np.stack([equilibrium_state(mech, Tu[j], P_ATM, rng) for j in range(nu)], axis=1)
    idx = np.arange(n) % nu
    T = Tu[idx] + rng.standard_normal(n)
    Y = Yu[:, idx] * (1.0 + 1e-3 * rng.standard_normal((mech.K, n)))
    Y /= Y.sum(0)
    Y = np.ascontiguousarray(Y)
    p = np.full(n, P_ATM)
    rtol, atolT, atolY, dt = 1e-6, 1e-6, 1e-12, 1e-9
    samp = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 98, replace=False)]))
    T_o, Y_o, it = oracle.reactor_step(mech, T[samp], p[samp], np.ascontiguousarray(Y[:, samp]), dt,
                                       atol_T=atolT, atol_Y=atolY)
    assert np.all(it > 0)
    wT = 1.0 / (rtol * np.abs(T[samp]) + atolT)
    wY = 1.0 / (rtol * np.abs(Y[:, samp]) + atolY)
    pt = torch.from_numpy(p).cuda()
    for precond, linearized in ((0, 0), (1, 0), (0, 2)):
        Tt, Yt = to_dev(T, Y)
        o = nk.reactor_opts(rtol=rtol, atol_T=atolT, atol_Y=atolY, newton_tol=1e-4, lin_tol=1e-6, max_newton=20,
                            krylov_dim=30, precond=precond, linearized=linearized)
        st = nk.reactor_step(m, Tt, pt, Yt, dt, o)
        assert st["converged"] == 1, (precond, linearized, st)
        sub = torch.from_numpy(samp).cuda()
        d = np.concatenate([((host(Tt[sub]) - T_o) * wT)[None], (host(Yt[:, sub]) - Y_o) * wY])
        assert np.sqrt(np.mean(d ** 2)) <= 1e-3, (precond, linearized)
        del Tt, Yt
        torch.cuda.empty_cache()
