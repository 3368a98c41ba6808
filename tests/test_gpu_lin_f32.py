"""Single-precision products from the float linearization (nk_rates_linearize_f32,
nk_rates_jvp_linearized_f32, nk_rhs_jvp_linearized_f32).

Storage: each reaction's coefficients are the double linearization's scaled by a power of two
and rounded to float, the S1 sum is kept as its double's two words and h_k/RT is rounded to
float; checked against nk_rates_linearize at the same states.

The products are checked against the oracle's complex-step JVPs with a bound derived from the
arithmetic.  Result k adds its terms in float (scaled by powers of two, which is exact): each
term carries the rounding of its stored coefficient, of the concentration tangent it multiplies
(formed in float from rounded inputs), of the product and of its share of dq_r, about 8u, and
the accumulation over the t_k reactions the species takes part in adds up to t_k u, u = 2^-24;
so |error_k| <= (t_k + 8) u sum_terms |term|, doubled for the density terms the kernel forms
per species instead of per column.  The sum of the terms' magnitudes is bounded, column by
column, by the oracle's per-entry Jacobian magnitudes (sum over reactions of |d forward| +
|d reverse|) times |v_j|; the temperature and heat-release rows take t = R."""
import numpy as np
import pytest
import torch

import oracle
import paper_2409_06404_gb300 as nk
from paper_2409_06404_gb300 import synth
from conftest import gpu_mechanism, to_dev, host, nu_matrix, R_GAS

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _flame(mech, n, seed=3):
    st = synth.states_flame(mech.K, 27, seed=seed)
    idx = np.linspace(0, st.n - 1, n).astype(int)
    return st.T[idx], st.p[idx], np.ascontiguousarray(st.Y[:, idx])


def _terms(mech):
    """Reactions each species takes part in, [K]."""
    t = np.zeros(mech.K, dtype=np.int64)
    for r in range(mech.R):
        sp = set(mech.reac_sp[mech.reac_ptr[r]:mech.reac_ptr[r + 1]]) | \
            set(mech.prod_sp[mech.prod_ptr[r]:mech.prod_ptr[r + 1]])
        for k in sp:
            t[k] += 1
    return t


def _bound(Js, vT, vY, t_rows):
    """2 (t + 8) u sum_j Js[:, :, j] |v_j| per point: [n, rows], and the magnitudes."""
    av = np.vstack([np.abs(vT)[None], np.abs(vY)]).T                 # [n, K+1]
    S = np.einsum("nrc,nc->nr", Js, av)
    return 2.0 * (t_rows[None, :] + 8) * U * S, S


def _check(got, ref, bound, S, what):
    # a floor far below any resolved entry: terms under the normal float range (2^-126) are
    # flushed; 1e-25 of the point's largest magnitude covers them
    floor = 1e-25 * S.max(axis=1, keepdims=True)
    err = np.abs(got - ref)
    ratio = err / (bound + floor)
    assert np.all(ratio <= 1.0), (what, float(ratio.max()), np.unravel_index(ratio.argmax(), ratio.shape))
    # and the bulk sits well inside it
    assert np.median(err / (U * S + floor)) < 8.0, what


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 700 + 21), ("h2_9sp_21rx", 1000), ("big_120sp_700rx", 150)])
def test_stored_floats(cuda, name, n):
    """Coefficient words are the double coefficients times a power of two, rounded to nearest
    (or dropped far below their reaction's largest); the two S1 words are its double; h_k/RT are
    the doubles rounded; one exponent word per reaction."""
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=21)
    Tt, pt, Yt = to_dev(T, p, Y)
    l64 = host(nk.rates_linearize(m, Tt, pt, Yt))
    l32 = host(nk.rates_linearize_f32(m, Tt, pt, Yt))
    nS = l64.shape[0] - mech.K - 1                                    # coefficient slots
    assert l32.dtype == np.float32 and l32.shape == (nk.linearization_slots_f32(m), n)
    assert l32.shape[0] == l64.shape[0] + 1 + mech.R + mech.K
    c64, c32 = l64[:nS], l32[:nS].astype(np.float64)
    nz = (c64 != 0) & (c32 != 0)
    k = np.round(np.log2(np.abs(c64[nz]) / np.abs(c32[nz])))
    back = np.ldexp(c32[nz], k.astype(np.int64))
    assert np.all(np.abs(back - c64[nz]) <= 2.0 ** -24 * np.abs(c64[nz]))   # rounded to nearest
    assert np.all(np.sign(c32[nz]) == np.sign(c64[nz]))
    # words dropped to zero stand for coefficients far below the largest at that point
    dropped = (c64 != 0) & (c32 == 0)
    big = np.abs(c64).max(axis=0, keepdims=True)
    assert np.all(np.abs(c64)[dropped] <= 2.0 ** -100 * np.broadcast_to(big, c64.shape)[dropped])
    words = np.ascontiguousarray(l32[nS:nS + 2]).view(np.uint32).astype(np.uint64)
    S1 = (words[0] | (words[1] << np.uint64(32))).view(np.float64)
    # S1 = sum_r q_r sum_k nu_kr c_p,k/R: the same sum, its reactions possibly split over another
    # number of parts (launch shapes differ), so equal to the summation order's rounding
    fwd, rev = oracle.rates_of_progress(mech, T, p, Y)
    dcp = nu_matrix(mech).T @ (oracle.thermo(mech, T, p, Y)["cp_k"] / R_GAS)     # [R, n]
    scale = ((np.abs(fwd) + np.abs(rev)) * np.abs(dcp)).sum(axis=0)
    assert np.all(np.abs(S1 - l64[nS]) <= 1e-12 * scale)
    assert np.array_equal(l32[nS + 2:nS + 2 + mech.K], l64[nS + 1:].astype(np.float32))
    ex = np.ascontiguousarray(l32[nS + 2 + mech.K:]).view(np.int32)
    assert ex.shape == (mech.R + mech.K, n) and np.all(np.abs(ex[:mech.R]) < 1100)
    # E_k: the largest exponent of the reactions species k takes part in
    er, ek = ex[:mech.R], ex[mech.R:]
    # (the exponent words are in the library's reaction order; E_k is their maximum over the
    # reactions of the species, whatever the order, so compare through the per-species sets)
    part_of = _terms(mech) > 0
    assert np.all(ek[~part_of] == -2000)
    assert np.all(ek[part_of] >= er.min(axis=0)[None]) and np.all(ek[part_of] <= er.max(axis=0)[None])
    assert np.all(ek[part_of].max(axis=0) == er.max(axis=0))


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 600 + 13), ("h2_9sp_21rx", 800), ("big_120sp_700rx", 120)])
def test_f32_rates_jvp_vs_complex_step(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=22)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize_f32(m, Tt, pt, Yt)
    _, Js = oracle.jacobian(mech, T, p, Y, scales=True)
    t_rows = np.concatenate([_terms(mech), [mech.R]])                 # rows omega_k, hrr
    for d in range(2):
        vT = synth.normal(n, 5100 + 2 * d) * 30.0
        vY = synth.normal((mech.K, n), 5101 + 2 * d) * (Y + 1e-12)
        vTt, vYt = to_dev(vT, vY)
        dw, dh = nk.rates_jvp_linearized_f32(m, Tt, pt, Yt, lin, vTt, vYt)
        dw_o, dh_o = oracle.jvp(mech, T, p, Y, vT, vY)
        bound, S = _bound(Js, vT, vY, t_rows)
        got = np.vstack([host(dw), host(dh)[None]]).T
        ref = np.vstack([dw_o, dh_o[None]]).T
        _check(got, ref, bound, S, (name, d))


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 500 + 7), ("h2_9sp_21rx", 800), ("big_120sp_700rx", 120)])
def test_f32_sources_jvp_vs_complex_step(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _flame(mech, n, seed=23)
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize_f32(m, Tt, pt, Yt)
    fT, fY = nk.rhs_eval(m, Tt, pt, Yt)
    _, Js = oracle.rhs_jacobian(mech, T, p, Y, scales=True)
    t_rows = np.concatenate([[mech.R], _terms(mech)])                 # rows fT, fY_k
    for d in range(2):
        vT = synth.normal(n, 5200 + 2 * d) * 30.0
        vY = synth.normal((mech.K, n), 5201 + 2 * d) * (Y + 1e-12)
        vTt, vYt = to_dev(vT, vY)
        dfT, dfY = nk.rhs_jvp_linearized_f32(m, Tt, pt, Yt, lin, fT, fY, vTt, vYt)
        dT_o, dY_o = oracle.rhs_jvp(mech, T, p, Y, vT, vY)
        bound, S = _bound(Js, vT, vY, t_rows)
        got = np.vstack([host(dfT)[None], host(dfY)]).T
        ref = np.vstack([dT_o[None], dY_o]).T
        _check(got, ref, bound, S, (name, d))


def test_f32_strided_chunk_and_argument_errors(cuda):
    """A chunk of a wider field with its linearization in a wider buffer gives the same bits;
    a double buffer is refused by the binding, a short ldl by the library."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    T, p, Y = _flame(mech, 300, seed=24)
    vT, vY = synth.normal(300, 5), synth.normal((mech.K, 300), 6) * (Y + 1e-12)
    Tt, pt, Yt, vTt, vYt = to_dev(T, p, Y, vT, vY)
    lin = nk.rates_linearize_f32(m, Tt, pt, Yt)
    dw, dh = nk.rates_jvp_linearized_f32(m, Tt, pt, Yt, lin, vTt, vYt)
    a, b = 37, 200
    big = torch.full((nk.linearization_slots_f32(m), 500), float("nan"), dtype=torch.float32, device="cuda")
    lin2 = nk.rates_linearize_f32(m, Tt[a:b], pt[a:b], Yt[:, a:b], lin=big)
    dw2, dh2 = nk.rates_jvp_linearized_f32(m, Tt[a:b], pt[a:b], Yt[:, a:b], lin2, vTt[a:b], vYt[:, a:b])
    assert torch.equal(dw2, dw[:, a:b]) and torch.equal(dh2, dh[a:b])
    with pytest.raises(ValueError):
        nk.rates_jvp_linearized_f32(m, Tt, pt, Yt, lin.double(), vTt, vYt)
    st = nk.lib().nk_rates_linearize_f32(m.handle, 300, 300, nk._ptr(Tt), nk._ptr(pt), nk._ptr(Yt), None,
                                         nk._ptr(lin), 299, None)
    assert st == 1                                                    # NK_EINVAL: ldl < n
