"""Dense Jacobian of the implicit-stage sources (nk_rhs_jacobian) against the oracle's
complex-step Jacobian (1e-10 of the per-entry derivative magnitudes), and the block-Jacobi
preconditioner (nk_block_jacobi_factor / _apply) against the blocks I - dt diag(w) J diag(1/w)
formed on the host from the checked Jacobian: the stored factors reproduce the row-scaled,
permuted block and z = P^-1 v solves it to double-precision backward error."""
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


def _edge(T, p, Y):
    """A pure species, absent species, a nearly pure mixture, T at the range ends."""
    T, Y = T.copy(), Y.copy()
    Y[:, 0] = 0.0
    Y[1, 0] = 1.0
    Y[2:5, 1] = 0.0
    Y[:, 1] /= Y[:, 1].sum()
    Y[:, 2] = 1e-12
    Y[0, 2] = 1.0 - (Y.shape[0] - 1) * 1e-12
    T[3], T[4] = 300.0, 3500.0
    return T, p, Y


def _jacobian(m, T, p, Y):
    Tt, pt, Yt = to_dev(T, p, Y)
    lin = nk.rates_linearize(m, Tt, pt, Yt)
    fT, fY = nk.rhs_eval(m, Tt, pt, Yt)
    return nk.rhs_jacobian(m, Tt, pt, Yt, lin, fT, fY), (Tt, pt, Yt, lin, fT, fY)


@pytest.mark.parametrize("name,n", [("ch4_53sp_325rx", 300 + 17), ("h2_9sp_21rx", 1000), ("big_120sp_700rx", 150)])
def test_jacobian_vs_complex_step(cuda, name, n):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    T, p, Y = _edge(*_flame(mech, n, seed=11))
    J, _ = _jacobian(m, T, p, Y)
    J_o, Js = oracle.rhs_jacobian(mech, T, p, Y, scales=True)
    assert J.shape == (mech.K + 1, mech.K + 1, n)
    # (at the pure mixture the oracle's complex step keeps a remainder of h^2/6 times a third
    # derivative, ~1e-190, where the exact entry is 0: an absolute floor far below any entry)
    assert scaled_err(np.moveaxis(host(J), 2, 0), J_o, Js + 1e-60) <= TOL


def test_jacobian_times_vector_is_the_jvp(cuda):
    """J v from the dense blocks against nk_rhs_jvp along the same directions (two independent
    CUDA paths), relative to the oracle's derivative magnitudes along v plus |J| |v|."""
    mech = synth.mechanism("ch4_53sp_325rx")
    m = gpu_mechanism("ch4_53sp_325rx")
    n = 500
    T, p, Y = _flame(mech, n, seed=12)
    J, (Tt, pt, Yt, *_rest) = _jacobian(m, T, p, Y)
    v = synth.normal((mech.K + 1, n), 77) * np.vstack([T[None], Y + 1e-12])
    vt = torch.from_numpy(v).cuda()
    dfT, dfY = nk.rhs_jvp(m, Tt, pt, Yt, vt[0].contiguous(), vt[1:].contiguous())
    Jv = host(torch.einsum("rcn,cn->rn", J, vt))
    absJv = host(torch.einsum("rcn,cn->rn", J.abs(), vt.abs()))
    _, _, sT, sY = oracle.rhs_jvp(mech, T, p, Y, v[0], np.ascontiguousarray(v[1:]), scales=True)
    scale = np.vstack([sT[None], sY]) + absJv
    got = np.vstack([host(dfT)[None], host(dfY)])
    assert scaled_err(Jv, got, scale) <= 1e-10


def _weights(T, Y, rtol=1e-6, atolT=1e-6, atolY=1e-12):
    x = np.vstack([T[None], Y])
    atol = np.full((x.shape[0], 1), atolY)
    atol[0] = atolT
    return 1.0 / (rtol * np.abs(x) + atol)


@pytest.mark.parametrize("name,n,dt", [("h2_9sp_21rx", 700, 1e-6), ("ch4_53sp_325rx", 200 + 9, 1e-7),
                                       ("ch4_53sp_325rx", 64, 0.0), ("big_120sp_700rx", 90, 1e-8)])
def test_block_jacobi_factors_and_solve(cuda, name, n, dt):
    mech = synth.mechanism(name)
    m = gpu_mechanism(name)
    N = mech.K + 1
    T, p, Y = _flame(mech, n, seed=13)
    _, (Tt, pt, Yt, lin, fT, fY) = _jacobian(m, T, p, Y)
    w = _weights(T, Y)
    F, perm = nk.block_jacobi_factor(m, Tt, pt, Yt, lin, fT, fY, torch.from_numpy(w).cuda(), dt)
    # the blocks from the oracle's Jacobian; an entry may differ by the Jacobian's parity
    # tolerance (1e-10 of the derivative magnitudes) plus the factorization's rounding
    J_o, Js = oracle.rhs_jacobian(mech, T, p, Y, scales=True)
    ratio = w.T[:, :, None] / w.T[:, None, :]
    P = np.eye(N)[None] - dt * ratio * J_o
    Ps = np.eye(N)[None] + dt * ratio * Js
    Fh = np.moveaxis(host(F), 2, 0)                                  # [n, N, N]
    pw = host(perm).astype(np.int64).T                               # [n, N] pivot words
    ph, ex = pw & 0xFFFF, pw >> 16                                   # pivot rows, their exponents
    assert np.all(np.sort(ph, axis=1) == np.arange(N)[None])       # a permutation per point
    D = np.ldexp(1.0, -ex)[:, :, None]
    Pp = np.take_along_axis(P, ph[:, :, None], axis=1) * D          # (D P)[perm]
    Pps = np.take_along_axis(Ps, ph[:, :, None], axis=1) * D
    # L U = (D P)[perm] with L unit lower, U upper (1/U_kk stored on the diagonal)
    L = np.tril(Fh, -1) + np.eye(N)[None]
    U = np.triu(Fh, 1) + np.eye(N)[None] / np.diagonal(Fh, axis1=1, axis2=2)[:, :, None] * np.eye(N)[None]
    LU = L @ U
    scale = np.abs(L) @ np.abs(U)
    assert np.all(np.abs(LU - Pp) <= 1e-10 * Pps + 1e-12 * scale + 1e-300)
    # row scales 2^-e put each row's largest entry in [1/2, 1)
    big = np.abs(LU).max(axis=2)
    assert np.all((big >= 0.5 * (1 - 1e-9)) & (big < 1.0 + 1e-9))
    # z = P^-1 v: backward error of the factored system, (D P)[perm] z = (D v)[perm] to a small
    # multiple of the rounding unit times |L| |U| |z| (the bound of LU with partial pivoting)
    v = synth.normal((N, n), 91)
    z = host(nk.block_jacobi_apply(m, F, perm, torch.from_numpy(v).cuda()))
    Dv = np.take_along_axis(v.T, ph, axis=1) * np.ldexp(1.0, -ex)     # [n, N], pivot order
    r = np.einsum("nrc,nc->nr", LU, z.T) - Dv
    back = np.einsum("nrc,nc->nr", scale, np.abs(z.T)) + np.abs(Dv)
    assert np.all(np.abs(r) <= 1e-12 * back + 1e-300)
    if dt == 0.0:                                                     # P = I: exact
        assert np.array_equal(z, v)


def test_block_jacobi_argument_errors(cuda):
    mech = synth.mechanism("h2_9sp_21rx")
    m = gpu_mechanism("h2_9sp_21rx")
    T, p, Y = _flame(mech, 32)
    _, (Tt, pt, Yt, lin, fT, fY) = _jacobian(m, T, p, Y)
    w = torch.from_numpy(_weights(T, Y)).cuda()
    with pytest.raises(nk.NkError):
        nk.block_jacobi_factor(m, Tt, pt, Yt, lin, fT, fY, w, -1.0)
    with pytest.raises(nk.NkError):
        nk.block_jacobi_factor(m, Tt, pt, Yt, lin, fT, fY, w, float("nan"))


def test_largest_supported_block(cuda):
    """K = 159 (K + 1 = 160, the largest block that fits in shared memory): factors and solve as
    above, with the blocks from nk_rhs_jacobian; K = 160 is refused."""
    mech = synth.make_mechanism(159, 400, 20, 20, seed=7)
    m = gpu_mechanism(mech)
    N, n, dt = mech.K + 1, 40, 1e-8
    st = synth.states_uniform(mech.K, n, seed=5, T_lo=900.0, T_hi=2400.0)
    T, p, Y = st.T, st.p, np.ascontiguousarray(st.Y)
    J, (Tt, pt, Yt, lin, fT, fY) = _jacobian(m, T, p, Y)
    w = _weights(T, Y)
    F, perm = nk.block_jacobi_factor(m, Tt, pt, Yt, lin, fT, fY, torch.from_numpy(w).cuda(), dt)
    Jh = np.moveaxis(host(J), 2, 0)
    P = np.eye(N)[None] - dt * (w.T[:, :, None] * Jh / w.T[:, None, :])
    Fh = np.moveaxis(host(F), 2, 0)
    pw = host(perm).astype(np.int64).T
    ph, ex = pw & 0xFFFF, pw >> 16
    assert np.all(np.sort(ph, axis=1) == np.arange(N)[None])
    Pp = np.take_along_axis(P, ph[:, :, None], axis=1) * np.ldexp(1.0, -ex)[:, :, None]
    L = np.tril(Fh, -1) + np.eye(N)[None]
    U = np.triu(Fh, 1) + np.eye(N)[None] / np.diagonal(Fh, axis1=1, axis2=2)[:, :, None] * np.eye(N)[None]
    scale = np.abs(L) @ np.abs(U)
    # (P from the Jacobian kernel, the factors from the set-up kernel: the same expressions, so
    # the entries agree to rounding, except where an entry is a cancellation; the 9-digit
    # tolerance on |L| |U| covers those)
    assert np.all(np.abs(L @ U - Pp) <= 1e-9 * scale + 1e-300)
    v = synth.normal((N, n), 92)
    z = host(nk.block_jacobi_apply(m, F, perm, torch.from_numpy(v).cuda()))
    Dv = np.take_along_axis(v.T, ph, axis=1) * np.ldexp(1.0, -ex)
    r = np.einsum("nrc,nc->nr", L @ U, z.T) - Dv
    assert np.all(np.abs(r) <= 1e-12 * (np.einsum("nrc,nc->nr", scale, np.abs(z.T)) + np.abs(Dv)) + 1e-300)
    big = synth.make_mechanism(160, 300, 10, 10, seed=8)
    mb = gpu_mechanism(big)
    with pytest.raises(nk.NkError):
        nk.reactor_workspace(mb, 16, 10, 1)
