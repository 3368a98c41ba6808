"""CPU oracle for the pointwise thermochemistry (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The CUDA library never does, and this package
imports nothing from the library: it takes a mechanism object with the generator's array
fields (see ``paper_2409_06404_gb300.synth.Mechanism``) and numpy state arrays.

The C++ source ``nkoracle.cpp`` is compiled with the host compiler at ``-O2`` without
fast-math and with OpenMP over points.  Its header comment lists the definitions it writes
out and where the paper names each quantity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nkoracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_c_dbl = ctypes.c_double
_p_dbl = ctypes.POINTER(ctypes.c_double)
_p_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (skipped when up to date)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Mech(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32), ("R", ctypes.c_int32), ("n_elem", ctypes.c_int32),
        ("W", _p_dbl), ("atoms", _p_i32), ("nasa_lo", _p_dbl), ("nasa_hi", _p_dbl), ("T_mid", _p_dbl),
        ("reac_ptr", _p_i32), ("reac_sp", _p_i32), ("reac_nu", _p_i32),
        ("prod_ptr", _p_i32), ("prod_sp", _p_i32), ("prod_nu", _p_i32),
        ("rtype", _p_i32), ("lnA", _p_dbl), ("beta", _p_dbl), ("Ea", _p_dbl),
        ("lnA0", _p_dbl), ("beta0", _p_dbl), ("Ea0", _p_dbl), ("troe", _p_dbl), ("eff", _p_dbl),
        ("mu_fit", _p_dbl), ("lam_fit", _p_dbl), ("D_fit", _p_dbl), ("p_ref", ctypes.c_double),
    ]


def build_variant(source_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source to ``out_path`` (used by the mutation tests
    that check the pins catch planted mistakes)."""
    src = out_path + ".cpp"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                    "-ffp-contract=off", "-o", out_path, src], check=True)
    return out_path


class use_library:
    """Context manager: route every oracle call through another compiled variant."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _lib_handle()
        self.saved = _lib
        _lib = None
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    P, I = _p_dbl, _i64
    M = ctypes.POINTER(_Mech)
    ci = ctypes.c_int
    lib.or_max_threads.restype = ci
    lib.or_thermo.argtypes = [M, I, I, P, P, P, P, P, P, P, P, P, P, ci]
    lib.or_nasa7_cs.argtypes = [M, ci, I, P, P, P, P, P, P]
    lib.or_rates.argtypes = [M, I, I, P, P, P, P, P, P, P, P, ci]
    lib.or_rates_of_progress.argtypes = [M, I, I, P, P, P, P, P, P, ci]
    lib.or_transport.argtypes = [M, I, I, P, P, P, P, P, P, ci]
    lib.or_rates_jacobian.argtypes = [M, I, I, P, P, P, P, P, P, ci]
    lib.or_rates_jvp.argtypes = [M, I, I, P, P, P, P, P, P, P, P, P, P, ci]
    lib.or_rates_grad_lnA.argtypes = [M, I, I, P, P, P, P, P, P, P, ci]
    lib.or_count_ops.argtypes = [M, _c_dbl, _c_dbl, P, ci, P]
    lib.or_rhs.argtypes = [M, I, I, P, P, P, P, P, P, P, ci]
    lib.or_rhs_jacobian.argtypes = [M, I, I, P, P, P, P, P, ci]
    lib.or_rhs_jvp.argtypes = [M, I, I, P, P, P, P, P, P, P, P, P, ci]
    lib.or_diffusion.argtypes = [M, I, I, P, P, P, P, P, P, P, P, ci]
    lib.or_reactor_step.argtypes = [M, I, I, P, P, P, _c_dbl, _c_dbl, _c_dbl, P, P, ctypes.POINTER(ctypes.c_int), ci]
    for f in ("or_thermo", "or_nasa7_cs", "or_rates", "or_rates_of_progress", "or_transport",
              "or_rates_jacobian", "or_rates_jvp", "or_rates_grad_lnA", "or_count_ops", "or_rhs", "or_rhs_jacobian",
              "or_rhs_jvp", "or_diffusion", "or_reactor_step"):
        getattr(lib, f).restype = None
    return lib


def max_threads() -> int:
    return _lib_handle().or_max_threads()


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(_p_dbl)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class _Packed:
    """Keeps the contiguous copies alive while the C struct points into them."""

    def __init__(self, mech):
        K, R = int(mech.K), int(mech.R)
        self.keep = {}

        def f(name, dtype):
            arr = _f64(getattr(mech, name)) if dtype == "f" else _i32(getattr(mech, name))
            self.keep[name] = arr
            return arr.ctypes.data_as(_p_dbl if dtype == "f" else _p_i32)

        atoms = getattr(mech, "atoms")
        self.s = _Mech(
            K=K, R=R, n_elem=int(np.asarray(atoms).shape[1]),
            W=f("W", "f"), atoms=f("atoms", "i"), nasa_lo=f("nasa_lo", "f"), nasa_hi=f("nasa_hi", "f"),
            T_mid=f("T_mid", "f"), reac_ptr=f("reac_ptr", "i"), reac_sp=f("reac_sp", "i"),
            reac_nu=f("reac_nu", "i"), prod_ptr=f("prod_ptr", "i"), prod_sp=f("prod_sp", "i"),
            prod_nu=f("prod_nu", "i"), rtype=f("rtype", "i"), lnA=f("lnA", "f"), beta=f("beta", "f"),
            Ea=f("Ea", "f"), lnA0=f("lnA0", "f"), beta0=f("beta0", "f"), Ea0=f("Ea0", "f"),
            troe=f("troe", "f"), eff=f("eff", "f"), mu_fit=f("mu_fit", "f"), lam_fit=f("lam_fit", "f"),
            D_fit=f("D_fit", "f"), p_ref=float(mech.p_ref),
        )
        self.K, self.R = K, R

    def ptr(self):
        return ctypes.byref(self.s)


def _state(T, p, Y, K):
    T = _f64(T).ravel()
    n = T.shape[0]
    p = _f64(np.broadcast_to(np.asarray(p, dtype=np.float64), (n,)))
    Y = _f64(Y)
    if Y.shape != (K, n):
        raise ValueError(f"Y must be [K={K}, n={n}], got {Y.shape}")
    return T, p, Y, n


def thermo(mech, T, p, Y, threads: int = 0) -> dict:
    """Mixture (mass based) and species (molar) thermodynamic properties."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    out = {k: np.empty(n) for k in ("cp_mix", "h_mix", "Wbar", "rho")}
    for k in ("cp_k", "h_k", "g_k"):
        out[k] = np.empty((pk.K, n))
    _lib_handle().or_thermo(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(out["cp_mix"]), _dp(out["h_mix"]),
                            _dp(out["Wbar"]), _dp(out["rho"]), _dp(out["cp_k"]), _dp(out["h_k"]),
                            _dp(out["g_k"]), threads)
    return out


def nasa7_cs(mech, k: int, T) -> dict:
    """Species k: molar cp, h, s and complex-step dh/dT, ds/dT at temperatures T."""
    pk = _Packed(mech)
    T = _f64(T).ravel()
    n = T.shape[0]
    out = {key: np.empty(n) for key in ("cp", "h", "s", "dh_dT", "ds_dT")}
    _lib_handle().or_nasa7_cs(pk.ptr(), int(k), n, _dp(T), _dp(out["cp"]), _dp(out["h"]), _dp(out["s"]),
                              _dp(out["dh_dT"]), _dp(out["ds_dT"]))
    return out


def rates(mech, T, p, Y, dlnA=None, threads: int = 0, scales: bool = False):
    """(omega [K, n], hrr [n]) and, with ``scales``, the cancellation scales (omega_scale, hrr_scale)."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    d = None if dlnA is None else _f64(dlnA)
    omega = np.empty((pk.K, n))
    hrr = np.empty(n)
    osc = np.empty((pk.K, n)) if scales else None
    hsc = np.empty(n) if scales else None
    _lib_handle().or_rates(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(d), _dp(omega), _dp(hrr),
                           _dp(osc), _dp(hsc), threads)
    if scales:
        return omega, hrr, osc, hsc
    return omega, hrr


def rates_of_progress(mech, T, p, Y, dlnA=None, threads: int = 0):
    """Per-reaction forward and reverse terms, each [R, n]."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    d = None if dlnA is None else _f64(dlnA)
    fwd = np.empty((pk.R, n))
    rev = np.empty((pk.R, n))
    _lib_handle().or_rates_of_progress(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(d), _dp(fwd), _dp(rev),
                                       threads)
    return fwd, rev


def transport(mech, T, p, Y, threads: int = 0):
    """(mu [n], lambda [n], Dmix [K, n])."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    mu = np.empty(n)
    lam = np.empty(n)
    D = np.empty((pk.K, n))
    _lib_handle().or_transport(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(mu), _dp(lam), _dp(D), threads)
    return mu, lam, D


def jacobian(mech, T, p, Y, dlnA=None, threads: int = 0, scales: bool = False):
    """Dense complex-step Jacobian [n, K+1, K+1]: rows (omega_k, hrr), columns (T, Y_k); with
    ``scales`` also the per-entry magnitudes sum_r |nu_kr| (|d fwd_r/dx| + |d rev_r/dx|)."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    d = None if dlnA is None else _f64(dlnA)
    J = np.empty((n, pk.K + 1, pk.K + 1))
    Js = np.empty_like(J) if scales else None
    _lib_handle().or_rates_jacobian(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(d), _dp(J), _dp(Js), threads)
    return (J, Js) if scales else J


def jvp(mech, T, p, Y, vT, vY, dlnA=None, threads: int = 0, scales: bool = False):
    """Complex-step J v: (d_omega [K, n], d_hrr [n]) and, with ``scales``, the magnitudes
    sum_r |nu_kr| (|d fwd_r| + |d rev_r|) and the heat-release analogue."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    vT = _f64(vT).ravel()
    vY = _f64(vY)
    d = None if dlnA is None else _f64(dlnA)
    dw = np.empty((pk.K, n))
    dh = np.empty(n)
    dws = np.empty((pk.K, n)) if scales else None
    dhs = np.empty(n) if scales else None
    _lib_handle().or_rates_jvp(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(d), _dp(vT), _dp(vY), _dp(dw),
                               _dp(dh), _dp(dws), _dp(dhs), threads)
    if scales:
        return dw, dh, dws, dhs
    return dw, dh


def grad_lnA(mech, T, p, Y, wbar, hbar=None, dlnA=None, threads: int = 0):
    """d/d lnA_r of sum_points [sum_k wbar_k omega_k + hbar hrr], [R]."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    wbar = _f64(wbar)
    hb = None if hbar is None else _f64(hbar).ravel()
    d = None if dlnA is None else _f64(dlnA)
    g = np.empty(pk.R)
    _lib_handle().or_rates_grad_lnA(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(d), _dp(wbar), _dp(hb),
                                    _dp(g), threads)
    return g


def rhs(mech, T, p, Y, threads: int = 0, scales: bool = False):
    """Implicit-stage chemistry sources at fixed p (Eq. 1a-b): (fT [n] = hrr/(rho c_p),
    fY [K, n] = W_k omega_k/rho) and, with ``scales``, their cancellation scales."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    fT = np.empty(n)
    fY = np.empty((pk.K, n))
    sT = np.empty(n) if scales else None
    sY = np.empty((pk.K, n)) if scales else None
    _lib_handle().or_rhs(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(fT), _dp(fY), _dp(sT), _dp(sY), threads)
    return (fT, fY, sT, sY) if scales else (fT, fY)


def rhs_jvp(mech, T, p, Y, vT, vY, threads: int = 0, scales: bool = False):
    """Complex-step directional derivative of the sources along (vT, vY): (dfT [n], dfY [K, n])
    and, with ``scales``, the derivative magnitudes."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    vT = _f64(vT).ravel()
    vY = _f64(vY)
    dfT = np.empty(n)
    dfY = np.empty((pk.K, n))
    sT = np.empty(n) if scales else None
    sY = np.empty((pk.K, n)) if scales else None
    _lib_handle().or_rhs_jvp(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(vT), _dp(vY), _dp(dfT), _dp(dfY),
                             _dp(sT), _dp(sY), threads)
    return (dfT, dfY, sT, sY) if scales else (dfT, dfY)


def rhs_jacobian(mech, T, p, Y, threads: int = 0, scales: bool = False):
    """Dense complex-step Jacobian [n, K+1, K+1] of the sources: rows (fT, fY_k), columns
    (T, Y_j); with ``scales`` also the per-entry derivative magnitudes."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    J = np.empty((n, pk.K + 1, pk.K + 1))
    Js = np.empty_like(J) if scales else None
    _lib_handle().or_rhs_jacobian(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(J), _dp(Js), threads)
    return (J, Js) if scales else J


def diffusion(mech, T, p, Y, D, gradX, threads: int = 0):
    """Mixture-averaged diffusion fluxes of Eq. 2 from D [K, n] and grad X [3, K, n]:
    (j [3, K, n] = rho Y_k V_k, Vc [3, n], hf [3, n] = sum_k c_p,k j_k)."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    D = _f64(D)
    gradX = _f64(gradX)
    if D.shape != (pk.K, n) or gradX.shape != (3, pk.K, n):
        raise ValueError("D must be [K, n] and gradX [3, K, n]")
    j = np.empty((3, pk.K, n))
    Vc = np.empty((3, n))
    hf = np.empty((3, n))
    _lib_handle().or_diffusion(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), _dp(D), _dp(gradX), _dp(j), _dp(Vc),
                               _dp(hf), threads)
    return j, Vc, hf


def reactor_step(mech, T, p, Y, dt: float, atol_T: float = 1e-8, atol_Y: float = 1e-16, threads: int = 0):
    """One implicit Euler step of dt (s) of the homogeneous constant-pressure reactor at every
    point, by dense Newton: (T1 [n], Y1 [K, n], Newton iterations [n], negative if not
    converged)."""
    pk = _Packed(mech)
    T, p, Y, n = _state(T, p, Y, pk.K)
    T1 = np.empty(n)
    Y1 = np.empty((pk.K, n))
    it = np.empty(n, dtype=np.intc)
    _lib_handle().or_reactor_step(pk.ptr(), n, n, _dp(T), _dp(p), _dp(Y), float(dt), float(atol_T), float(atol_Y),
                                  _dp(T1), _dp(Y1), it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), threads)
    return T1, Y1, it


def count_ops(mech, T: float, p: float, Y, which: str = "rates") -> dict:
    """Operations the definition performs at one point (add, mul, div, exp, log, pow, sqrt)."""
    pk = _Packed(mech)
    y = _f64(Y).ravel()
    c = np.zeros(7)
    _lib_handle().or_count_ops(pk.ptr(), float(T), float(p), _dp(y), 0 if which == "rates" else 1, _dp(c))
    return dict(zip(("add", "mul", "div", "exp", "log", "pow", "sqrt"), c.tolist()))
