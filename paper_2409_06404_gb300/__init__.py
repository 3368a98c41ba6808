"""Pointwise thermochemistry for spectral-element reacting-flow solvers on GB300.

Python binding of libnkchem.so (C ABI in include/nkchem.h): argument marshalling only.
Every computation runs in the library's CUDA kernels; there is no CPU fallback, and every
function raises if the library is not built or a call fails.

PyTorch provides device memory and streams: state arrays are CUDA float64 tensors,
T and p of shape [n], Y of shape [K, n] (species rows; a row stride ld >= n is allowed,
e.g. a column slice of a larger [K, N] field, and the outputs then use the same stride).
Calls are enqueued on the current torch CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "NkError", "Mechanism", "mechanism_load", "thermo_eval", "rates_eval", "transport_eval",
    "rates_jvp", "rates_vjp", "rates_vjp_workspace", "RatesFn", "rates", "library_path", "lib",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libnkchem.so")
_lock = threading.Lock()
_lib = None

NK_FP64, NK_MIXED, NK_FP64_NATIVE, NK_JIT = 0, 1, 2, 3
_PRECISION = {"fp64": NK_FP64, "mixed": NK_MIXED, "fp64_native": NK_FP64_NATIVE, "jit": NK_JIT,
              NK_FP64: NK_FP64, NK_MIXED: NK_MIXED, NK_FP64_NATIVE: NK_FP64_NATIVE, NK_JIT: NK_JIT}
_STATUS = {0: "NK_OK", 1: "NK_EINVAL", 2: "NK_EALIGN", 3: "NK_ECUDA", 4: "NK_ENOMEM", 5: "NK_EUNSUPPORTED"}

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_p_i32 = ctypes.POINTER(ctypes.c_int32)
_p_dbl = ctypes.POINTER(ctypes.c_double)


class NkError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _Desc(ctypes.Structure):
    """Mirror of nk_mech_desc."""
    _fields_ = [
        ("K", _i32), ("R", _i32), ("n_elem", _i32),
        ("W", _p_dbl), ("atoms", _p_i32), ("nasa_lo", _p_dbl), ("nasa_hi", _p_dbl), ("T_mid", _p_dbl),
        ("reac_ptr", _p_i32), ("reac_sp", _p_i32), ("reac_nu", _p_i32),
        ("prod_ptr", _p_i32), ("prod_sp", _p_i32), ("prod_nu", _p_i32),
        ("rtype", _p_i32), ("lnA", _p_dbl), ("beta", _p_dbl), ("Ea", _p_dbl),
        ("lnA0", _p_dbl), ("beta0", _p_dbl), ("Ea0", _p_dbl), ("troe", _p_dbl), ("eff", _p_dbl),
        ("mu_fit", _p_dbl), ("lam_fit", _p_dbl), ("D_fit", _p_dbl), ("p_ref", ctypes.c_double),
    ]


class _ReactorOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol_T", ctypes.c_double), ("atol_Y", ctypes.c_double),
                ("newton_tol", ctypes.c_double), ("lin_tol", ctypes.c_double), ("max_newton", _i32),
                ("krylov_dim", _i32), ("precond", _i32), ("linearized", _i32)]


class _ReactorStats(ctypes.Structure):
    _fields_ = [("converged", _i32), ("newton_iters", _i32), ("krylov_iters", _i32),
                ("update_wrms", ctypes.c_double), ("residual_wrms", ctypes.c_double)]


_SIGS = {
    "nk_version": (_i32, []),
    "nk_last_error": (ctypes.c_char_p, []),
    "nk_mechanism_load": (ctypes.c_int, [ctypes.POINTER(_Desc), ctypes.POINTER(_vp)]),
    "nk_mechanism_free": (ctypes.c_int, [_vp]),
    "nk_mechanism_info": (ctypes.c_int, [_vp, _p_i32, _p_i32]),
    "nk_thermo_eval": (ctypes.c_int, [_vp, _i64, _i64] + [_vp] * 10 + [_vp]),
    "nk_rates_eval": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nk_transport_eval": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nk_rates_jvp": (ctypes.c_int, [_vp, _i64, _i64] + [_vp] * 10 + [_vp]),
    "nk_diffusion_fluxes": (ctypes.c_int, [_vp, _i64, _i64] + [_vp] * 8 + [_vp]),
    "nk_reactor_workspace": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(_ReactorOpts), ctypes.POINTER(ctypes.c_size_t)]),
    "nk_rhs_jvp_linearized": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64] + [_vp] * 6 + [_vp]),
    "nk_mechanism_jit": (ctypes.c_int, [_vp]),
    "nk_host_eval_workspace": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(ctypes.c_size_t)]),
    "nk_host_eval": (ctypes.c_int, [_vp, _i64] + [_vp] * 8 + [ctypes.c_int, _i64, _vp, ctypes.c_size_t, _vp]),
    "nk_jit_source": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_size_t)]),
    "nk_rhs_jacobian": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _vp]),
    "nk_block_jacobi_factor": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64,
                                              ctypes.c_double, _vp, _vp, _i64, _vp]),
    "nk_block_jacobi_apply": (ctypes.c_int, [_vp, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "nk_reactor_step": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(_ReactorOpts),
                                       ctypes.POINTER(_ReactorStats), _vp, ctypes.c_size_t, _vp]),
    "nk_rhs_eval": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nk_rhs_jvp": (ctypes.c_int, [_vp, _i64, _i64] + [_vp] * 10 + [_vp]),
    "nk_rates_linearization_slots": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "nk_rates_linearize": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp]),
    "nk_rates_linearize_f32": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp]),
    "nk_rates_linearization_slots_f32": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "nk_rates_jvp_linearized_f32": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                                                   _vp]),
    "nk_rhs_jvp_linearized_f32": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64] + [_vp] * 6 + [_vp]),
    "nk_rates_jvp_linearized": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                                               _vp]),
    "nk_rates_linearization_slots_compact": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "nk_rates_linearize_compact": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "nk_rates_jvp_linearized_compact": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp,
                                                       _vp, _vp]),
    "nk_rhs_jvp_linearized_compact": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64] + [_vp] * 6 + [_vp]),
    "nk_rates_vjp_workspace": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(ctypes.c_size_t)]),
    "nk_rates_vjp": (ctypes.c_int, [_vp, _i64, _i64] + [_vp] * 10 + [ctypes.c_size_t, _vp]),
    "nk_rates_vjp_noalloc": (ctypes.c_int, [_vp, _i64, _i64] + [_vp] * 9 + [_vp]),
}


def library_path() -> str:
    return _LIB_PATH


def lib():
    """The loaded libnkchem.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                                   "`python -m paper_2409_06404_gb300.build`")
            L = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise NkError(status, lib().nk_last_error().decode())


# ------------------------------------------------------------------------------ mechanism
def _desc_from(mech):
    import numpy as np

    keep = []

    def f(name):
        a = np.ascontiguousarray(np.asarray(getattr(mech, name), dtype=np.float64))
        keep.append(a)
        return a.ctypes.data_as(_p_dbl)

    def i(name):
        a = np.ascontiguousarray(np.asarray(getattr(mech, name), dtype=np.int32))
        keep.append(a)
        return a.ctypes.data_as(_p_i32)

    atoms = np.asarray(mech.atoms)
    d = _Desc(K=int(mech.K), R=int(mech.R), n_elem=int(atoms.shape[1]), W=f("W"), atoms=i("atoms"),
              nasa_lo=f("nasa_lo"), nasa_hi=f("nasa_hi"), T_mid=f("T_mid"), reac_ptr=i("reac_ptr"),
              reac_sp=i("reac_sp"), reac_nu=i("reac_nu"), prod_ptr=i("prod_ptr"), prod_sp=i("prod_sp"),
              prod_nu=i("prod_nu"), rtype=i("rtype"), lnA=f("lnA"), beta=f("beta"), Ea=f("Ea"),
              lnA0=f("lnA0"), beta0=f("beta0"), Ea0=f("Ea0"), troe=f("troe"), eff=f("eff"),
              mu_fit=f("mu_fit"), lam_fit=f("lam_fit"), D_fit=f("D_fit"), p_ref=float(mech.p_ref))
    return d, keep


class Mechanism:
    """A mechanism loaded on the current CUDA device (nk_mechanism_load)."""

    def __init__(self, mech):
        d, keep = _desc_from(mech)
        h = _vp()
        _check(lib().nk_mechanism_load(ctypes.byref(d), ctypes.byref(h)))
        del keep
        self._h = h
        K, R = _i32(), _i32()
        _check(lib().nk_mechanism_info(h, ctypes.byref(K), ctypes.byref(R)))
        self.K, self.R = K.value, R.value

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("mechanism has been freed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(lib().nk_mechanism_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mechanism_load(mech) -> Mechanism:
    return Mechanism(mech)


def mechanism_jit(m: Mechanism) -> None:
    """nk_mechanism_jit: compile the mechanism-specialised rates kernel (precision "jit") now."""
    _check(lib().nk_mechanism_jit(m.handle))


def jit_source(mech) -> str:
    """nk_jit_source: the CUDA source the library generates for a mechanism (host only)."""
    d, keep = _desc_from(mech)
    n = ctypes.c_size_t(0)
    lib().nk_jit_source(ctypes.byref(d), None, ctypes.byref(n))     # the size, then the text
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().nk_jit_source(ctypes.byref(d), buf, ctypes.byref(n)))
    del keep
    return buf.value.decode()


# ------------------------------------------------------------------------------ helpers
def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _state(m, T, p, Y):
    torch = _torch()
    for name, t in (("T", T), ("p", p), ("Y", Y)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
            raise TypeError(f"{name} must be a CUDA float64 tensor")
    if T.dim() != 1 or not T.is_contiguous():
        raise ValueError("T must be a contiguous 1-D tensor")
    n = T.shape[0]
    if p.shape != (n,) or not p.is_contiguous():
        raise ValueError("p must be a contiguous tensor of shape [n]")
    if Y.dim() != 2 or tuple(Y.shape) != (m.K, n) or (n > 1 and Y.stride(1) != 1):
        raise ValueError(f"Y must be [K={m.K}, n={n}] with unit stride along points")
    ld = max(Y.stride(0), n) if (n > 0 and m.K > 1) else n
    return n, ld


def _rows_ok(t, n, ld, K):
    """[K, n] with unit stride along points and row stride ld (strides of size-1 dims are free)."""
    return (n <= 1 or t.stride(1) == 1) and (K <= 1 or n == 0 or t.stride(0) == ld)


def _species_out(m, n, ld, like, out=None):
    torch = _torch()
    if out is not None:
        if tuple(out.shape) != (m.K, n) or out.dtype != torch.float64 or not _rows_ok(out, n, ld, m.K):
            raise ValueError("species output must be [K, n] float64 with the row stride of Y")
        return out
    if ld == n:
        return torch.empty((m.K, n), dtype=torch.float64, device=like.device)
    return torch.empty((m.K, ld), dtype=torch.float64, device=like.device)[:, :n]


def _point_out(n, like, out=None):
    torch = _torch()
    return out if out is not None else torch.empty(n, dtype=torch.float64, device=like.device)


def _vec(v, n, name):
    torch = _torch()
    if v is None:
        return None
    if not isinstance(v, torch.Tensor) or not v.is_cuda or v.dtype != torch.float64 or v.shape != (n,) \
            or not v.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape [{n}]")
    return v


def _species_in(m, v, n, ld, name):
    torch = _torch()
    if not isinstance(v, torch.Tensor) or not v.is_cuda or v.dtype != torch.float64 \
            or tuple(v.shape) != (m.K, n) or not _rows_ok(v, n, ld, m.K):
        raise ValueError(f"{name} must be a CUDA float64 [K, n] tensor with the row stride of Y")
    return v


# ------------------------------------------------------------------------------ entry points
def thermo_eval(m: Mechanism, T, p, Y, species: bool = True, stream=None) -> dict:
    """nk_thermo_eval: mixture cp, h (mass based), Wbar, rho and species cp_k, h_k, g_k (molar)."""
    n, ld = _state(m, T, p, Y)
    out = {k: _point_out(n, T) for k in ("cp_mix", "h_mix", "Wbar", "rho")}
    if species:
        for k in ("cp_k", "h_k", "g_k"):
            out[k] = _species_out(m, n, ld, T)
    _check(lib().nk_thermo_eval(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(out["cp_mix"]),
                                _ptr(out["h_mix"]), _ptr(out["Wbar"]), _ptr(out["rho"]), _ptr(out.get("cp_k")),
                                _ptr(out.get("h_k")), _ptr(out.get("g_k")), _stream(stream)))
    return out


def rates_eval(m: Mechanism, T, p, Y, dlnA=None, precision="fp64", omega=None, hrr=None, stream=None):
    """nk_rates_eval: (omega [K, n] mol/m^3/s, hrr [n] W/m^3)."""
    n, ld = _state(m, T, p, Y)
    _vec(dlnA, m.R, "dlnA")
    omega = _species_out(m, n, ld, T, omega)
    hrr = _point_out(n, T, hrr)
    _check(lib().nk_rates_eval(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(omega), _ptr(hrr),
                               _PRECISION[precision], _stream(stream)))
    return omega, hrr


def host_eval_workspace(m: Mechanism, chunk: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().nk_host_eval_workspace(m.handle, int(chunk), ctypes.byref(b)))
    return b.value


def host_eval(m: Mechanism, T, p, Y, precision="fp64", chunk=65536, workspace=None, outputs=None, stream=None):
    """nk_host_eval: rates and transport of host-resident CPU tensors (float64, contiguous; T, p [n],
    Y [K, n]), chunked over streams.  Returns the host outputs (omega, hrr, mu, lambda, Dmix);
    pass page-locked tensors (and preallocated ``outputs``) for asynchronous copies."""
    import torch
    for name, t in (("T", T), ("p", p), ("Y", Y)):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous host float64 tensor")
    n = T.shape[0]
    if p.shape != (n,) or Y.shape != (m.K, n):
        raise ValueError("T, p must be [n] and Y [K, n]")
    if outputs is None:
        pin = T.is_pinned()
        mk = (lambda *s: torch.empty(*s, dtype=torch.float64, pin_memory=pin))
        outputs = (mk(m.K, n), mk(n), mk(n), mk(n), mk(m.K, n))
    if workspace is None and n > 0:
        workspace = torch.empty(host_eval_workspace(m, min(chunk, n)), dtype=torch.uint8, device="cuda")
    _check(lib().nk_host_eval(m.handle, n, _ptr(T), _ptr(p), _ptr(Y), *[_ptr(o) for o in outputs],
                              _PRECISION[precision], int(chunk), _ptr(workspace),
                              0 if workspace is None else workspace.numel(), _stream(stream)))
    return outputs


def transport_eval(m: Mechanism, T, p, Y, precision="fp64", mu=None, lam=None, Dmix=None, stream=None):
    """nk_transport_eval: (mu [n] Pa s, lambda [n] W/m/K, Dmix [K, n] m^2/s)."""
    n, ld = _state(m, T, p, Y)
    mu = _point_out(n, T, mu)
    lam = _point_out(n, T, lam)
    Dmix = _species_out(m, n, ld, T, Dmix)
    _check(lib().nk_transport_eval(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(mu), _ptr(lam), _ptr(Dmix),
                                   _PRECISION[precision], _stream(stream)))
    return mu, lam, Dmix


def rates_jvp(m: Mechanism, T, p, Y, vT, vY, dlnA=None, primal=False, stream=None):
    """nk_rates_jvp: (d_omega, d_hrr) = J (vT, vY); with primal=True also (omega, hrr)."""
    n, ld = _state(m, T, p, Y)
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    _vec(dlnA, m.R, "dlnA")
    d_omega = _species_out(m, n, ld, T)
    d_hrr = _point_out(n, T)
    omega = _species_out(m, n, ld, T) if primal else None
    hrr = _point_out(n, T) if primal else None
    _check(lib().nk_rates_jvp(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(vT), _ptr(vY),
                              _ptr(omega), _ptr(hrr), _ptr(d_omega), _ptr(d_hrr), _stream(stream)))
    if primal:
        return d_omega, d_hrr, omega, hrr
    return d_omega, d_hrr


def diffusion_fluxes(m: Mechanism, T, p, Y, Dmix, gradX, want_vc=True, want_hf=True, stream=None):
    """nk_diffusion_fluxes: (j [3, K, n], Vc [3, n] or None, hf [3, n] or None) from the
    mixture-averaged D_k [K, n] and mole-fraction gradients [3, K, n]."""
    import torch
    n, ld = _state(m, T, p, Y)
    for name, a, shape in (("Dmix", Dmix, (m.K, n)), ("gradX", gradX, (3, m.K, n))):
        if tuple(a.shape) != shape or not a.is_contiguous() or a.dtype != torch.float64 or a.device != T.device:
            raise ValueError(f"{name} must be a contiguous float64 {shape} tensor on the state's device")
    if ld != n:
        raise ValueError("diffusion_fluxes takes contiguous states (ld = n)")
    j = torch.empty((3, m.K, n), dtype=torch.float64, device=T.device)
    Vc = torch.empty((3, n), dtype=torch.float64, device=T.device) if want_vc else None
    hf = torch.empty((3, n), dtype=torch.float64, device=T.device) if want_hf else None
    _check(lib().nk_diffusion_fluxes(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(Dmix), _ptr(gradX), _ptr(j),
                                     _ptr(Vc), _ptr(hf), _stream(stream)))
    return j, Vc, hf


def reactor_opts(rtol=1e-6, atol_T=1e-6, atol_Y=1e-14, newton_tol=0.1, lin_tol=1e-3, max_newton=10,
                 krylov_dim=20, precond=0, linearized=0) -> _ReactorOpts:
    """Options of nk_reactor_step (weighted RMS tolerances; precond 1 = per-point block Jacobi
    made at x0, 2 = its factors from the last call reused; linearized 1 = GMRES products from a
    stored linearization per Newton iteration, 2 = the same rounded to float with
    single-precision products; see include/nkchem.h)."""
    return _ReactorOpts(rtol, atol_T, atol_Y, newton_tol, lin_tol, max_newton, krylov_dim, precond, linearized)


def reactor_workspace(m: Mechanism, n: int, krylov_dim: int = 20, precond: int = 0, linearized: int = 0) -> int:
    b = ctypes.c_size_t()
    o = reactor_opts(krylov_dim=krylov_dim, precond=precond, linearized=linearized)
    _check(lib().nk_reactor_workspace(m.handle, int(n), ctypes.byref(o), ctypes.byref(b)))
    return b.value


def reactor_step(m: Mechanism, T, p, Y, dt: float, opts: _ReactorOpts = None, workspace=None, stream=None) -> dict:
    """nk_reactor_step: one implicit Euler step of dt at every point, in place on T [n] and the
    contiguous Y [K, n]; returns the solver statistics."""
    import torch
    n, ld = _state(m, T, p, Y)
    if ld != n:
        raise ValueError("reactor_step takes a contiguous Y [K, n]")
    opts = opts or reactor_opts()
    if workspace is None and n > 0 and 1 <= opts.krylov_dim <= 30 and opts.precond in (0, 1, 2) \
            and opts.linearized in (0, 1, 2):
        workspace = torch.empty(reactor_workspace(m, n, opts.krylov_dim, opts.precond, opts.linearized),
                                dtype=torch.uint8, device=T.device)
    st = _ReactorStats()
    _check(lib().nk_reactor_step(m.handle, n, _ptr(T), _ptr(p), _ptr(Y), float(dt), ctypes.byref(opts),
                                 ctypes.byref(st), _ptr(workspace), 0 if workspace is None else workspace.numel(),
                                 _stream(stream)))
    return {f: getattr(st, f) for f, _ in _ReactorStats._fields_}


def rhs_eval(m: Mechanism, T, p, Y, dlnA=None, precision="fp64", fT=None, fY=None, stream=None):
    """nk_rhs_eval: implicit-stage chemistry sources (fT [n] = dT/dt in K/s, fY [K, n] = dY/dt
    in 1/s) at fixed p."""
    n, ld = _state(m, T, p, Y)
    _vec(dlnA, m.R, "dlnA")
    fY = _species_out(m, n, ld, T, fY)
    fT = _point_out(n, T, fT)
    _check(lib().nk_rhs_eval(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(fT), _ptr(fY),
                             _PRECISION[precision], _stream(stream)))
    return fT, fY


def rhs_jvp(m: Mechanism, T, p, Y, vT, vY, dlnA=None, primal=False, stream=None):
    """nk_rhs_jvp: (dfT, dfY) = J_f (vT, vY) of the sources; with primal=True also (fT, fY)."""
    n, ld = _state(m, T, p, Y)
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    _vec(dlnA, m.R, "dlnA")
    dfY = _species_out(m, n, ld, T)
    dfT = _point_out(n, T)
    fY = _species_out(m, n, ld, T) if primal else None
    fT = _point_out(n, T) if primal else None
    _check(lib().nk_rhs_jvp(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(vT), _ptr(vY),
                            _ptr(fT), _ptr(fY), _ptr(dfT), _ptr(dfY), _stream(stream)))
    if primal:
        return dfT, dfY, fT, fY
    return dfT, dfY


def rhs_jvp_linearized(m: Mechanism, T, p, Y, lin, fT, fY, vT, vY, stream=None):
    """nk_rhs_jvp_linearized: (dfT, dfY) = J_f (vT, vY) from a stored linearization and the
    sources at the same state."""
    n, ld = _state(m, T, p, Y)
    _check_lin(m, lin, n)
    _vec(fT, n, "fT")
    _species_in(m, fY, n, ld, "fY")
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    dfY = _species_out(m, n, ld, T)
    dfT = _point_out(n, T)
    _check(lib().nk_rhs_jvp_linearized(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin), lin.stride(0),
                                       _ptr(fT), _ptr(fY), _ptr(vT), _ptr(vY), _ptr(dfT), _ptr(dfY), _stream(stream)))
    return dfT, dfY


def linearization_slots(m: Mechanism) -> int:
    """Doubles per point of a stored rates linearization."""
    v = _i64()
    _check(lib().nk_rates_linearization_slots(m.handle, ctypes.byref(v)))
    return v.value


def rates_linearize(m: Mechanism, T, p, Y, dlnA=None, lin=None, stream=None):
    """nk_rates_linearize: the state-only data of the rates JVP at (T, p, Y), a device tensor
    [slots, n] to pass to rates_jvp_linearized with the same state."""
    import torch
    n, ld = _state(m, T, p, Y)
    _vec(dlnA, m.R, "dlnA")
    if lin is None:
        lin = torch.empty((linearization_slots(m), max(n, 1)), dtype=torch.float64, device=T.device)
    _check(lib().nk_rates_linearize(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(lin),
                                    lin.stride(0), _stream(stream)))
    return lin


def rates_jvp_linearized(m: Mechanism, T, p, Y, lin, vT, vY, stream=None):
    """nk_rates_jvp_linearized: (d_omega, d_hrr) = J (vT, vY) from a stored linearization."""
    n, ld = _state(m, T, p, Y)
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    if lin.dim() != 2 or lin.shape[0] != linearization_slots(m) or lin.stride(1) != 1 or lin.shape[1] < n:
        raise ValueError("lin must be a [slots, >= n] row-major tensor from rates_linearize")
    d_omega = _species_out(m, n, ld, T)
    d_hrr = _point_out(n, T)
    _check(lib().nk_rates_jvp_linearized(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin), lin.stride(0),
                                         _ptr(vT), _ptr(vY), _ptr(d_omega), _ptr(d_hrr), _stream(stream)))
    return d_omega, d_hrr


def linearization_slots_compact(m: Mechanism) -> int:
    """Doubles per point of the per-reaction (compact) rates linearization."""
    v = _i64()
    _check(lib().nk_rates_linearization_slots_compact(m.handle, ctypes.byref(v)))
    return v.value


def rates_linearize_compact(m: Mechanism, T, p, Y, dlnA=None, lin=None, primal=False, stream=None):
    """nk_rates_linearize_compact: the per-reaction linearization at (T, p, Y), a device tensor
    [slots_compact, n]; with primal=True also (omega, hrr) at the state from the same pass:
    returns (lin, omega, hrr)."""
    import torch
    n, ld = _state(m, T, p, Y)
    _vec(dlnA, m.R, "dlnA")
    if lin is None:
        lin = torch.empty((linearization_slots_compact(m), max(n, 1)), dtype=torch.float64, device=T.device)
    _check_lin(m, lin, n, compact=True)
    omega = _species_out(m, n, ld, T) if primal else None
    hrr = _point_out(n, T) if primal else None
    _check(lib().nk_rates_linearize_compact(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(lin),
                                            lin.stride(0), _ptr(omega), _ptr(hrr), _stream(stream)))
    return (lin, omega, hrr) if primal else lin


def rates_jvp_linearized_compact(m: Mechanism, T, p, Y, lin, vT, vY, stream=None):
    """nk_rates_jvp_linearized_compact: (d_omega, d_hrr) = J (vT, vY) from rates_linearize_compact."""
    n, ld = _state(m, T, p, Y)
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    _check_lin(m, lin, n, compact=True)
    d_omega = _species_out(m, n, ld, T)
    d_hrr = _point_out(n, T)
    _check(lib().nk_rates_jvp_linearized_compact(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin),
                                                 lin.stride(0), _ptr(vT), _ptr(vY), _ptr(d_omega), _ptr(d_hrr),
                                                 _stream(stream)))
    return d_omega, d_hrr


def rhs_jvp_linearized_compact(m: Mechanism, T, p, Y, lin, fT, fY, vT, vY, stream=None):
    """nk_rhs_jvp_linearized_compact: (dfT, dfY) = J_f (vT, vY) from rates_linearize_compact and the
    sources at the same state."""
    n, ld = _state(m, T, p, Y)
    _check_lin(m, lin, n, compact=True)
    _vec(fT, n, "fT")
    _species_in(m, fY, n, ld, "fY")
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    dfY = _species_out(m, n, ld, T)
    dfT = _point_out(n, T)
    _check(lib().nk_rhs_jvp_linearized_compact(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin),
                                               lin.stride(0), _ptr(fT), _ptr(fY), _ptr(vT), _ptr(vY), _ptr(dfT),
                                               _ptr(dfY), _stream(stream)))
    return dfT, dfY


def linearization_slots_f32(m: Mechanism) -> int:
    """32-bit words per point of the single-precision rates linearization."""
    v = _i64()
    _check(lib().nk_rates_linearization_slots_f32(m.handle, ctypes.byref(v)))
    return v.value


def rates_linearize_f32(m: Mechanism, T, p, Y, dlnA=None, lin=None, stream=None):
    """nk_rates_linearize_f32: the rates linearization in single precision (per-reaction power-
    of-two scales), a device float32 tensor [slots_f32, n] for the single-precision products."""
    import torch
    n, ld = _state(m, T, p, Y)
    _vec(dlnA, m.R, "dlnA")
    if lin is None:
        lin = torch.empty((linearization_slots_f32(m), max(n, 1)), dtype=torch.float32, device=T.device)
    _check_lin(m, lin, n, torch.float32)
    _check(lib().nk_rates_linearize_f32(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(lin),
                                        lin.stride(0), _stream(stream)))
    return lin


def rates_jvp_linearized_f32(m: Mechanism, T, p, Y, lin, vT, vY, stream=None):
    """nk_rates_jvp_linearized_f32: (d_omega, d_hrr) = J (vT, vY) in single precision from
    rates_linearize_f32 (results in float64 tensors)."""
    import torch
    n, ld = _state(m, T, p, Y)
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    _check_lin(m, lin, n, torch.float32)
    d_omega = _species_out(m, n, ld, T)
    d_hrr = _point_out(n, T)
    _check(lib().nk_rates_jvp_linearized_f32(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin), lin.stride(0),
                                             _ptr(vT), _ptr(vY), _ptr(d_omega), _ptr(d_hrr), _stream(stream)))
    return d_omega, d_hrr


def rhs_jvp_linearized_f32(m: Mechanism, T, p, Y, lin, fT, fY, vT, vY, stream=None):
    """nk_rhs_jvp_linearized_f32: (dfT, dfY) = J_f (vT, vY) in single precision from
    rates_linearize_f32 and the sources at the same state."""
    import torch
    n, ld = _state(m, T, p, Y)
    _check_lin(m, lin, n, torch.float32)
    _vec(fT, n, "fT")
    _species_in(m, fY, n, ld, "fY")
    _vec(vT, n, "vT")
    _species_in(m, vY, n, ld, "vY")
    dfY = _species_out(m, n, ld, T)
    dfT = _point_out(n, T)
    _check(lib().nk_rhs_jvp_linearized_f32(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin), lin.stride(0),
                                           _ptr(fT), _ptr(fY), _ptr(vT), _ptr(vY), _ptr(dfT), _ptr(dfY),
                                           _stream(stream)))
    return dfT, dfY


def rhs_jacobian(m: Mechanism, T, p, Y, lin, fT, fY, stream=None):
    """nk_rhs_jacobian: the dense Jacobian [K+1, K+1, n] of the sources (rows fT, fY_k; columns
    T, Y_j) from a stored linearization (rates_linearize) and the sources (rhs_eval, fp64) at
    the same state."""
    import torch
    n, ld = _state(m, T, p, Y)
    _check_lin(m, lin, n)
    _vec(fT, n, "fT")
    _species_in(m, fY, n, ld, "fY")
    N = m.K + 1
    J = torch.empty((N, N, max(n, 1)), dtype=torch.float64, device=T.device)
    _check(lib().nk_rhs_jacobian(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin), lin.stride(0), _ptr(fT),
                                 _ptr(fY), _ptr(J), J.stride(1), _stream(stream)))
    return J[:, :, :n]


def block_jacobi_factor(m: Mechanism, T, p, Y, lin, fT, fY, w, dt: float, stream=None):
    """nk_block_jacobi_factor: LU factors (float64 [K+1, K+1, n], pivot order) of the row-scaled
    per-point blocks I - dt diag(w) J diag(1/w), w [K+1, n] (row 0 for T), and the pivot words
    (int32 [K+1, n]: row index | row exponent << 16)."""
    import torch
    n, ld = _state(m, T, p, Y)
    _check_lin(m, lin, n)
    _vec(fT, n, "fT")
    _species_in(m, fY, n, ld, "fY")
    N = m.K + 1
    if w.dtype != torch.float64 or w.dim() != 2 or w.shape[0] != N or w.shape[1] < n or w.stride(1) != 1:
        raise ValueError("w must be a float64 [K+1, >= n] row-major tensor")
    F = torch.empty((N, N, max(n, 1)), dtype=torch.float64, device=T.device)
    piv = torch.empty((N, max(n, 1)), dtype=torch.int32, device=T.device)
    _check(lib().nk_block_jacobi_factor(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(lin), lin.stride(0),
                                        _ptr(fT), _ptr(fY), _ptr(w), w.stride(0), float(dt), _ptr(F), _ptr(piv),
                                        F.stride(1), _stream(stream)))
    return F[:, :, :n], piv[:, :n]


def block_jacobi_apply(m: Mechanism, F, piv, v, stream=None):
    """nk_block_jacobi_apply: z = P^-1 v per point for float64 v [K+1, n]."""
    import torch
    N = m.K + 1
    if F.dtype != torch.float64 or F.dim() != 3 or F.shape[:2] != (N, N) or F.stride(2) != 1:
        raise ValueError("F must be float64 [K+1, K+1, n] from block_jacobi_factor")
    n = F.shape[2]
    if piv.dtype != torch.int32 or piv.shape != (N, n) or piv.stride(0) != F.stride(1):
        raise ValueError("piv must be the int32 [K+1, n] tensor from the same block_jacobi_factor call")
    if v.dtype != torch.float64 or v.shape != (N, n) or v.stride(1) != 1:
        raise ValueError("v must be a float64 [K+1, n] row-major tensor")
    z = torch.empty_like(v)
    _check(lib().nk_block_jacobi_apply(m.handle, n, _ptr(F), _ptr(piv), F.stride(1), _ptr(v), v.stride(0),
                                       _ptr(z), z.stride(0), _stream(stream)))
    return z


def _check_lin(m, lin, n, dtype=None, compact=False):
    import torch
    dtype = dtype or torch.float64
    if compact:
        slots = linearization_slots_compact(m)
    else:
        slots = linearization_slots(m) if dtype == torch.float64 else linearization_slots_f32(m)
    if lin.dtype != dtype:
        raise ValueError(f"lin must be {dtype}, got {lin.dtype}")
    if lin.dim() != 2 or lin.shape[0] != slots or lin.stride(1) != 1 or lin.shape[1] < n:
        raise ValueError("lin must be a [slots, >= n] row-major tensor from rates_linearize(_f32)")


def rates_vjp_workspace(m: Mechanism, n: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().nk_rates_vjp_workspace(m.handle, int(n), ctypes.byref(b)))
    return b.value


def rates_vjp(m: Mechanism, T, p, Y, bar_omega, bar_hrr=None, dlnA=None, want_lnA=True, workspace=None,
              stream=None):
    """nk_rates_vjp: (gT [n], gY [K, n], g_lnA [R] or None) = J^T (bar_omega, bar_hrr)."""
    torch = _torch()
    n, ld = _state(m, T, p, Y)
    _species_in(m, bar_omega, n, ld, "bar_omega")
    _vec(bar_hrr, n, "bar_hrr")
    _vec(dlnA, m.R, "dlnA")
    gT = _point_out(n, T)
    gY = _species_out(m, n, ld, T)
    g = torch.empty(m.R, dtype=torch.float64, device=T.device) if want_lnA else None
    nbytes = rates_vjp_workspace(m, n) if want_lnA else 0
    if want_lnA and (workspace is None or workspace.numel() * workspace.element_size() < nbytes):
        workspace = torch.empty(max(nbytes, 8), dtype=torch.uint8, device=T.device)
    _check(lib().nk_rates_vjp(m.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(dlnA), _ptr(bar_omega),
                              _ptr(bar_hrr), _ptr(gT), _ptr(gY), _ptr(g), _ptr(workspace) if want_lnA else None,
                              nbytes, _stream(stream)))
    return gT, gY, g


# ------------------------------------------------------------------------------ autograd
def _make_rates_fn():
    torch = _torch()

    class RatesFn(torch.autograd.Function):
        """(omega, hrr) = rates(T, p, Y, dlnA) with the hand-written VJP as backward and the
        hand-written JVP as forward-mode derivative.  p is not differentiated."""

        @staticmethod
        def forward(ctx, mech, T, p, Y, dlnA):
            omega, hrr = rates_eval(mech, T, p, Y, dlnA)
            ctx.mech = mech
            ctx.save_for_backward(T, p, Y, dlnA)
            ctx.save_for_forward(T, p, Y, dlnA)
            return omega, hrr

        @staticmethod
        def backward(ctx, bar_omega, bar_hrr):
            T, p, Y, dlnA = ctx.saved_tensors
            if bar_omega is None:
                bar_omega = torch.zeros_like(Y)
            bar_omega = bar_omega.contiguous()
            bar_hrr = None if bar_hrr is None else bar_hrr.contiguous()
            want = ctx.needs_input_grad[4]
            gT, gY, g = rates_vjp(ctx.mech, T, p, Y.contiguous(), bar_omega, bar_hrr, dlnA, want_lnA=want)
            return None, gT, None, gY, g

        @staticmethod
        def jvp(ctx, _m, tT, _tp, tY, tA):
            T, p, Y, dlnA = ctx.saved_tensors
            if tA is not None and bool(torch.any(tA != 0)):
                raise NotImplementedError("forward-mode derivative with respect to dlnA is not provided")
            tT = torch.zeros_like(T) if tT is None else tT.contiguous()
            tY = torch.zeros_like(Y) if tY is None else tY.contiguous()
            d_omega, d_hrr = rates_jvp(ctx.mech, T, p, Y.contiguous(), tT, tY, dlnA)
            return d_omega, d_hrr

    return RatesFn


_RatesFn = None


def __getattr__(name):
    global _RatesFn
    if name == "RatesFn":
        if _RatesFn is None:
            _RatesFn = _make_rates_fn()
        return _RatesFn
    raise AttributeError(name)


def rates(mech: Mechanism, T, p, Y, dlnA=None):
    """Differentiable (omega, hrr); dlnA defaults to zeros (no gradient)."""
    torch = _torch()
    if dlnA is None:
        dlnA = torch.zeros(mech.R, dtype=torch.float64, device=T.device)
    fn = __getattr__("RatesFn")
    return fn.apply(mech, T, p, Y, dlnA)
