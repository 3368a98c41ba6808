#!/usr/bin/env python
"""Benchmark of the pointwise thermochemistry hot path on GB300.

Workload: the 53-species / 325-reaction synthetic mechanism (20 third-body, 25 Troe) on a
flame-like field of 4,096 hexahedral elements x 8^3 GLL points = 2,097,152 points
(polynomial order 7, Sec. 3.3 of the paper), FP64 state in HBM (inputs 0.92 GB, larger
than L2, so no flush between iterations is needed).

One step = one pass of every row of the hot path over all points, each through the C ABI:
  thermo_eval (FP64), rates_eval (FP64), transport_eval (FP64), rates_eval (mixed),
  transport_eval (mixed), rates_jvp, rates_vjp (with the ln A reduction).
Each launch is bracketed by CUDA events on the launching stream.  The headline value is
Mpoints/s of rates + transport in FP64 (points / (t_rates + t_transport) summed over the
timed steps); the mixed form, JVP/forward and VJP/forward ratios come from the same steps.
After the timed steps, the all-double forms of rates and transport (NK_FP64_NATIVE, the
plain-FP64 arithmetic the FP64 form is checked against), the implicit-stage sources and their
JVP (nk_rhs_eval, nk_rhs_jvp), the diffusion fluxes (nk_diffusion_fluxes) and the stored
linearization with one JVP from it (nk_rates_linearize, nk_rates_jvp_linearized; and rounded
to float with a single-precision JVP, the _f32 entries) are timed the same way in a separate loop
("fp64_native_value", rows); they are not part of a step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs the same workload on its own GPU (weak scaling, no
collective in the data path); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpoints/s rates+transport (FP64 vs mixed), % roofline; VJP/forward time ratio"
UNIT = "Mpoints/s"
MECH = "ch4_53sp_325rx"
WORKLOAD = "flame_4096el"
# FP64 peak of GB300: 1.25 TFLOP/s nominal dense FP64 (vendor figure at the maximum SM clock)
FP64_PEAK_TFLOPS = 1.25
# flops charged per exp/log/pow: table-driven exponential after Tang (1989): argument
# reduction (2 FMA), degree-5 polynomial (5 FMA), table scaling (1 multiply) = 15 flops
TRANSC_FLOPS = 15.0


# ---------------------------------------------------------------------------------- flop model
def _entries(mech, r):
    reac = [(int(mech.reac_sp[i]), int(mech.reac_nu[i])) for i in range(mech.reac_ptr[r], mech.reac_ptr[r + 1])]
    prod = [(int(mech.prod_sp[i]), int(mech.prod_nu[i])) for i in range(mech.prod_ptr[r], mech.prod_ptr[r + 1])]
    return reac, prod


def algorithmic_flops(mech) -> dict:
    """FP64 flops per point of each row (FMA = 2, exp/log = TRANSC_FLOPS).  Minimal arithmetic
    of the evaluated definitions, independent of how a kernel organises it."""
    import numpy as np
    t = TRANSC_FLOPS
    K, R = mech.K, mech.R
    P = K * (K - 1) // 2
    n_eff = [int(np.sum(mech.eff[r] != 1.0)) if mech.rtype[r] else 0 for r in range(R)]
    pre = 2 * t + 4 + K * (3 + 14)                 # ln T, 1/T, rho; y_k, sum, C_k, g_k/RT
    per_rxn, per_rxn_d = 0.0, 0.0
    for r in range(R):
        reac, prod = _entries(mech, r)
        ne = len(reac) + len(prod)
        nu_r = sum(nu for _, nu in reac)
        nu_p = sum(nu for _, nu in prod)
        f = 4 + 2 * ne + 2 + (nu_r - 1) + (nu_p - 1) + 2 * t + 3 + 2 * ne
        if mech.rtype[r] == 1:
            f += 1 + 2 * n_eff[r]
        if mech.rtype[r] == 2:
            f += 2 * n_eff[r] + 4 + 2 + t + (3 if mech.troe[r, 3] > 0 else 2) * t + 4 + t + 12 + 3 + t + 2 + t + 2
        per_rxn += f
        # tangent (JVP) or adjoint (VJP) of the same operations: the product rule doubles every
        # multiply, plus the chain factors of each exponential
        per_rxn_d += f + (4 + 2 * ne + 2 + 2 * (nu_r + nu_p) + 8 + 2 * ne) + (40 if mech.rtype[r] == 2 else 0)
    hrr = K * 14 + 2
    rates = pre + per_rxn + hrr
    transport = (t + 4 + 3 * K                      # ln T, Wbar, X_k
                 + P * (6 + t + 1 + 4)              # ln D_jk cubic, exp, pressure scale, two FMA
                 + K * 4                            # numerators (prefix/suffix) and division
                 + K * (6 + 2 * t + 4)              # lambda_k, 1/lambda_k, two FMA
                 + K * (6 + t + 2)                  # mu_k^1/2, sigma_k, tau_k
                 + K * 4 + K * K * 6                # X tau, X tau^2; three FMA per pair
                 + K * 8)                           # Wilke denominators and the mixture sum
    thermo = 2 * t + 4 + K * (3 + 10 + 12 + 14 + 4)
    jvp = pre + K * 16 + per_rxn_d + hrr * 2 + K * 10
    vjp = pre + K * 24 + per_rxn_d + 10 * R + K * 8
    rhs = rates + K * 12 + 4                        # W_k/rho factors, c_p, 1/(rho c_p)
    rhs_jvp = jvp + K * 24 + 12                     # primal omega, c_p and d c_p, both source tangents
    # per direction from stored coefficients: dq_r = A tT + sum_e B_e dC_e (+ L d[M]), the scatter
    n_ent = sum(len(_entries(mech, r)[0]) + len(_entries(mech, r)[1]) for r in range(R))
    jvp_lin = 2 * R + 2 * n_ent + 2 * n_ent + sum(2 * n_eff[r] + 4 for r in range(R) if mech.rtype[r]) \
        + K * (6 + 4) + K * 2 + 4
    return {"thermo": thermo, "rates_fp64": rates, "transport_fp64": transport, "rates_fp64_native": rates,
            "rates_jit": rates,
            "transport_fp64_native": transport, "rates_mixed": rates, "transport_mixed": transport, "jvp": jvp,
            "vjp": vjp, "rhs_fp64": rhs, "rhs_jvp": rhs_jvp, "linearize": jvp, "jvp_linearized": jvp_lin,
            "linearize_f32": jvp, "jvp_linearized_f32": jvp_lin,
            "diffusion": K * (3 + 6 + 6 + 9 + 10) + 12}


# ---------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------- helpers
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _emit(obj):
    print(json.dumps(obj), flush=True)


def _sources_sha256(paths):
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic(kernel_row):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary, if none of
    the kernel's source files changed since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel_row)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    try:
        h = _sources_sha256(rec["sources"])
    except (OSError, KeyError):
        return None
    return rec["bytes_per_launch"] if h == rec.get("sources_sha256") else None


def _oracle_sample(n_points):
    """The oracle as it stands on a bounded sample of the workload (first n_points points)."""
    import oracle
    from paper_2409_06404_gb300 import synth
    mech = synth.mechanism(MECH)
    st = synth.workload_states(WORKLOAD, mech.K, n_points=n_points)
    return oracle, mech, st


def cpu_baseline(st_full, n_points=524288):
    """Oracle rates + transport (FP64) on the first n_points points, all host cores."""
    import numpy as np
    import oracle
    from paper_2409_06404_gb300 import synth
    mech = synth.mechanism(MECH)
    n_points = min(n_points, st_full.n)
    T, p, Y = st_full.T[:n_points], st_full.p[:n_points], np.ascontiguousarray(st_full.Y[:, :n_points])
    t0 = time.perf_counter()
    oracle.rates(mech, T, p, Y)
    oracle.transport(mech, T, p, Y)
    dt = time.perf_counter() - t0
    return {"value": n_points / dt / 1e6, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"first {n_points} points ({n_points // 512} elements) of the {WORKLOAD} workload, "
                      f"rates + transport FP64, OpenMP over points, {dt:.1f} s"}


# ---------------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    n_points = 32768
    oracle, mech, st = _oracle_sample(n_points)

    def step():
        oracle.rates(mech, st.T, st.p, st.Y)
        oracle.transport(mech, st.T, st.p, st.Y)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = n_points * args.steps / dt / 1e6
    cores = oracle.max_threads()
    _emit({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"{MECH} on {WORKLOAD} (2,097,152 points); each step a "
                                  f"{n_points}-point sample", "mechanism": MECH, "points": n_points},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"first {n_points} points of {WORKLOAD} per step, rates + transport FP64"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ---------------------------------------------------------------------------------- implicit stage
def implicit_stage(nk, m, T, p, Y, n_dir, steps, stream):
    """One implicit-stage sweep as a Newton-Krylov stage issues it: one forward (thermo FP64,
    rates and transport mixed) and n_dir exact JVPs along N(0, 1) directions, against the
    plain-FP64 forward and n_dir finite-difference JVPs (NITSOL step per point,
    sigma = sqrt((1 + |x|) eps) / |v|) on the same GPU.  Directions are generated before the
    timed region; each sweep is timed with CUDA events on the launching stream."""
    import torch
    n, K = T.shape[0], Y.shape[0]
    gen = torch.Generator(device=T.device).manual_seed(5000)
    dirs = [(torch.randn(n, generator=gen, dtype=torch.float64, device=T.device),
             torch.randn((K, n), generator=gen, dtype=torch.float64, device=T.device)) for _ in range(n_dir)]
    eps = 2.220446049250313e-16
    xnorm = torch.sqrt(T * T + (Y * Y).sum(0))

    def ours():
        nk.thermo_eval(m, T, p, Y)
        nk.rates_eval(m, T, p, Y, precision="mixed")
        nk.transport_eval(m, T, p, Y, precision="mixed")
        out = None
        for vT, vY in dirs:
            out = nk.rates_jvp(m, T, p, Y, vT, vY)
        return out

    def fd():
        nk.thermo_eval(m, T, p, Y)
        w0, h0 = nk.rates_eval(m, T, p, Y)
        nk.transport_eval(m, T, p, Y)
        out = None
        for vT, vY in dirs:
            sig = torch.sqrt((1.0 + xnorm) * eps) / torch.sqrt(vT * vT + (vY * vY).sum(0))
            w1, h1 = nk.rates_eval(m, T + sig * vT, p, Y + sig * vY)
            out = ((w1 - w0) / sig, (h1 - h0) / sig)
        return out

    def timed(f):
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return sum(ts) / len(ts)

    lin = None
    try:
        lin = torch.empty((nk.linearization_slots(m), n), dtype=torch.float64, device=T.device)
    except RuntimeError:                       # the stored data do not fit: recompute only
        pass

    def ours_lin():
        nk.thermo_eval(m, T, p, Y)
        nk.rates_eval(m, T, p, Y, precision="mixed")
        nk.transport_eval(m, T, p, Y, precision="mixed")
        nk.rates_linearize(m, T, p, Y, lin=lin)
        out = None
        for vT, vY in dirs:
            out = nk.rates_jvp_linearized(m, T, p, Y, lin, vT, vY)
        return out

    t_ours, t_fd = timed(ours), timed(fd)
    t_lin = timed(ours_lin) if lin is not None else None
    # accuracy of the difference quotient against the exact JVP, last direction
    dw, dh = nk.rates_jvp(m, T, p, Y, *dirs[-1])
    fw, fh = fd()
    sc = dw.abs().amax(0).clamp_min(1e-300)
    fd_err = ((fw - dw).abs().amax(0) / sc).median().item()
    res = {"points": n, "directions": n_dir, "sweep_ms": t_ours, "fd_fp64_sweep_ms": t_fd,
           "speedup_vs_fd": t_fd / t_ours, "fd_jvp_median_rel_err": fd_err,
           "sweep": "thermo (FP64) + rates, transport (mixed) + exact JVPs recomputed per direction",
           "fd_sweep": "thermo, rates, transport (FP64) + FP64 rates at x + sigma v per direction"}
    if t_lin is not None:
        res.update({"sweep_linearized_ms": t_lin, "speedup_linearized_vs_fd": t_fd / t_lin,
                    "sweep_linearized": "the same forward + one stored linearization + exact JVPs from it"})
    return res


# ---------------------------------------------------------------------------------- reactor step
def reactor_states(nk, m, mech, n, dev, seed=6053):
    """Near-equilibrium states for the implicit reactor step: chemical equilibria at 512
    temperatures in [1300, 2600] K and 1 atm from element potentials (X_k proportional to
    exp(-g_k/RT + sum_e lambda_e a_ek), normalised by a uniform shift found by bisection; g_k
    from nk_thermo_eval), tiled over the n points and perturbed by 1e-3 in Y and ~1 K in T."""
    import numpy as np
    import torch
    nu, K = 512, mech.K
    rng = np.random.default_rng(seed)
    Tu = np.linspace(1300.0, 2600.0, nu)
    f64 = dict(dtype=torch.float64, device=dev)
    th = nk.thermo_eval(m, torch.tensor(Tu, **f64), torch.full((nu,), 101325.0, **f64),
                        torch.full((K, nu), 1.0 / K, **f64))
    gRT = th["g_k"].cpu().numpy() / (8.314462618 * Tu[None, :])            # [K, nu]
    a = mech.atoms.astype(float)
    lam = np.linalg.lstsq(np.hstack([a, np.ones((K, 1))]), gRT, rcond=None)[0][:-1]
    lam = lam + 0.5 * rng.standard_normal(lam.shape)
    base = -gRT + a @ lam
    na = a.sum(axis=1)[:, None]
    lo, hi = np.full(nu, -1e4), np.full(nu, 1e4)
    for _ in range(200):                                                  # sum_k X_k(t) = 1, monotone in t
        t = 0.5 * (lo + hi)
        z = base + t[None, :] * na
        zm = z.max(axis=0)
        big = zm + np.log(np.exp(z - zm).sum(axis=0)) > 0.0
        hi, lo = np.where(big, t, hi), np.where(big, lo, t)
    X = np.exp(base + 0.5 * (lo + hi)[None, :] * na)
    Yu = X * mech.W[:, None]
    Yu /= Yu.sum(axis=0)
    idx = torch.arange(n, device=dev) % nu
    gen = torch.Generator(device=dev).manual_seed(seed)
    T = torch.tensor(Tu, **f64)[idx] + torch.randn(n, generator=gen, **f64)
    Y = torch.tensor(Yu, **f64)[:, idx] * (1.0 + 1e-3 * torch.randn((K, n), generator=gen, **f64))
    Y /= Y.sum(0)
    return T, torch.full((n,), 101325.0, **f64), Y.contiguous()


def reactor_row(nk, m, mech, n, dev, stream, dt=1e-9, dt_large=1e-5):
    """One implicit Euler step over n near-equilibrium points (nk_reactor_step), each after one
    untimed step from the same states; CUDA events on the launching stream.  The paper's
    unpreconditioned GMRES at dt (products recomputing the rates, from a stored linearization per
    Newton iteration, and from that linearization rounded to float in single precision), and with the per-point block-Jacobi preconditioner at dt and at
    dt_large, each with its set-up (precond 1) and with the factors of the previous call reused
    (precond 2, as a stiff ODE solver keeps its Newton matrix over steps)."""
    import torch
    T0, p, Y0 = reactor_states(nk, m, mech, n, dev)
    kw = dict(rtol=1e-6, atol_T=1e-6, atol_Y=1e-12, newton_tol=1e-4, lin_tol=1e-6, max_newton=20, krylov_dim=30)
    ws = torch.empty(max(nk.reactor_workspace(m, n, kw["krylov_dim"], 1, 1),
                         nk.reactor_workspace(m, n, kw["krylov_dim"], 0, 2)), dtype=torch.uint8, device=dev)
    T, Y = T0.clone(), Y0.clone()

    def run(step, precond, linearized=0):
        o = nk.reactor_opts(precond=precond, linearized=linearized, **kw)
        for timed in (False, True):
            T.copy_(T0)
            Y.copy_(Y0)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = nk.reactor_step(m, T, p, Y, step, o, workspace=ws)
            b.record(stream)
            torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        return {"dt_s": step, "ms": ms, "newton_iters": st["newton_iters"], "krylov_iters": st["krylov_iters"],
                "converged": st["converged"], "ms_per_krylov_iter": ms / max(st["krylov_iters"], 1)}

    res = {"points": n,
           "workload": f"{MECH}, near-equilibrium states (1300-2600 K, perturbed 1e-3), one implicit Euler step, "
                       f"GMRES(30), rtol 1e-6, atol_T 1e-6, atol_Y 1e-12, newton_tol 1e-4, lin_tol 1e-6"}
    res.update(run(dt, 0))
    res["linearized"] = run(dt, 0, 1)
    res["linearized_f32"] = run(dt, 0, 2)
    res["block_jacobi"] = run(dt, 1)
    res["block_jacobi_linearized"] = run(dt, 1, 1)
    res["block_jacobi_reused"] = run(dt, 2)
    res["block_jacobi_large_dt"] = run(dt_large, 1)
    res["block_jacobi_large_dt_reused"] = run(dt_large, 2)
    return res


# ---------------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2409_06404_gb300 as nk
    from paper_2409_06404_gb300 import synth

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    mech = synth.mechanism(MECH)
    st = synth.workload_states(WORKLOAD, mech.K, n_elements=args.elements)
    n, K, R = st.n, mech.K, mech.R
    m = nk.mechanism_load(mech)
    T = torch.from_numpy(st.T).to(dev)
    p = torch.from_numpy(st.p).to(dev)
    Y = torch.from_numpy(st.Y).to(dev)
    gen = torch.Generator(device=dev).manual_seed(5000 + rank)
    vT = torch.randn(n, generator=gen, dtype=torch.float64, device=dev)
    vY = torch.randn((K, n), generator=gen, dtype=torch.float64, device=dev)
    wbar = torch.randn((K, n), generator=gen, dtype=torch.float64, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    out = {k: torch.empty(n, **f64) for k in ("cp", "h", "wb", "rho", "hrr", "mu", "lam", "hrr_m", "mu_m", "lam_m",
                                               "dh", "gT")}
    out.update({k: torch.empty((K, n), **f64) for k in ("w", "D", "w_m", "D_m", "dw", "gY")})
    g_lnA = torch.empty(R, **f64)
    lin = torch.empty((nk.linearization_slots(m), n), **f64)    # stored linearization (~18 KB per point)
    lin32 = torch.empty((nk.linearization_slots_f32(m), n), dtype=torch.float32, device=dev)   # single precision
    gradX = torch.randn((3, K, n), generator=gen, **f64)         # mole-fraction gradients (synthetic)
    jflux = torch.empty((3, K, n), **f64)
    Vc = torch.empty((3, n), **f64)
    hflux = torch.empty((3, n), **f64)
    wsb = torch.empty(max(nk.rates_vjp_workspace(m, n), 8), dtype=torch.uint8, device=dev)
    L = nk.lib()
    s = torch.cuda.current_stream()
    sp = nk._vp(s.cuda_stream)
    P = lambda t: nk._vp(t.data_ptr())
    h = m.handle

    def chk(st_):
        if st_ != 0:
            raise nk.NkError(st_, L.nk_last_error().decode())

    rows = {
        "thermo": lambda: chk(L.nk_thermo_eval(h, n, n, P(T), P(p), P(Y), P(out["cp"]), P(out["h"]), P(out["wb"]),
                                               P(out["rho"]), None, None, None, sp)),
        "rates_fp64": lambda: chk(L.nk_rates_eval(h, n, n, P(T), P(p), P(Y), None, P(out["w"]), P(out["hrr"]), 0, sp)),
        "transport_fp64": lambda: chk(L.nk_transport_eval(h, n, n, P(T), P(p), P(Y), P(out["mu"]), P(out["lam"]),
                                                          P(out["D"]), 0, sp)),
        "rates_mixed": lambda: chk(L.nk_rates_eval(h, n, n, P(T), P(p), P(Y), None, P(out["w_m"]), P(out["hrr_m"]),
                                                   1, sp)),
        "transport_mixed": lambda: chk(L.nk_transport_eval(h, n, n, P(T), P(p), P(Y), P(out["mu_m"]),
                                                           P(out["lam_m"]), P(out["D_m"]), 1, sp)),
        "jvp": lambda: chk(L.nk_rates_jvp(h, n, n, P(T), P(p), P(Y), None, P(vT), P(vY), None, None, P(out["dw"]),
                                          P(out["dh"]), sp)),
        "vjp": lambda: chk(L.nk_rates_vjp(h, n, n, P(T), P(p), P(Y), None, P(wbar), None, P(out["gT"]), P(out["gY"]),
                                          P(g_lnA), P(wsb), wsb.numel(), sp)),
    }
    forms = {
        "rates_fp64_native": lambda: chk(L.nk_rates_eval(h, n, n, P(T), P(p), P(Y), None, P(out["w"]),
                                                         P(out["hrr"]), 2, sp)),
        "transport_fp64_native": lambda: chk(L.nk_transport_eval(h, n, n, P(T), P(p), P(Y), P(out["mu"]),
                                                                 P(out["lam"]), P(out["D"]), 2, sp)),
        "rhs_fp64": lambda: chk(L.nk_rhs_eval(h, n, n, P(T), P(p), P(Y), None, P(out["hrr"]), P(out["w"]), 0, sp)),
        "rhs_jvp": lambda: chk(L.nk_rhs_jvp(h, n, n, P(T), P(p), P(Y), None, P(vT), P(vY), None, None,
                                            P(out["dh"]), P(out["dw"]), sp)),
        "diffusion": lambda: chk(L.nk_diffusion_fluxes(h, n, n, P(T), P(p), P(Y), P(out["D"]), P(gradX), P(jflux),
                                                        P(Vc), P(hflux), sp)),
        "linearize": lambda: chk(L.nk_rates_linearize(h, n, n, P(T), P(p), P(Y), None, P(lin), n, sp)),
        "jvp_linearized": lambda: chk(L.nk_rates_jvp_linearized(h, n, n, P(T), P(p), P(Y), P(lin), n, P(vT), P(vY),
                                                                P(out["dw"]), P(out["dh"]), sp)),
        "rates_jit": lambda: chk(L.nk_rates_eval(h, n, n, P(T), P(p), P(Y), None, P(out["w"]), P(out["hrr"]), 3, sp)),
        "linearize_f32": lambda: chk(L.nk_rates_linearize_f32(h, n, n, P(T), P(p), P(Y), None, P(lin32), n, sp)),
        "jvp_linearized_f32": lambda: chk(L.nk_rates_jvp_linearized_f32(h, n, n, P(T), P(p), P(Y), P(lin32), n,
                                                                        P(vT), P(vY), P(out["dw"]), P(out["dh"]),
                                                                        sp)),
    }
    # the mechanism-specialised kernel is compiled (NVRTC) before any timing
    t_jit = time.perf_counter()
    nk.mechanism_jit(m)
    jit_compile_s = time.perf_counter() - t_jit
    launches_per_step = {"thermo": 1, "rates_fp64": 1, "transport_fp64": 1, "rates_mixed": 1,
                         "transport_mixed": 1, "jvp": 1, "vjp": 2}
    names = list(rows)

    for _ in range(args.warmup):
        for f in rows.values():
            f()
    torch.cuda.synchronize()
    ev = {k: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)] for k in names}
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            for k in names:
                ev[k][i][0].record(s)
                rows[k]()
                ev[k][i][1].record(s)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if ws > 1:
        dist.barrier()
    ms = {k: [a.elapsed_time(b) for a, b in ev[k]] for k in names}
    step_ms = [ev[names[0]][i][0].elapsed_time(ev[names[-1]][i][1]) for i in range(args.steps)]

    # ---- the all-double forms, for comparison (not part of a step)
    for f in forms.values():
        f()
    torch.cuda.synchronize()
    fev = {k: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)] for k in forms}
    for i in range(args.steps):
        for k, f in forms.items():
            fev[k][i][0].record(s)
            f()
            fev[k][i][1].record(s)
    torch.cuda.synchronize()
    ms.update({k: [a.elapsed_time(b) for a, b in fev[k]] for k in forms})

    # ---- implicit reactor step (not part of a step)
    reactor = reactor_row(nk, m, mech, n, dev, s) if args.reactor else None

    # ---- implicit-stage sweep (not part of a step)
    stage = None
    if args.stage_dirs > 0:
        if args.stage_elements in (None, args.elements):
            stage = implicit_stage(nk, m, T, p, Y, args.stage_dirs, 3, s)
        else:
            st5 = synth.workload_states("flame_32768el" if args.stage_elements == 32768 else WORKLOAD, K,
                                        n_elements=args.stage_elements)
            T5, p5, Y5 = (torch.from_numpy(a).to(dev) for a in (st5.T, st5.p, st5.Y))
            del st5
            stage = implicit_stage(nk, m, T5, p5, Y5, args.stage_dirs, 2, s)
            del T5, p5, Y5
        stage["workload"] = f"{MECH} on {stage['points']} points"

    fwd_ms = sum(ms["rates_fp64"]) + sum(ms["transport_fp64"])
    nat_ms = sum(ms["rates_fp64_native"]) + sum(ms["transport_fp64_native"])
    mix_ms = sum(ms["rates_mixed"]) + sum(ms["transport_mixed"])
    tot_ms = sum(step_ms)
    vals = torch.tensor([fwd_ms, nat_ms, mix_ms, tot_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(vals, op=dist.ReduceOp.MAX)
    fwd_ms, nat_ms, mix_ms, tot_ms = vals.tolist()
    value = ws * n * args.steps / (fwd_ms * 1e-3) / 1e6
    native_value = ws * n * args.steps / (nat_ms * 1e-3) / 1e6
    mixed_value = ws * n * args.steps / (mix_ms * 1e-3) / 1e6

    # ---- end to end through the public API with host buffers (pinned), FP64 forward
    e2e = None
    if not args.no_e2e:
        hT = torch.from_numpy(st.T).pin_memory()
        hp = torch.from_numpy(st.p).pin_memory()
        hY = torch.from_numpy(st.Y).pin_memory()
        ho = {k: torch.empty(n, dtype=torch.float64).pin_memory() for k in ("hrr", "mu", "lam")}
        ho.update({k: torch.empty((K, n), dtype=torch.float64).pin_memory() for k in ("w", "D")})

        chunk = 65536                  # (65536 to 1M measured: smaller chunks hide the copies best)
        wse = torch.empty(nk.host_eval_workspace(m, min(chunk, n)), dtype=torch.uint8, device=dev)

        def e2e_step():
            # the C-ABI entry for host-resident fields: chunked H2D, FP64 rates and transport, D2H
            chk(L.nk_host_eval(h, n, P(hT), P(hp), P(hY), P(ho["w"]), P(ho["hrr"]), P(ho["mu"]), P(ho["lam"]),
                               P(ho["D"]), 0, chunk, P(wse), wse.numel(), sp))

        e2e_step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(args.steps):
            e2e_step()
        b.record(s)
        torch.cuda.synchronize()
        e_ms = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(e_ms, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * n * args.steps / (e_ms.item() * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": (2 + K) * 8 * n, "d2h_bytes_per_step": (2 * K + 3) * 8 * n,
               "api": f"nk_host_eval: page-locked host T, p, Y in and omega, hrr, mu, lambda, D_k out; chunks of "
                      f"{chunk} points over three streams (copies overlap the FP64 kernels)"}

    if rank != 0:
        return
    # ---- roofline of the dominant kernel (ALU bound: FP64 pipe)
    fl = algorithmic_flops(mech)
    avg = {k: sum(v) / len(v) for k, v in ms.items() if k in names}
    avg_f = {k: sum(v) / len(v) for k, v in ms.items() if k in forms}
    dom = max(names, key=lambda k: avg[k])
    achieved = fl[dom] * n / (avg[dom] * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": _traffic(dom),
            "peak_source": "nominal dense FP64 of GB300 (1.25 TFLOP/s), no measured FP64 peak in MEASURED_PEAKS.json",
            "basis": "FP64 flops of the evaluated definitions (FMA = 2, exp/log = 15) per point x points / "
                     "kernel time; the FP64 form evaluates its exponent chains as float pairs on the FP32 "
                     "pipe, so it is not confined to the FP64 pipe's rate",
            "flops_per_point": fl[dom]}
    both = {**avg, **avg_f}
    rows_out = {k: {"ms": both[k], "mpts": n / (both[k] * 1e-3) / 1e6,
                    "tflops": fl[k] * n / (both[k] * 1e-3) / 1e12} for k in names + list(forms)}
    fwd_avg = avg["rates_fp64"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{MECH} (53 species, 325 reactions: 20 third-body, 25 Troe) on {WORKLOAD}: "
                               f"{args.elements} elements x 512 GLL points = {n} points, FP64 SoA",
                   "mechanism": MECH, "points": n, "value_basis": "points / (rates_fp64 + transport_fp64 time)",
                   "step": names, "forms_after_steps": list(forms),
                   "l2": "inputs (0.92 GB) larger than L2; no flush"},
        "mixed_value": mixed_value,
        "fp64_native_value": native_value,
        "vjp_over_fwd": avg["vjp"] / fwd_avg, "jvp_over_fwd": avg["jvp"] / fwd_avg,
        "rows": rows_out,
        "roofline": roof,
        "gpu_launches": sum(launches_per_step.values()) * args.steps,
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
    }
    line["jit"] = {"compile_s": jit_compile_s, "rates_jit_ms": avg_f["rates_jit"],
                   "rates_fp64_native_ms": avg_f["rates_fp64_native"], "rates_fp64_ms": avg["rates_fp64"],
                   "form": "NK_JIT: all-double arithmetic of NK_FP64_NATIVE in a kernel generated for the "
                           "mechanism (straight-line code, literals), NVRTC-compiled at first use"}
    if stage is not None:
        line["implicit_stage"] = stage
    if reactor is not None:
        line["reactor_step"] = reactor
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(st)
    _emit(line)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--elements", type=int, default=4096,
                    help="flame field size in elements (a cube; 4096 = the benchmark workload)")
    ap.add_argument("--no-reactor", dest="reactor", action="store_false",
                    help="skip the implicit reactor step measurement")
    ap.add_argument("--stage-dirs", type=int, default=10,
                    help="JVP directions of the implicit-stage sweep (0 skips it)")
    ap.add_argument("--stage-elements", type=int, default=None,
                    help="elements of the implicit-stage field (default: --elements; 32768 = 16,777,216 points)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
