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
import ctypes
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
# nominal dense FP64 of GB300 (vendor figure), for context beside the measured pipe rates
FP64_NOMINAL_TFLOPS = 1.25


# ---------------------------------------------------------------------------------- roofline inputs
# Kernels of this library are bound by the FP64 pipe or the FP32 (FMA) pipes.  Their per-pipe
# roofline: the pipe operations a kernel issues per point (ncu counters of the same kernels,
# profiles/pipe_counts.json) x points / CUDA-event time, against the pipe's operation rate measured
# in this run by the probe library.  The algorithmic operation counts of the definitions (the
# oracle's instrumented scalar, profiles/algorithmic_ops.json) are reported beside them.
PROBE_KINDS = {"dfma": 0, "dmul": 1, "dadd": 2, "ffma": 3, "fmul": 4, "fadd": 5}


def pipe_peaks():
    """Thread-level operations per second of the FP64 pipe (double multiply-add, multiply, add) and
    the FP32 FMA pipes (float), measured now: independent streams on every SM, 8 blocks of 256
    threads per SM, best of 5 CUDA-event-timed launches (libnkprobe.so)."""
    import ctypes
    from paper_2409_06404_gb300 import build as nkbuild
    L = ctypes.CDLL(nkbuild.PROBE_LIB)
    L.nkp_pipe_rate.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_double)]
    L.nkp_pipe_rate.restype = ctypes.c_int
    out = {}
    for name, kind in PROBE_KINDS.items():
        v = ctypes.c_double()
        st = L.nkp_pipe_rate(kind, 8, 2048 if kind < 3 else 32768, 5, ctypes.byref(v))
        if st != 0:
            raise RuntimeError(f"pipe probe {name} failed ({st})")
        out[name] = v.value
    return out


def hbm_peak_gbs():
    """The measured copy bandwidth in MEASURED_PEAKS.json (GB/s), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def _json_profile(name):
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def pipe_counts():
    """Per-point pipe operation counts of each row's kernels (profiles/pipe_counts.json), for the rows
    none of whose source files changed since the capture."""
    rec = _json_profile("pipe_counts.json") or {}
    good = {}
    for row, r in rec.get("rows", {}).items():
        try:
            if _sources_sha256(r["sources"]) == r["sources_sha256"]:
                good[row] = r
        except (OSError, KeyError):
            continue
    return good


def row_pipes(row_counts, n, ms, peaks):
    """Per-pipe fractions of one row: warp instructions per point x 32 lanes x n / time, against the
    probe's multiply-add rate of that pipe (a warp instruction occupies the pipe for a full warp,
    whatever its active lanes)."""
    t = ms * 1e-3
    res = {}
    for pipe, peak in (("fp64", peaks["dfma"]), ("fma", peaks["ffma"])):
        ops = row_counts[f"{pipe}_warp_inst_per_point"] * 32.0
        achieved = ops * n / t
        res[pipe] = {"ops_per_point": ops, "gops": achieved / 1e9, "peak_gops": peak / 1e9, "frac": achieved / peak}
    return res


def algorithmic(mech_name):
    rec = _json_profile("algorithmic_ops.json")
    if not rec:
        return {}
    return rec.get("mechanisms", {}).get(mech_name, {}).get("per_point", {})


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


def _oracle_rate(oracle, mech, T, p, Y, threads):
    t0 = time.perf_counter()
    oracle.rates(mech, T, p, Y, threads=threads)
    oracle.transport(mech, T, p, Y, threads=threads)
    dt = time.perf_counter() - t0
    return T.shape[0] / dt / 1e6, dt


def cpu_baseline(st_full, n_points=524288):
    """The oracle as it stands (rates + transport, FP64) on bounded samples of the workloads, on all
    host cores (OpenMP over points) and on one thread: the benchmark field (first n_points points)
    and the configurations of the 9- and 120-species mechanisms."""
    import numpy as np
    import oracle
    from paper_2409_06404_gb300 import synth
    mech = synth.mechanism(MECH)
    n_points = min(n_points, st_full.n)
    T, p, Y = st_full.T[:n_points], st_full.p[:n_points], np.ascontiguousarray(st_full.Y[:, :n_points])
    v, dt = _oracle_rate(oracle, mech, T, p, Y, 0)
    n1 = min(16384, n_points)
    v1, dt1 = _oracle_rate(oracle, mech, T[:n1], p[:n1], np.ascontiguousarray(Y[:, :n1]), 1)
    res = {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "nproc": os.cpu_count(), "kind": "oracle",
           "sample": f"first {n_points} points ({n_points // 512} elements) of the {WORKLOAD} workload, "
                     f"rates + transport FP64, OpenMP over points, {dt:.1f} s",
           "one_thread": {"value": v1, "unit": UNIT, "cores": 1,
                          "sample": f"first {n1} points of {WORKLOAD}, {dt1:.1f} s"}}
    configs = {}
    for name, wl, n_all, n_one in (("h2_9sp_21rx", "uniform_64el", 32768, 32768),
                                   ("big_120sp_700rx", "flame_4096el", 65536, 4096)):
        mc = synth.mechanism(name)
        sc = synth.workload_states(wl, mc.K, n_points=n_all)
        va, da = _oracle_rate(oracle, mc, sc.T, sc.p, sc.Y, 0)
        vo, do = _oracle_rate(oracle, mc, sc.T[:n_one], sc.p[:n_one], np.ascontiguousarray(sc.Y[:, :n_one]), 1)
        configs[name] = {"all_cores": va, "one_thread": vo, "unit": UNIT,
                         "sample": f"first {n_all} points of {wl} ({da:.1f} s); one thread: first {n_one} "
                                   f"({do:.1f} s)"}
    res["configs"] = configs
    return res


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
    """Implicit-stage sweeps as a Newton-Krylov stage issues them: a forward at the state and n_dir
    exact JVPs along seeded N(0, 1) directions, against the plain-FP64 forward and n_dir
    finite-difference JVPs (NITSOL step per point, sigma = sqrt((1 + |x|) eps) / |v|) on the same
    GPU.  Exact sweeps:
      recompute  thermo (FP64), rates and transport (mixed), then nk_rates_jvp per direction (the
                 rates of progress formed again for every product);
      compact    thermo (FP64), transport (mixed), nk_rates_linearize_compact, which also gives the
                 rates at the state (FP64), then nk_rates_jvp_linearized_compact per direction;
      per-entry  the same forward as recompute plus nk_rates_linearize, then
                 nk_rates_jvp_linearized per direction (only where its data fit: not at 16.8M points).
    Beside them, not one of them (its products are single precision): the same forward plus
    nk_rates_linearize_f32, then nk_rates_jvp_linearized_f32 per direction, with its error against
    the exact FP64 JVP.
    Every call goes through the C ABI into buffers allocated before timing, and the difference
    quotients use in-place operations, so no arm waits on the allocator inside its spans.  Each
    direction is drawn (seeded, on the device) before its product, outside the timed spans; a
    sweep's time is the sum of CUDA-event spans around its forward and its n_dir products on the
    launching stream (one direction buffer stays resident instead of n_dir)."""
    import torch
    n, K = T.shape[0], Y.shape[0]
    f64 = dict(dtype=torch.float64, device=T.device)
    L = nk.lib()
    sp = nk._vp(stream.cuda_stream)
    P = lambda t: nk._vp(t.data_ptr())
    h = m.handle

    def chk(st_):
        if st_ != 0:
            raise nk.NkError(st_, L.nk_last_error().decode())

    vT, dh, hrr, cp, hm, mu, lam, Tp, h1 = (torch.empty(n, **f64) for _ in range(9))
    vY, dw, w, D, Yp, w1 = (torch.empty((K, n), **f64) for _ in range(6))
    w0, h0 = torch.empty((K, n), **f64), torch.empty(n, **f64)
    eps = 2.220446049250313e-16

    def direction(d):
        g = torch.Generator(device=T.device).manual_seed(5000 + d)
        torch.randn(n, generator=g, out=vT)
        torch.randn((K, n), generator=g, out=vY)

    def sweep(forward, product):
        spans = []

        def span(fn):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            spans.append((a, b))
            return out

        ctx = span(forward)
        for d in range(n_dir):
            direction(d)
            span(lambda: product(ctx))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in spans)

    def timed(forward, product):
        sweep(forward, product)                       # warm-up
        return sum(sweep(forward, product) for _ in range(steps)) / steps

    def thermo():
        chk(L.nk_thermo_eval(h, n, n, P(T), P(p), P(Y), P(cp), P(hm), None, None, None, None, None, sp))

    def rates(prec, Tx, Yx, wo, ho):
        chk(L.nk_rates_eval(h, n, n, P(Tx), P(p), P(Yx), None, P(wo), P(ho), prec, sp))

    def transport(prec):
        chk(L.nk_transport_eval(h, n, n, P(T), P(p), P(Y), P(mu), P(lam), P(D), prec, sp))

    def fwd_mixed():
        thermo()
        rates(1, T, Y, w, hrr)
        transport(1)

    def recompute(_):
        chk(L.nk_rates_jvp(h, n, n, P(T), P(p), P(Y), None, P(vT), P(vY), None, None, P(dw), P(dh), sp))

    def fwd_fd():
        xnorm = torch.sqrt(T * T + torch.linalg.vector_norm(Y, dim=0) ** 2)
        thermo()
        rates(0, T, Y, w0, h0)
        transport(0)
        return xnorm

    def fd(xnorm):
        sig = torch.sqrt((1.0 + xnorm) * eps) / torch.sqrt(vT * vT + torch.linalg.vector_norm(vY, dim=0) ** 2)
        torch.addcmul(T, sig, vT, out=Tp)
        torch.addcmul(Y, sig, vY, out=Yp)
        rates(0, Tp, Yp, w1, h1)
        torch.sub(w1, w0, out=dw).div_(sig)
        torch.sub(h1, h0, out=dh).div_(sig)

    res = {"points": n, "directions": n_dir, "steps": steps,
           "timing": "sum of CUDA-event spans around the forward and each product; directions drawn "
                     "outside the spans; every arm into preallocated buffers"}
    res["fd_fp64_sweep_ms"] = t_fd = timed(fwd_fd, fd)
    res["sweep_recompute_ms"] = t_re = timed(fwd_mixed, recompute)
    res["speedup_recompute_vs_fd"] = t_fd / t_re

    # the per-reaction stored linearization, where it fits beside the field and the buffers above
    slots_c = nk.linearization_slots_compact(m)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    linc = None
    if slots_c * n * 8 < free - (4 << 30):
        linc = torch.empty((slots_c, n), **f64)
    if linc is not None:
        def fwd_compact():
            thermo()
            transport(1)
            chk(L.nk_rates_linearize_compact(h, n, n, P(T), P(p), P(Y), None, P(linc), n, P(w), P(hrr), sp))

        def compact(_):
            chk(L.nk_rates_jvp_linearized_compact(h, n, n, P(T), P(p), P(Y), P(linc), n, P(vT), P(vY), P(dw),
                                                  P(dh), sp))

        res["sweep_compact_ms"] = t_c = timed(fwd_compact, compact)
        res["speedup_compact_vs_fd"] = t_fd / t_c
        res["compact_bytes"] = slots_c * n * 8
        # accuracy of the difference quotient against the exact JVP, last direction
        direction(n_dir - 1)
        compact(None)
        exact = dw.clone()
        fd(fwd_fd())
        sc = exact.abs().amax(0).clamp_min(1e-300)
        res["fd_jvp_median_rel_err"] = ((dw - exact).abs().amax(0) / sc).median().item()
        del exact, sc, linc
        torch.cuda.empty_cache()
    # the single-precision per-entry linearization (the products the reactor's FP32 Krylov basis
    # takes), where it fits; reported beside the FP64-exact arms, not as one of them
    slots_f = nk.linearization_slots_f32(m)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if slots_f * n * 4 < free - (4 << 30):
        linf = torch.empty((slots_f, n), dtype=torch.float32, device=T.device)

        def fwd_f32():
            fwd_mixed()
            chk(L.nk_rates_linearize_f32(h, n, n, P(T), P(p), P(Y), None, P(linf), n, sp))

        def prod_f32(_):
            chk(L.nk_rates_jvp_linearized_f32(h, n, n, P(T), P(p), P(Y), P(linf), n, P(vT), P(vY), P(dw), P(dh),
                                              sp))

        res["sweep_f32_ms"] = t_f = timed(fwd_f32, prod_f32)
        res["speedup_f32_vs_fd"] = t_fd / t_f
        res["f32_bytes"] = slots_f * n * 4
        # its products against the exact FP64 JVP (recomputed), last direction; the exact one is
        # kept in the difference quotient's buffer w1, the comparison runs in column chunks
        direction(n_dir - 1)
        recompute(None)
        w1.copy_(dw)
        prod_f32(None)
        rel = torch.empty(n, **f64)
        for a in range(0, n, 1 << 20):
            e, x = w1[:, a:a + (1 << 20)], dw[:, a:a + (1 << 20)]
            rel[a:a + (1 << 20)] = (x - e).abs().amax(0) / e.abs().amax(0).clamp_min(1e-300)
        res["f32_jvp_median_rel_err"] = rel.median().item()
        res["f32_jvp_max_rel_err"] = rel.max().item()
        del rel, linf
        torch.cuda.empty_cache()
    lin = None
    try:
        lin = torch.empty((nk.linearization_slots(m), n), **f64)
    except RuntimeError:                           # the per-entry data do not fit
        pass
    if lin is not None:
        def fwd_lin():
            fwd_mixed()
            chk(L.nk_rates_linearize(h, n, n, P(T), P(p), P(Y), None, P(lin), n, sp))

        def per_entry(_):
            chk(L.nk_rates_jvp_linearized(h, n, n, P(T), P(p), P(Y), P(lin), n, P(vT), P(vY), P(dw), P(dh), sp))

        res["sweep_linearized_ms"] = t_l = timed(fwd_lin, per_entry)
        res["speedup_linearized_vs_fd"] = t_fd / t_l
        del lin
        torch.cuda.empty_cache()
    best = min((k for k in ("sweep_compact_ms", "sweep_linearized_ms", "sweep_recompute_ms") if k in res),
               key=lambda k: res[k])
    res["sweep_ms"] = res[best]
    res["sweep_form"] = best[len("sweep_"):-len("_ms")]
    res["speedup_vs_fd"] = t_fd / res[best]
    return res


# ---------------------------------------------------------------------------------- other configurations
def config_rows(nk, dev, stream):
    """Rates + transport of the other mechanisms, each launch through the C ABI, CUDA events on the
    launching stream around `reps` back-to-back launches (after 3 untimed ones):
      h2_9sp_21rx on 64 elements x 512 = 32,768 points (uniform states), FP64: inputs 2.9 MB, L2-resident,
        so the per-launch times include launch latency;
      h2_9sp_21rx on the 4,096-element flame field (2,097,152 points), FP64 and mixed: the paper's
        mechanism size at a production point count (its own figures are for this size);
      big_120sp_700rx on the 4,096-element flame field (2,097,152 points), FP64 and mixed.
    Results are keyed by mechanism, the 9-species production row as h2_9sp_21rx@flame_4096el."""
    import torch
    from paper_2409_06404_gb300 import synth
    L = nk.lib()
    sp = nk._vp(stream.cuda_stream)
    P = lambda t: nk._vp(t.data_ptr())
    res = {}
    for name, wl, reps, forms in (("h2_9sp_21rx", "uniform_64el", 50, ("fp64",)),
                                  ("h2_9sp_21rx", "flame_4096el", 20, ("fp64", "mixed")),
                                  ("big_120sp_700rx", "flame_4096el", 5, ("fp64", "mixed"))):
        mech = synth.mechanism(name)
        st = synth.workload_states(wl, mech.K)
        n, K = st.n, mech.K
        m = nk.mechanism_load(mech)
        T, p, Y = (torch.from_numpy(a).to(dev) for a in (st.T, st.p, st.Y))
        f64 = dict(dtype=torch.float64, device=dev)
        w, D = torch.empty((K, n), **f64), torch.empty((K, n), **f64)
        h, mu, lam = torch.empty(n, **f64), torch.empty(n, **f64), torch.empty(n, **f64)
        rec = {"points": n, "K": K, "R": mech.R, "workload": wl, "reps": reps}
        for form in forms:
            prec = nk._PRECISION[form]

            def rates():
                st_ = L.nk_rates_eval(m.handle, n, n, P(T), P(p), P(Y), None, P(w), P(h), prec, sp)
                if st_ != 0:
                    raise nk.NkError(st_, L.nk_last_error().decode())

            def trans():
                st_ = L.nk_transport_eval(m.handle, n, n, P(T), P(p), P(Y), P(mu), P(lam), P(D), prec, sp)
                if st_ != 0:
                    raise nk.NkError(st_, L.nk_last_error().decode())

            t = {}
            for key, f in (("rates", rates), ("transport", trans)):
                for _ in range(3):
                    f()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    f()
                b.record(stream)
                torch.cuda.synchronize()
                t[key] = a.elapsed_time(b) / reps
            rec[form] = {"rates_ms": t["rates"], "transport_ms": t["transport"],
                         "mpts": n / ((t["rates"] + t["transport"]) * 1e-3) / 1e6}
        m.close()
        del T, p, Y, w, D, h, mu, lam
        torch.cuda.empty_cache()
        res[name if name not in res else f"{name}@{wl}"] = rec
    return res


# ---------------------------------------------------------------------------------- reactor step
def reactor_states(nk, m, mech, n, dev, seed=6053, blend=0.0):
    """Near-equilibrium states for the implicit reactor step: chemical equilibria at 512
    temperatures in [1300, 2600] K and 1 atm from element potentials (X_k proportional to
    exp(-g_k/RT + sum_e lambda_e a_ek), normalised by a uniform shift found by bisection; g_k
    from nk_thermo_eval), tiled over the n points and perturbed by 1e-3 in Y and ~1 K in T.
    With blend > 0, Y = (1 - blend) Y_eq + blend Y_D with Y_D ~ Dirichlet(0.3) per point: the
    equilibria of the synthetic mechanisms hold most species near 1e-157, where chemistry is
    frozen; a blend of 1e-20 lifts them to ~1e-22 and the step has stiff chemistry to solve."""
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
    if blend > 0.0:
        g = torch.distributions.Gamma(torch.tensor(0.3, **f64), torch.tensor(1.0, **f64))
        torch.manual_seed(seed)
        D = g.sample((K, n)).to(dev)
        Y = (1.0 - blend) * Y + blend * D / D.sum(0)
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
                "converged": st["converged"], "ms_per_krylov_iter": ms / max(st["krylov_iters"], 1),
                "update_wrms": st["update_wrms"]}

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
    res["moving"] = reactor_moving_row(nk, m, mech, dev, stream)
    return res


def reactor_moving_row(nk, m, mech, dev, stream, n=65536, dt=1e-11, dt_hard=1e-10):
    """The block-Jacobi reactor step on states where chemistry moves: the near-equilibrium states
    blended with 1e-20 of a Dirichlet(0.3) composition (reactor_states), on n points (the Newton-
    Krylov solve over all points is global: the more points, the stiffer the hardest one it must
    resolve), each after one untimed step from the same states.  At dt the step converges in a
    few Newton iterations; at dt_hard (reported under "dt_hard") it takes 11-13 iterations and
    whether it meets the Newton tolerance within them turns on rounding (the factors' solve
    order has flipped it), so it is reported as measured."""
    import torch
    T0, p, Y0 = reactor_states(nk, m, mech, n, dev, blend=1e-20)
    kw = dict(rtol=1e-6, atol_T=1e-6, atol_Y=1e-12, newton_tol=1e-4, lin_tol=1e-6, max_newton=20, krylov_dim=30)
    ws = torch.empty(nk.reactor_workspace(m, n, kw["krylov_dim"], 1, 0), dtype=torch.uint8, device=dev)
    T, Y = T0.clone(), Y0.clone()

    def rows(step):
        res = {"dt_s": step}
        for name, precond in (("block_jacobi", 1), ("block_jacobi_reused", 2)):
            o = nk.reactor_opts(precond=precond, **kw)
            for _ in (0, 1):
                T.copy_(T0)
                Y.copy_(Y0)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st = nk.reactor_step(m, T, p, Y, step, o, workspace=ws)
                b.record(stream)
                torch.cuda.synchronize()
            wT = 1.0 / (kw["rtol"] * T0.abs() + kw["atol_T"])
            wY = 1.0 / (kw["rtol"] * Y0.abs() + kw["atol_Y"])
            chg = torch.sqrt((((T - T0) * wT) ** 2).sum() + (((Y - Y0) * wY) ** 2).sum()) / (((Y.shape[0] + 1) * n) ** 0.5)
            res[name] = {"ms": a.elapsed_time(b), "newton_iters": st["newton_iters"],
                         "krylov_iters": st["krylov_iters"], "converged": st["converged"],
                         "update_wrms": st["update_wrms"], "step_change_wrms": float(chg)}
        return res

    out = {"points": n, "states": "near-equilibrium states blended with 1e-20 of a Dirichlet(0.3) composition "
                                  "(species lifted from ~1e-157 to ~1e-22)"}
    out.update(rows(dt))
    out["dt_hard"] = rows(dt_hard)
    return out


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
    linc = torch.empty((nk.linearization_slots_compact(m), n), **f64)   # per-reaction form (~9.4 KB per point)
    gradX = torch.randn((3, K, n), generator=gen, **f64)         # mole-fraction gradients (synthetic)
    jflux = torch.empty((3, K, n), **f64)
    Vc = torch.empty((3, n), **f64)
    hflux = torch.empty((3, n), **f64)
    wsb = torch.empty(max(nk.rates_vjp_workspace(m, n), 8), dtype=torch.uint8, device=dev)
    # block-Jacobi preconditioner of the implicit stage: the sources at the state, the solver's
    # weights 1/(rtol |y| + atol), the LU factors (~23 KB per point) and one vector to solve for
    N1 = K + 1
    fTb, fYb = torch.empty(n, **f64), torch.empty((K, n), **f64)
    wts = torch.empty((N1, n), **f64)
    wts[0] = 1.0 / (1e-6 * T + 1e-6)
    wts[1:] = 1.0 / (1e-6 * Y + 1e-12)
    Fb = torch.empty((N1, N1, n), **f64)
    pivb = torch.empty((N1, n), dtype=torch.int32, device=dev)
    vb = torch.randn((N1, n), generator=gen, **f64)
    zb = torch.empty((N1, n), **f64)
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
        "linearize_compact": lambda: chk(L.nk_rates_linearize_compact(h, n, n, P(T), P(p), P(Y), None, P(linc), n,
                                                                      P(out["w"]), P(out["hrr"]), sp)),
        "jvp_linearized_compact": lambda: chk(L.nk_rates_jvp_linearized_compact(h, n, n, P(T), P(p), P(Y), P(linc),
                                                                                n, P(vT), P(vY), P(out["dw"]),
                                                                                P(out["dh"]), sp)),
        # (after "linearize": the factors are formed from the stored linearization)
        "block_factor": lambda: chk(L.nk_block_jacobi_factor(h, n, n, P(T), P(p), P(Y), P(lin), n, P(fTb), P(fYb),
                                                             P(wts), n, ctypes.c_double(1e-9), P(Fb), P(pivb), n,
                                                             sp)),
        "block_apply": lambda: chk(L.nk_block_jacobi_apply(h, n, P(Fb), P(pivb), n, P(vb), n, P(zb), n, sp)),
    }
    chk(L.nk_rhs_eval(h, n, n, P(T), P(p), P(Y), None, P(fTb), P(fYb), 0, sp))
    # the mechanism-specialised kernel is compiled (NVRTC) before any timing
    t_jit = time.perf_counter()
    nk.mechanism_jit(m)
    jit_compile_s = time.perf_counter() - t_jit
    launches_per_step = {"thermo": 1, "rates_fp64": 2, "transport_fp64": 1, "rates_mixed": 2,
                         "transport_mixed": 1, "jvp": 1, "vjp": 3}
    names = list(rows)

    for _ in range(args.warmup):
        for f in rows.values():
            f()
    torch.cuda.synchronize()
    peaks = pipe_peaks()
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

    # ---- the other mechanisms' configurations (not part of a step)
    configs = config_rows(nk, dev, s) if args.configs else None

    # ---- implicit reactor step (not part of a step)
    reactor = reactor_row(nk, m, mech, n, dev, s) if args.reactor else None

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

    # ---- implicit-stage sweep (not part of a step), after the workload's buffers are released
    stage = None
    if args.stage_dirs > 0:
        del lin, lin32, linc, gradX, jflux, Vc, hflux, out, wsb, vT, vY, wbar
        torch.cuda.empty_cache()
        if args.stage_elements in (0, args.elements):
            stage = implicit_stage(nk, m, T, p, Y, args.stage_dirs, 3, s)
        else:
            st5 = synth.workload_states("flame_32768el" if args.stage_elements == 32768 else WORKLOAD, K,
                                        n_elements=args.stage_elements)
            T5, p5, Y5 = (torch.from_numpy(a).to(dev) for a in (st5.T, st5.p, st5.Y))
            del st5
            stage = implicit_stage(nk, m, T5, p5, Y5, args.stage_dirs, 2, s)
            del T5, p5, Y5
        torch.cuda.empty_cache()
        stage["workload"] = f"{MECH} on {stage['points']} points"

    if rank != 0:
        return
    # ---- per-pipe rooflines of every row with committed pipe counts, and the dominant kernel's
    avg = {k: sum(v) / len(v) for k, v in ms.items() if k in names}
    avg_f = {k: sum(v) / len(v) for k, v in ms.items() if k in forms}
    both = {**avg, **avg_f}
    counts = pipe_counts()
    alg = algorithmic(MECH)
    rows_out = {}
    for k in names + list(forms):
        r = {"ms": both[k], "mpts": n / (both[k] * 1e-3) / 1e6}
        if k in counts:
            pp = row_pipes(counts[k], n, both[k], peaks)
            r["pipe_frac"] = {q: v["frac"] for q, v in pp.items()}
            r["pipe"] = max(pp, key=lambda q: pp[q]["frac"])
            r["frac"] = pp[r["pipe"]]["frac"]
        base = k.split("_")[0]
        if base in ("rates", "transport") and base in alg and k != "rates_jit":
            r["alg_tflops"] = alg[base]["flops"] * n / (both[k] * 1e-3) / 1e12
        if k == "block_apply":
            # algorithmic bytes: the factors (N^2 doubles), the pivot words, v read and z written
            N1 = K + 1
            bpp = N1 * N1 * 8 + N1 * 4 + 2 * N1 * 8
            r["bytes_per_point"] = bpp
            r["hbm_gbs"] = bpp * n / (both[k] * 1e-3) / 1e9
            r["hbm_frac_of_measured"] = r["hbm_gbs"] / hbm_peak_gbs() if hbm_peak_gbs() else None
        rows_out[k] = r
    dom = max(names, key=lambda k: avg[k])
    peak_src = ("measured in this run: libnkprobe.so, independent multiply-add streams on every SM "
                "(profiles/pipe_peaks_gb300.md has a committed run); MEASURED_PEAKS.json has no FP64 or "
                "FP32-pipe figure")
    if dom in counts:
        pp = row_pipes(counts[dom], n, avg[dom], peaks)
        bind = max(pp, key=lambda q: pp[q]["frac"])
        roof = {"bound": "alu", "kernel": dom, "pipe": bind, "achieved": pp[bind]["gops"],
                "peak": pp[bind]["peak_gops"], "unit": "Gop/s", "frac": pp[bind]["frac"], "traffic": _traffic(dom),
                "pipes": pp, "peak_source": peak_src,
                "basis": "pipe operations per point (ncu warp instructions of the row's kernels x 32 lanes, "
                         "profiles/pipe_counts.json) x points / CUDA-event time of the launch, against the "
                         "pipe's multiply-add rate; frac = the largest over the FP64 and FMA pipes"}
    else:
        roof = {"bound": "alu", "kernel": dom, "pipe": None, "achieved": None, "peak": peaks["dfma"] / 1e9,
                "unit": "Gop/s", "frac": None, "traffic": _traffic(dom), "peak_source": peak_src,
                "basis": "no pipe counts for the current sources of this kernel"}
    roof["algorithmic"] = {"source": "profiles/algorithmic_ops.json (oracle's instrumented scalar)",
                           "per_point": alg}
    fwd_avg = avg["rates_fp64"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{MECH} (53 species, 325 reactions: 20 third-body, 25 Troe) on {WORKLOAD}: "
                               f"{args.elements} elements x 512 GLL points = {n} points, FP64 SoA",
                   "mechanism": MECH, "points": n, "value_basis": "points / (rates_fp64 + transport_fp64 time)",
                   "step": names, "forms_after_steps": list(forms),
                   "l2": "inputs (0.92 GB) larger than L2; no flush",
                   "arithmetic": "FP64 form (NK_FP64): exponent chains (ln k_f, the Gibbs and enthalpy sums, ln K_c, "
                                 "the Troe falloff chain, the third-body sums, the logarithms of the concentration "
                                 "products) and all of transport in double-float "
                                 "pairs (48-bit) on the FP32 pipe; the rate terms' values, the forward-minus-reverse "
                                 "differences and every accumulation in double; results within 1e-10 of the FP64 "
                                 "definitions.  The all-double form is fp64_native_value"},
        "mixed_value": mixed_value,
        "fp64_native_value": native_value,
        "vjp_over_fwd": avg["vjp"] / fwd_avg, "jvp_over_fwd": avg["jvp"] / fwd_avg,
        "rows": rows_out,
        "roofline": roof,
        "pipe_peaks_gops": {k: v / 1e9 for k, v in peaks.items()},
        "fp64_tflops_measured": 2.0 * peaks["dfma"] / 1e12, "fp64_tflops_nominal": FP64_NOMINAL_TFLOPS,
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
    if configs is not None:
        line["configs"] = configs
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
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the 9- and 120-species configuration rows")
    ap.add_argument("--stage-dirs", type=int, default=10,
                    help="JVP directions of the implicit-stage sweep (0 skips it)")
    ap.add_argument("--stage-elements", type=int, default=32768,
                    help="elements of the implicit-stage field (a cube; 32768 = 16,777,216 points, the "
                         "implicit-stage workload; 0 = the benchmark field)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
