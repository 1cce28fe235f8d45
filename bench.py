"""Benchmark: gradient evaluations per second of the Paraexp direct-adjoint loop on GB300.

One step = one full direct-adjoint loop (direct solve, adjoint solve, objective and
gradient) through the C ABI of libpxa, inputs resident in HBM.

Default workload (the 1D viscous Burgers configuration): n = 1024, nu = 0.005,
T = 2, classical RK4 with dt = 1e-4 (K = 20000 steps), FP64, forcing control with
random Fourier coefficients (k <= 16), tracking objective against a seeded target,
P = 32 subintervals; the direct problem is serial, the adjoint is Paraexp (hybrid
scheme). ``--workload advdiff1d`` runs the 1D advection-diffusion configuration
(n = 256, CN with K = 4096, P = 8, Krylov m = 30).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gradient evals/s: batched Paraexp vs serial stepping, same GPU, rel.err<=1e-8"
FP64_PEAK_GFLOPS = 1250.0  # nominal dense FP64 of GB300 (1.25 TFLOP/s)
SMS = 152

WORKLOADS = {
    "burgers1d": dict(kind="burgers1d", n=1024, nu=0.005, T=2.0, K=20000, P=32, M=25, m=20,
                      tol=1e-9, checkpoints=5, label="1D viscous Burgers n=1024 nu=0.005 T=2 RK4 dt=1e-4 FP64 P=32"),
    "advdiff1d": dict(kind="advdiff1d", n=256, c=1.0, nu=0.01, T=1.0, K=4096, P=8, m=30, sub=1,
                      tol=1e-11, label="1D advection-diffusion n=256 nu=0.01 T=1 CN 4096 steps FP64 P=8 (Krylov m autotuned)"),
    "advdiff2d": dict(kind="advdiff2d", n=512, nu=1e-3, T=1.0, K=1024, P=64,
                      label="2D advection-diffusion 512x512 nu=1e-3 T=1 RK4 1024 steps FP32 stepping P=64"),
    "advdiff2d_lanes": dict(kind="lanes2d", n=2048, lanes=64, steps=10,
                            label="2D RK4 FP32 lanes kernel, 64 lanes x 2048^2 (1 GiB per state array)"),
    "advdiff1d_lanes": dict(kind="lanes1d", n=1 << 22, lanes=64, steps=10,
                            label="1D FP32 CN band lanes kernel, 64 lanes x 2^22 points (1 GiB per state array), "
                                  "c=1 nu=1e-6 dt=h/8 (21-tap band)"),
    "spmv_csr": dict(kind="spmv", n=1 << 25, label="CSR sparse matrix-vector product, the 1D advection-diffusion "
                                                    "stencil (c=1, nu=0.01) in CSR form, 2^25 rows x 3 entries, FP64"),
    "burgers2d": dict(kind="burgers2d", n=256, nu=2e-3, T=1.0, K=5120, P=128, lbfgs_iters=20,
                      label="2D viscous Burgers (u, v) 256x256 nu=2e-3 T=1 RK4 dt=1/5120 FP32 stepping P=128, "
                            "initial-state control, terminal tracking objective"),
    "batched1d": dict(kind="batched1d", count=256, c=1.0, T=1.0, K=4096, P=16,
                      label="256 independent 1D advection-diffusion problems, n ~ U{128..2048}, "
                            "nu ~ logU[1e-3, 1e-1], T=1 CN 4096 steps, P=16, FP32 stepping, "
                            "homogeneous parts by the FP32 band of M^(K/P), FP64 superposition"),
}
# FP32 peak from unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# Algorithmic FP64 operations per grid point per step of each kernel (counted from the
# kernels' arithmetic; the roofline divides them by the measured kernel time).
FLOPS_RK4_DIRECT = 48.0       # four stages of N(u) + s f (8 each), stage states and weights 13, J 3
FLOPS_BAND_PREPASS = 190.0    # stage states 36, Jacobian rows 28, tangent column of M_s 124, source 2
FLOPS_BAND_SWEEP = 18.0       # nine FMAs of a row of M_s^T
FLOPS_BAND_GRAD = 32.0        # transposed stage recursion kbar4..kbar1 and the weighted sum
FLOPS_RK4_ADJOINT = 109.0     # stage re-stepping adjoint: recompute 36, four transposed stages 70, source 3
FLOPS_RK4_ADJOINT_HOM = 106.0  # the same without the objective's source
FLOPS_CN_BAND_TAP = 2.0       # one FMA per tap of the circulant CN band per point per step
# FP64 warp instructions on one warp's path per step (the step-time floor is this count
# x 64 cycles: one FP64 warp instruction per 64 cycles per SM sub-partition on GB300)
FP64_INSTR_RK4_STEP = 27
FP64_INSTR_BAND_STEP = 9
SM_CLOCK_HZ = 2.07e9
# CTAs per thread-block cluster of the 1D advection-diffusion lane and band-chain kernels
# (fixed in the kernels: every lane and the chain run on one cluster of 8 CTAs)
AD1_LANE_CLUSTER = 8
AD1_CHAIN_CLUSTER = 8
# Method flops of one Crank-Nicolson step per grid point (the tridiagonal right-hand side
# 5, the periodic tridiagonal solve by Sherman-Morrison and Thomas 8): what the method
# computes, independent of how the library evaluates the step
FLOPS_CN_STEP = 13.0
GATE = 1e-8  # the metric's accuracy gate on FP64 gradients against the serial oracle

# DRAM bytes per launch from the committed ncu captures (profiles/*.md); None when the
# kernel changed after the capture.
TRAFFIC = {
    "ad1_chain_kernel": 82.7e3,
    "cn_lanes_kernel": 16128.0,
    "spmv_csr_kernel": 1744881408 + 257540352,
    # the direct solve is 8 chunk launches of 61.95 KB DRAM reads each (the trajectory
    # rows stay in L2 during the launch)
    "bu1_rk4_sweep_kernel": 8 * 61.95e3,  # the shared-memory form (grids with > 744 points per CTA)
    "bu1_rk4_wave_kernel": None,
    "bu1_band_sweep_kernel": 1.6407e9 + 0.1587e9,
    # the four-step chain: 4 segment launches of 348.8 MB read + 10.5 MB written each
    "bu1_band_chain4_kernel": 4 * (348767488.0 + 10518528.0),
    "bu1_band_prepass_kernel": 8 * (30.49e6 + 357.0e6),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="burgers1d", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="grid size override for the 2D workloads")
    ap.add_argument("--once", action="store_true",
                    help="profiling run: W warm-up gradients then one more of the headline "
                         "configuration (1D, batched and 2D workloads), default cluster sizes, no "
                         "autotuning")
    ap.add_argument("--K", type=int, default=0,
                    help="with --once on the 1D and 2D Burgers workloads: this many time steps at the "
                         "workload's dt (a shorter window for profiling captures)")
    ap.add_argument("--no-compare", dest="no_compare", action="store_true",
                    help="skip the Paraexp-against-serial comparison of the other workloads")
    ap.add_argument("--checkpoints", type=int, default=0,
                    help="with --once on the Burgers workload: the multi-checkpoint scheme with this many intervals")
    return ap.parse_args()


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.rows.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 2 + i and r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def reduce_max(x: float) -> float:
    """Max over the ranks of the process group (identity without one); NCCL reduces on
    the GPU, gloo on the host."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Replicas: every rank processes units_per_rank units; the job takes the slowest
    rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def rel_err(a, b):
    """Larger of the point-wise error relative to max|b| and the norm-wise relative error."""
    a, b = np.asarray(a, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()
    pw = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    nw = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    return max(pw, nw)


def gate_mark(err, tol=GATE):
    return None if err is None else ("pass" if err <= tol else "fail")


def make_inputs(w):
    from paper_2004_00546_gb300 import inputs as I

    if w["kind"] == "burgers1d":
        p = I.burgers1d_problem(n=w["n"])
        return {"control": p["f"], "target": p["g"]}
    p = I.advdiff1d_problem(n=w["n"])
    return {"control": p["q0"]}


def make_ctx(X, w, phi):
    ctx = X.Context()
    if w["kind"] == "burgers1d":
        ctx.set_operator(X.BURGERS_1D, w["n"], nu=w["nu"])
        ctx.set_time(w["T"], w["K"], X.RK4, w["P"])
        ctx.set_krylov(w["m"], w["tol"], phi, 1)
        ctx.set_magnus(w["M"])
    else:
        ctx.set_operator(X.ADVDIFF_1D, w["n"], c=w["c"], nu=w["nu"])
        ctx.set_time(w["T"], w["K"], X.CN, w["P"])
        ctx.set_krylov(w["m"], w["tol"], phi, w["sub"])
    return ctx


def oracle_gradient(w, inp, K=None):
    """Serial FP64 oracle (the plain definition of the discrete gradient)."""
    import oracle as O

    K = w["K"] if K is None else K
    T = w["T"] * K / w["K"]
    if w["kind"] == "burgers1d":
        J, g = O.bu1_gradient_serial(inp["control"], inp["target"], w["nu"], T, K)
    else:
        J, g, _ = O.ad1_cn_gradient_serial(inp["control"], w["c"], w["nu"], T, K)
    return J, g


def time_mode(X, torch, ctx, mode, steps, warmup, flush, timing=False):
    """Per-step CUDA-event times (ms) on the context's stream, L2 flushed between steps."""
    n = ctx.n
    grad = torch.empty(n, dtype=torch.float64, device="cuda")
    Jd = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ctx.set_timing(timing)  # phase events, captured in the graph with the kernels
    ctx.set_graph(True)
    for _ in range(warmup):
        ctx.gradient(mode, grad)
    times, phases = [], []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.gradient_async(mode, Jd, grad)
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.sync()  # also reads the phase events of the step (timing on)
        times.append(e0.elapsed_time(e1))
        if timing:
            phases.append(ctx.stats())
    return times, phases, grad


def time_pair(X, torch, make, steps, warmup, flush):
    """Paraexp and serial stepping of one workload timed the same way: the same steps and
    warm-up, graph replays, L2 flushed before every step, CUDA events on the context's
    stream. make(mode) returns a configured context. Returns {name: (mean ms, gradient)}."""
    out = {}
    for name, mode in (("paraexp", X.PARAEXP), ("serial", X.SERIAL)):
        ctx = make(mode)
        times, _, g = time_mode(X, torch, ctx, mode, steps, warmup, flush)
        out[name] = (float(np.mean(times)), g.detach().cpu().numpy())
        ctx.close()
    return out


def mode_phase_means(X, torch, make, flush, steps=3):
    """Phase times (ms, CUDA events on the streams each phase runs on) of each mode,
    averaged over a few graph replays after the timed pair."""
    out = {}
    for name, mode in (("paraexp", X.PARAEXP), ("serial", X.SERIAL)):
        ctx = make(mode)
        _, phs, _ = time_mode(X, torch, ctx, mode, steps, 1, flush, timing=True)
        out[name] = {k: float(np.mean([p[k] for p in phs])) for k in
                     ("ms_direct_inhom", "ms_direct_hom", "ms_adjoint_prep", "ms_adjoint_inhom", "ms_adjoint_hom",
                      "ms_total")}
        ctx.close()
    return out


def speedup_model(scheme, ph, T, P, T_H=None):
    """The paper's speedup formulas with the rates measured on this GPU (time per unit of
    simulated time, from the phase times of each mode).

    linear (Alg. 1, Eq. LinSpeedup): s^-1 = 1/P + (P-1)/P (tau_H + tau_H')/(tau_I + tau_I'),
    tau_I, tau_I' from serial stepping (its direct and adjoint sweeps over [0, T]), tau_H,
    tau_H' from the Paraexp chains (spanning T (P-1)/P). The formula assumes P lanes each
    as fast as one serial sweep; `lanes_efficiency` is that ideal (T/P)(tau_I + tau_I')
    over the measured lane time.
    hybrid (Sec. 3.3, Eq. hybridSpeedup): s^-1 = (T tau_I + (T/P) tau_I' + T_H tau_H') /
    (T (tau_I + tau_I')), with the serial direct's tau_I, the serial adjoint's tau_I' and
    the Paraexp chain's tau_H' over its span T_H; its limit for many subintervals is
    (tau_I + tau_I')/(tau_I + tau_H')."""
    par, ser = ph["paraexp"], ph["serial"]
    out = {"scheme": scheme, "measured": ser["ms_total"] / par["ms_total"] if par["ms_total"] > 0 else None}
    if scheme == "linear":
        tI, tIa = ser["ms_direct_inhom"] / T, ser["ms_adjoint_inhom"] / T
        span = T * (P - 1) / P
        tH, tHa = par["ms_direct_hom"] / span, par["ms_adjoint_hom"] / span
        inv = 1.0 / P + (P - 1) / P * (tH + tHa) / (tI + tIa)
        lanes = par["ms_direct_inhom"] + par["ms_adjoint_inhom"]
        out.update({"tau_I": tI, "tau_I_adj": tIa, "tau_H": tH, "tau_H_adj": tHa, "predicted": 1.0 / inv,
                    "limit": (tI + tIa) / (tH + tHa) if tH + tHa > 0 else None,
                    "lanes_efficiency": (T / P) * (tI + tIa) / lanes if lanes > 0 else None})
    else:
        tI = ser["ms_direct_inhom"] / T
        tIa = (ser["ms_total"] - ser["ms_direct_inhom"]) / T
        T_H = T if T_H is None else T_H
        tHa = par["ms_adjoint_hom"] / T_H
        inv = (T * tI + (T / P) * tIa + T_H * tHa) / (T * (tI + tIa))
        out.update({"tau_I": tI, "tau_I_adj": tIa, "tau_H_adj": tHa, "T_H": T_H, "predicted": 1.0 / inv,
                    "limit": (tI + tIa) / (tI + tHa)})
    out["units"] = "tau: ms of GPU time per unit of simulated time"
    return out


def pair_entry(label, res, g_ref, tol, note):
    """One workload of the Paraexp-against-serial comparison."""
    pe, se = rel_err(res["paraexp"][1], g_ref), rel_err(res["serial"][1], g_ref)
    return {"workload": label, "paraexp_ms": res["paraexp"][0], "serial_ms": res["serial"][0],
            "speedup": res["serial"][0] / res["paraexp"][0], "rel_err_paraexp": pe, "rel_err_serial": se,
            "tolerance": tol, "gate": gate_mark(pe, tol), "note": note}


def compare_advdiff1d(args, X, torch, flush):
    """C1: Paraexp with the stepper's subinterval propagator as one circulant band per link
    against serial stepping (both with the lanes on the band of M^4), and Paraexp with the
    autotuned Krylov propagator; errors against the serial FP64 oracle."""
    w = WORKLOADS["advdiff1d"]
    inp = make_inputs(w)
    ctl = torch.as_tensor(inp["control"], device="cuda")

    def make(mode, prop=X.PROP_BAND):
        ctx = make_ctx(X, w, X.PHI_STEPPER)
        ctx.set_control(ctl)
        if mode == X.PARAEXP and prop == X.PROP_BAND:
            ctx.set_propagator(X.PROP_BAND, 150)
        return ctx

    res = time_pair(X, torch, make, args.steps, args.warmup, flush)
    _, g_ref = oracle_gradient(w, inp)
    e = pair_entry(w["label"].replace(" (Krylov m autotuned)", ""), res, g_ref, GATE,
                   "homogeneous parts: the stepper's subinterval propagator M^(K/P) as one circulant band "
                   "per link (exact for this periodic constant-coefficient operator)")
    e["phases_ms"] = mode_phase_means(X, torch, make, flush)
    e["speedup_model"] = speedup_model("linear", e["phases_ms"], w["T"], w["P"])
    # the benchmark spec's Krylov propagator, autotuned (m, substeps), timed the same way
    ctx = make(X.PARAEXP, X.PROP_KRYLOV)
    ctx.autotune(X.PARAEXP, torch.empty(w["n"], dtype=torch.float64, device="cuda"))
    st = ctx.stats()
    times, _, g = time_mode(X, torch, ctx, X.PARAEXP, args.steps, args.warmup, flush)
    ctx.close()
    ek = rel_err(g.cpu().numpy(), g_ref)
    e["paraexp_krylov"] = {"ms": float(np.mean(times)), "speedup": e["serial_ms"] / float(np.mean(times)),
                           "rel_err": ek, "gate": gate_mark(ek), "krylov_m": st["krylov_m"],
                           "krylov_substeps": st["krylov_substeps"]}
    return e


def compare_batched(args, X, torch, flush):
    """C4: 256 problems of uneven size; Paraexp (stepper's propagator as a band of M^(K/P),
    FP32) against serial stepping, and Paraexp with every homogeneous part by the FP64
    Krylov exponential; errors against the FP64 oracle on sampled problems."""
    import oracle as O
    from paper_2004_00546_gb300 import inputs as I

    w = WORKLOADS["batched1d"]
    prob = I.batch1d_problem(count=w["count"], seed=2007)
    cnt, K, P, off = w["count"], w["K"], w["P"], prob["offsets"]
    q0 = torch.as_tensor(prob["q0"], device="cuda")
    J = torch.empty(cnt, dtype=torch.float64, device="cuda")
    g = torch.empty_like(q0)
    order = np.argsort(-prob["n"])
    stiff = np.argsort(-(prob["nu"] * prob["n"] ** 2))
    sample = list(dict.fromkeys(list(order[:4]) + list(stiff[:4])))

    def timed(b, mode):
        for _ in range(args.warmup):
            b.gradient(mode, q0, J, g)
        t = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.gradient_async(mode, q0, J, g)
            e1.record()
            torch.cuda.synchronize()
            b.sync()
            t.append(e0.elapsed_time(e1))
        return float(np.mean(t)), g.cpu().numpy()

    def timed_once(b, mode):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.gradient_async(mode, q0, J, g)
        e1.record()
        torch.cuda.synchronize()
        b.sync()
        return float(e0.elapsed_time(e1)), g.cpu().numpy()

    out = {}
    kry_setting = None
    for name, mode, ratio in (("paraexp", X.PARAEXP, None), ("paraexp_phases", X.PARAEXP, None),
                              ("serial", X.SERIAL, None), ("paraexp_krylov_fp64", X.PARAEXP, 1e30)):
        b = X.Batch()
        b.set(prob["n"], prob["nu"], c=w["c"], T=w["T"], K=K, P=P)
        b.set_schedule(0 if name == "paraexp_phases" else 1)
        if ratio is None:
            b.set_power(True)
            if mode == X.PARAEXP:
                b.autotune(mode, q0, J, g)
            out[name] = timed(b, mode) + (b.problem_info()[2],)
        else:
            # every homogeneous part by the Krylov exponential: the first (m, substep reach)
            # whose a-posteriori estimates meet the 1e-8 tolerance on every problem
            b.set_homogeneous(ratio)
            # (seconds per gradient: the stiff problems need up to ~75 substeps per link, so
            # it is timed on one step after the trial gradient that checks the estimates)
            for m, reach in ((48, 0.01), (48, 0.005)):
                b.set_krylov(m, 1e-8, reach)
                try:
                    b.gradient(mode, q0, J, g)
                except X.PxaError as e:
                    if e.code != X.ERR_NOT_CONVERGED:
                        raise
                    continue
                kry_setting = {"krylov_m": m, "krylov_reach": reach,
                               "substeps_max": b.stats()["substeps_max"], "timed_steps": 1}
                out[name] = timed_once(b, mode) + (b.problem_info()[2],)
                break
        b.close()
    errs = {}
    if "paraexp_krylov_fp64" not in out:
        out["paraexp_krylov_fp64"] = (float("nan"), None, None)
    for name, (_, gh, kry) in out.items():
        if gh is None:
            errs[name] = None
            continue
        e = []
        for i in (sample if name != "paraexp_krylov_fp64" else sample[:4]):
            q = prob["q0"][off[i]:off[i + 1]]
            if kry[i]:
                _, go, _ = O.ad1_cn_gradient_paraexp(q, w["c"], prob["nu"][i], w["T"], K, P, O.PHI_EXP)
            else:
                _, go, _ = O.ad1_cn_gradient_serial(q, w["c"], prob["nu"][i], w["T"], K)
            e.append(rel_err(gh[off[i]:off[i + 1]], go))
        errs[name] = max(e)
    tol = 5e-4  # FP32 stepping: 2 K u_32 for K = 4096 (the full-size test's bound)
    entry = {"workload": w["label"], "paraexp_ms": out["paraexp"][0], "serial_ms": out["serial"][0],
             "speedup": out["serial"][0] / out["paraexp"][0], "rel_err_paraexp": errs["paraexp"],
             "rel_err_serial": errs["serial"], "tolerance": tol, "gate": gate_mark(errs["paraexp"], tol),
             "sample": "8 problems (the 4 largest grids, the 4 stiffest); errors against the FP64 oracle",
             "paraexp_phases_ms": out["paraexp_phases"][0], "rel_err_paraexp_phases": errs["paraexp_phases"],
             "schedule": "one persistent launch with device-side dependencies (paraexp_phases_ms: seven launches)",
             "note": "FP32 stepping; the homogeneous parts use the stepper's own propagator M^(K/P) as one "
                     "FP32 circulant band per link (not FP64 Krylov); FP64 superposition",
             "paraexp_krylov_fp64": {"ms": None if kry_setting is None else out["paraexp_krylov_fp64"][0],
                                     "speedup": None if kry_setting is None else
                                     out["serial"][0] / out["paraexp_krylov_fp64"][0],
                                     "rel_err": errs["paraexp_krylov_fp64"], "setting": kry_setting,
                                     "sample": "the 4 largest grids, against the oracle's Paraexp with exp(tau A)",
                                     "note": "every homogeneous part by the FP64 Krylov exponential exp(tau A) "
                                             "(the paper's propagator), FP32 lanes"}}
    return entry


def compare_advdiff2d(args, X, torch, flush):
    """C3: the hybrid scheme (serial FP32 direct, Paraexp adjoint) against serial stepping
    of both. The Paraexp adjoint's homogeneous chain runs either as exact transposed RK4
    steps (the stepper chain) or as the power series of the stepper's subinterval
    propagator (PXA_PROP_POLY: about m operator applications per subinterval instead of
    4 K/P); the faster of the two within the FP32 tolerance of serial stepping is the
    entry's Paraexp time. The full-size FP64 oracle takes about 700 s on one core, so the
    entry gives the difference of the GPU gradients (the tests hold them to the oracle at
    8^2-120^2 and to each other at this size)."""
    w = WORKLOADS["advdiff2d"]
    res, info = {}, {}
    for name, mode, prop in (("paraexp_stepper", X.PARAEXP, None), ("paraexp_poly", X.PARAEXP, X.PROP_POLY),
                             ("serial", X.SERIAL, None)):
        ctx, keep = ctx_2d(X, torch, w, w["n"], w["P"], w["K"])
        if prop is not None:
            ctx.set_propagator(prop, 200)
        times, _, g = time_mode(X, torch, ctx, mode, args.steps, args.warmup, flush)
        res[name] = (float(np.mean(times)), g.detach().cpu().numpy())
        st = ctx.stats()
        info[name] = {"degree": st["prop_degree"], "segments_per_subinterval": st["prop_substeps"],
                      "tail_bound": st["prop_tail"]}
        ctx.close()
        del keep
    d = {k: rel_err(res[k][1], res["serial"][1]) for k in ("paraexp_stepper", "paraexp_poly")}
    ok = [k for k in d if d[k] <= 1e-4]
    head = min(ok, key=lambda k: res[k][0]) if ok else "paraexp_stepper"

    def make(mode):
        c2, kp = ctx_2d(X, torch, w, w["n"], w["P"], w["K"])
        if mode == X.PARAEXP and head == "paraexp_poly":
            c2.set_propagator(X.PROP_POLY, 200)
        c2._keep = kp
        return c2

    phases = mode_phase_means(X, torch, make, flush)
    return {"workload": w["label"], "paraexp_ms": res[head][0], "serial_ms": res["serial"][0],
            "speedup": res["serial"][0] / res[head][0], "homogeneous": head, "rel_err_paraexp": None,
            "rel_err_serial": None, "rel_diff_paraexp_vs_serial": d[head], "tolerance": 1e-4,
            "gate": gate_mark(d[head], 1e-4),
            "paraexp_stepper_chain": {"ms": res["paraexp_stepper"][0], "rel_diff_vs_serial": d["paraexp_stepper"],
                                      "speedup": res["serial"][0] / res["paraexp_stepper"][0]},
            "paraexp_poly_chain": dict(info["paraexp_poly"], ms=res["paraexp_poly"][0],
                                       rel_diff_vs_serial=d["paraexp_poly"],
                                       speedup=res["serial"][0] / res["paraexp_poly"][0]),
            "phases_ms": phases,
            # the chain spans the P-1 lower subintervals (the top one is a lane)
            "speedup_model": speedup_model("hybrid", phases, w["T"], w["P"], T_H=w["T"] * (w["P"] - 1) / w["P"]),
            "note": "FP32 stepping, FP64 accumulation; the FP64 oracle at full size is not run here"}


def bu2_setup(X, torch, w):
    """The 2D Burgers context with the target made from the seeded true initial state."""
    from paper_2004_00546_gb300 import inputs as I

    p = I.burgers2d_problem(n=w["n"])
    ctx = X.Context()
    ctx.set_operator_burgers_2d(w["n"], w["nu"])
    ctx.set_time(w["T"], w["K"], X.RK4, w["P"])
    ic_true = torch.as_tensor(p["true_ic"], device="cuda")
    target = torch.empty_like(ic_true)
    ctx.direct_state(ic_true, target)
    ctx.set_target(target)
    x = torch.as_tensor(p["other_ic"], device="cuda")
    ctx.set_control(x)
    return ctx, {"target": target, "x": x, "p": p}


def compare_burgers2d(args, X, torch, flush):
    """C5: with the terminal objective the hybrid scheme's adjoint lanes have no source, so
    the Paraexp and serial gradients run the same kernels; timed the same way."""
    w = WORKLOADS["burgers2d"]
    ctx, keep = bu2_setup(X, torch, w)
    res = {}
    for name, mode in (("paraexp", X.PARAEXP), ("serial", X.SERIAL)):
        times, _, g = time_mode(X, torch, ctx, mode, max(3, args.steps // 4), args.warmup, flush)
        res[name] = (float(np.mean(times)), g.detach().cpu().numpy())
    ctx.close()
    d = rel_err(res["paraexp"][1], res["serial"][1])
    return {"workload": w["label"], "paraexp_ms": res["paraexp"][0], "serial_ms": res["serial"][0],
            "speedup": res["serial"][0] / res["paraexp"][0], "rel_err_paraexp": None, "rel_err_serial": None,
            "rel_diff_paraexp_vs_serial": d, "tolerance": 4 * w["K"] * 2.0 ** -24,
            "gate": gate_mark(d, 4 * w["K"] * 2.0 ** -24),
            "note": "terminal objective: the adjoint lanes vanish, Paraexp = serial by construction; FP32 stepping; "
                    "the FP64 oracle at full size is not run here (the tests hold both to it at 16^2-48^2 and check "
                    "the full size by central differences)"}


def run_bu2(args, w, rank, world):
    """2D viscous Burgers: one gradient (direct + adjoint) per step, then the 20-iteration
    L-BFGS loop of the configuration (outside the timed region), reporting J per iteration."""
    import torch

    from paper_2004_00546_gb300 import build, lbfgs, pxa as X

    build.build()
    X.load()
    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    ctx, keep = bu2_setup(X, torch, w)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    with ClockSampler(dev_index) as clk:
        times, _, g = time_mode(X, torch, ctx, X.PARAEXP, args.steps, args.warmup, flush)
    _, phases, _ = time_mode(X, torch, ctx, X.PARAEXP, 3, 1, flush, timing=True)
    total_ms = reduce_max(float(sum(times)))
    ph = {k: float(np.mean([p[k] for p in phases])) for k in ("ms_direct_inhom", "ms_adjoint_hom", "ms_total")}
    graph_kernels = ctx.stats()["graph_kernels"]  # kernels of the timed graph replays
    # end to end through the host-buffer entry point
    ctx.set_timing(False)
    n2 = 2 * w["n"] * w["n"]
    xh = np.ascontiguousarray(keep["p"]["other_ic"])
    gh = np.empty(n2)
    ctx.gradient_host(X.PARAEXP, xh, gh)
    te = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.gradient_host(X.PARAEXP, xh, gh)
        te.append(time.perf_counter() - t0)
    # the configuration's optimisation loop from the zero initial state
    t0 = time.perf_counter()
    res = lbfgs.minimize(ctx, torch.zeros(n2, dtype=torch.float64, device="cuda"), iters=w["lbfgs_iters"],
                         mode=X.PARAEXP)
    t_lbfgs = time.perf_counter() - t0
    # FLOPs per point per step: direct 4 stages x 2 fields x ~15 + stage states and weights
    # ~20 = 140; adjoint: 3 recomputed stages ~100 + 4 transposed Jacobians x 2 fields x ~22 ~ 180
    pts = w["n"] * w["n"]
    flop = (140.0 + 280.0) * pts * w["K"]
    ach = flop / (ph["ms_total"] * 1e-3) / 1e12
    cpu = {}
    if rank == 0:
        import oracle as O

        Ks = 4
        p = keep["p"]
        n = w["n"]
        q = p["other_ic"]
        tgt = keep["target"].cpu().numpy()
        t1 = time.perf_counter()
        O.bu2_gradient_serial(q[:n * n].reshape(n, n), q[n * n:].reshape(n, n), tgt[:n * n].reshape(n, n),
                              tgt[n * n:].reshape(n, n), w["nu"], w["T"] * Ks / w["K"], Ks)
        dt_cpu = (time.perf_counter() - t1) * w["K"] / Ks
        cpu = {"value": 1.0 / dt_cpu, "unit": "gradient evals/s", "cores": 1, "kind": "oracle",
               "sample": f"scaled sample: the first {Ks} of {w['K']} steps (direct + adjoint), scaled by {w['K']}/{Ks}"}
    line = {"metric": METRIC, "value": whole_job_rate(args.steps, world, total_ms), "unit": "gradient evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 stepping, f64 objective", "data": "synthetic (seeded Fourier fields, amplitude 0.15)",
            "config": {"workload": w["label"], "l2": "flushed between steps (256 MiB write)"},
            "phases_ms": ph,
            "roofline": {"bound": "alu", "kernel": "bu2_step_kernel + bu2_adj_step_kernel (one launch per step each)",
                         "unit": "TFLOP/s", "peak": FP32_PEAK_TFLOPS, "achieved": ach, "frac": ach / FP32_PEAK_TFLOPS,
                         "traffic": None, "peak_kind": "FP32 from unit counts and clocks",
                         "note": "latency-bound: 10240 launches of 256 tiles per gradient"},
            "lbfgs": {"iterations": len(res.J) - 1, "J": res.J, "grad_norm": res.grad_norm, "evals": res.evals,
                      "seconds": t_lbfgs, "J_ratio": res.J[-1] / res.J[0]},
            "cpu_baseline": cpu,
            "e2e": {"value": world / float(np.mean(te)), "unit": "gradient evals/s", "h2d_bytes_per_step": 8 * n2,
                    "d2h_bytes_per_step": 8 * n2 + 8},
            "clocks": clk.summary(),
            "gpu_launches": (graph_kernels * args.steps) if graph_kernels > 0 else (2 * w["K"] + 6) * args.steps}
    ctx.close()
    return line


def run_ours(args, w, rank, world):
    import torch

    from paper_2004_00546_gb300 import build, pxa as X

    build.build()
    X.load()
    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    inp = make_inputs(w)
    ctl = torch.as_tensor(inp["control"], device="cuda")
    tgt = torch.as_tensor(inp["target"], device="cuda") if "target" in inp else None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    variants = {}
    phis = [("paraexp_stepper", X.PARAEXP, X.PHI_STEPPER), ("paraexp_exp", X.PARAEXP, X.PHI_EXP),
            ("serial", X.SERIAL, X.PHI_STEPPER)]
    if w["kind"] == "advdiff1d":
        # the paper's own homogeneous propagator, the real Leja points method, for exp
        # and for the CN power (which keeps Paraexp equal to serial stepping)
        phis.insert(2, ("paraexp_exp_relpm", X.PARAEXP, X.PHI_EXP))
        phis.insert(0, ("paraexp_stepper_relpm", X.PARAEXP, X.PHI_STEPPER))
        # the subinterval propagator itself as a circulant band (exact for this periodic
        # constant-coefficient operator): exp(tau A), and the CN power M^(K/P)
        phis.insert(3, ("paraexp_exp_band", X.PARAEXP, X.PHI_EXP))
        phis.insert(0, ("paraexp_stepper_band", X.PARAEXP, X.PHI_STEPPER))
    if w["kind"] == "burgers1d":
        # the multi-checkpoint scheme (Sec. 3.5): C + 1 checkpoints, every interval re-stepped
        # and solved by the Paraexp adjoint over its own P subintervals (not a headline
        # candidate: it trades a second direct pass for memory)
        phis.append((f"checkpoints{w['checkpoints']}_paraexp_stepper", X.PARAEXP, X.PHI_STEPPER))
    grads = {}
    tuned = {}
    for name, mode, phi in phis:
        ctx = make_ctx(X, w, phi)
        ctx.set_control(ctl)
        if tgt is not None:
            ctx.set_target(tgt)
        best_ms = None
        ctx.set_graph(True)  # candidates are timed as graph replays, the path timed below
        if name.startswith("checkpoints"):
            ctx.set_checkpoints(w["checkpoints"])
        if name.endswith("_relpm"):
            ctx.set_propagator(X.PROP_RELPM, 150)
        elif name.endswith("_band"):
            ctx.set_propagator(X.PROP_BAND, 150)
        elif not (w["kind"] == "burgers1d" and phi == X.PHI_EXP):
            # autotuner (outside any timed region): Krylov m / substeps, or cluster sizes
            best_ms = ctx.autotune(mode, torch.empty(w["n"], dtype=torch.float64, device="cuda"))
        st = ctx.stats()
        tuned[name] = {"krylov_m": st["krylov_m"], "krylov_substeps": st["krylov_substeps"],
                       "clusters": [st["cluster_direct"], st["cluster_lanes"], st["cluster_chain"]],
                       "groups": [st["group_direct"], st["group_sweep"]],
                       "partition_r": round(float(st["partition_r"]), 6),
                       "tau_ratio": round(float(st["tau_ratio"]), 6),
                       "autotune_best_ms": best_ms}
        times, _, g = time_mode(X, torch, ctx, mode, max(1, min(args.steps, 3)), 1, flush)
        variants[name] = {"ms_per_step": float(np.mean(times)), "mode": name, "tuned": tuned[name],
                          "workspace_bytes": int(ctx.stats()["workspace_bytes"])}
        grads[name] = g.detach().cpu().numpy()
        ctx.close()

    # accuracy of each variant against the serial FP64 oracle (one full gradient)
    cpu = {}
    if rank == 0:
        t0 = time.perf_counter()
        J_ref, g_ref = oracle_gradient(w, inp)
        dt_cpu = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt_cpu, "unit": "gradient evals/s", "cores": 1, "kind": "oracle",
               "sample": f"one full serial FP64 gradient of the {w['kind']} workload ({dt_cpu:.2f} s)"}
        for name in variants:
            variants[name]["rel_err"] = rel_err(grads[name], g_ref)
            variants[name]["gate_1e-8"] = gate_mark(variants[name]["rel_err"])

    # the headline: fastest Paraexp variant whose gradient meets rel.err <= 1e-8
    ok = [k for k in variants if k.startswith("paraexp") and variants[k].get("rel_err", 0.0) <= 1e-8]
    head = min(ok, key=lambda k: variants[k]["ms_per_step"]) if ok else "paraexp_stepper"
    phi = X.PHI_EXP if head.startswith("paraexp_exp") else X.PHI_STEPPER
    ctx = make_ctx(X, w, phi)
    ctx.set_control(ctl)
    if tgt is not None:
        ctx.set_target(tgt)
    tv = tuned[head]
    if w["kind"] == "advdiff1d" and head.endswith("_relpm"):
        ctx.set_krylov(w["m"], w["tol"], phi, w["sub"])
        ctx.set_propagator(X.PROP_RELPM, 150)
    elif w["kind"] == "advdiff1d" and head.endswith("_band"):
        ctx.set_krylov(w["m"], w["tol"], phi, w["sub"])
        ctx.set_propagator(X.PROP_BAND, 150)
    elif w["kind"] == "advdiff1d":
        ctx.set_krylov(tv["krylov_m"], w["tol"], phi, tv["krylov_substeps"])
    else:
        ctx.set_cluster(*tv["clusters"])
        ctx.set_groups(*tv["groups"])
        ctx.set_partition(tv["partition_r"])

    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev_index) as clk:
        times, _, _ = time_mode(X, torch, ctx, X.PARAEXP, args.steps, args.warmup, flush)
    total_ms = reduce_max(float(sum(times)))
    value = whole_job_rate(args.steps, world, total_ms)
    _, phases, _ = time_mode(X, torch, ctx, X.PARAEXP, max(2, min(args.steps, 3)), 1, flush, timing=True)
    phases_source = "phase events of graph replays after the timed region (the timed replays record none)"
    if any(p["ms_total"] < 0 for p in phases):
        # phase events could not be read from the graph: take them from launches without a
        # graph, after the timed region
        ctx.set_timing(True)
        ctx.set_graph(False)
        phases = []
        for _ in range(max(2, min(args.steps, 3))):
            flush.zero_()
            ctx.gradient(X.PARAEXP, torch.empty(w["n"], dtype=torch.float64, device="cuda"))
            phases.append(ctx.stats())
        phases_source = "phase events of separate runs without a graph (after the timed region)"

    # end to end through the host-buffer entry point: H2D of the control, D2H of the gradient
    ctx.set_timing(False)
    ctx.set_graph(True)
    gh = np.empty(w["n"])
    ch = np.ascontiguousarray(inp["control"])
    ctx.gradient_host(X.PARAEXP, ch, gh)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.gradient_host(X.PARAEXP, ch, gh)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": world / float(np.mean(e2e_t)), "unit": "gradient evals/s",
           "h2d_bytes_per_step": 8 * w["n"], "d2h_bytes_per_step": 8 * w["n"] + 8}

    # Paraexp against serial stepping on every workload of the metric, each pair timed the
    # same way (steps, warm-up, L2 flush); errors against the FP64 oracle
    comparison = None
    if w["kind"] == "burgers1d" and not args.no_compare:
        _, g_ref = oracle_gradient(w, inp) if rank == 0 else (None, None)

        def make_bu(mode):
            c2 = make_ctx(X, w, X.PHI_STEPPER)
            c2.set_control(ctl)
            c2.set_target(tgt)
            tvv = tuned["paraexp_stepper" if mode == X.PARAEXP else "serial"]
            c2.set_cluster(*tvv["clusters"])
            c2.set_groups(*tvv["groups"])
            c2.set_partition(tvv["partition_r"])
            return c2

        res = time_pair(X, torch, make_bu, args.steps, args.warmup, flush)
        # plain serial stepping: the adjoint takes one transposed step per exchange (no
        # product records), timed the same way
        c1 = make_bu(X.SERIAL)
        c1.set_adjoint(X.ADJ_BANDED_SINGLE)
        t1, _, g1 = time_mode(X, torch, c1, X.SERIAL, args.steps, args.warmup, flush)
        c1.close()
        one_step = (float(np.mean(t1)), g1.detach().cpu().numpy())
        # the phases of each mode (events on the streams each phase runs on), after the pair
        mode_phases = {}
        for name, mode in (("paraexp", X.PARAEXP), ("serial", X.SERIAL)):
            c2 = make_bu(mode)
            _, phs, _ = time_mode(X, torch, c2, mode, 3, 1, flush, timing=True)
            mode_phases[name] = {k2: float(np.mean([p2[k2] for p2 in phs])) for k2 in
                                 ("ms_direct_inhom", "ms_adjoint_prep", "ms_adjoint_hom", "ms_total",
                                  "ms_side_prepass", "ms_side_pair", "ms_side_quad", "ms_side_lanes")}
            c2.close()
        comparison = {}
        if rank == 0:
            comparison["C2"] = pair_entry(
                w["label"], res, g_ref, GATE,
                "hybrid scheme: serial RK4 direct in both modes; the time-varying homogeneous adjoint is "
                "carried by the stepper's own transposed step maps, so its chain sweeps all K steps like the "
                "serial adjoint")
            comparison["C2"]["phases_ms"] = mode_phases
            # the banded chain covers the top subinterval too (with its source): T_H = T
            comparison["C2"]["speedup_model"] = speedup_model("hybrid", mode_phases, w["T"], w["P"], T_H=w["T"])
            comparison["C2"]["serial_one_step_ms"] = one_step[0]
            comparison["C2"]["rel_err_serial_one_step"] = rel_err(one_step[1], g_ref)
            comparison["C2"]["speedup_vs_one_step"] = one_step[0] / res["paraexp"][0]
            comparison["C2"]["serial_note"] = (
                "serial_ms: serial RK4 direct, adjoint chain on four-step product records built beside "
                "the direct (the fastest serial form here); serial_one_step_ms: the adjoint one transposed "
                "step at a time")
            comparison["C1"] = compare_advdiff1d(args, X, torch, flush)
            comparison["C3"] = compare_advdiff2d(args, X, torch, flush)
            comparison["C4"] = compare_batched(args, X, torch, flush)
            comparison["C5"] = compare_burgers2d(args, X, torch, flush)

    # roofline of the dominant kernel, from the per-phase CUDA events of the timed steps
    ph = {k: float(np.mean([p[k] for p in phases])) for k in
          ("ms_direct_inhom", "ms_direct_hom", "ms_adjoint_prep", "ms_adjoint_inhom",
           "ms_adjoint_hom", "ms_total", "ms_side_prepass", "ms_side_pair", "ms_side_quad",
           "ms_side_lanes")}
    side_chunks = int(phases[-1]["side_chunks"]) if phases else 0
    st = ctx.stats()
    n, K, P = w["n"], w["K"], w["P"]
    k = K // P
    floors = {}
    if w["kind"] == "burgers1d":
        cl = ctx.cluster_sizes()
        # the direct: the register-wavefront form runs when a CTA's chunk (n / cluster size)
        # has at most 744 points, else the shared-memory form
        direct = "bu1_rk4_wave_kernel" if (n + cl[0] - 1) // cl[0] <= 744 else "bu1_rk4_sweep_kernel"
        kernels = {
            # name: (ms per launch, algorithmic FP64 flop per launch, SMs used, DRAM bytes per launch)
            direct: (ph["ms_direct_inhom"], FLOPS_RK4_DIRECT * n * K, cl[0], TRAFFIC.get(direct)),
        }
        floors[direct] = K * FP64_INSTR_RK4_STEP * 64 / SM_CLOCK_HZ * 1e3
        if st["adjoint_band"] and side_chunks > 0:
            # overlapped with the direct chunks on the side streams: kernel times from
            # events recorded on those streams, summed over the chunks
            kernels["bu1_band_prepass_kernel"] = (ph["ms_side_prepass"], FLOPS_BAND_PREPASS * n * (K + 1),
                                                  SMS, TRAFFIC.get("bu1_band_prepass_kernel"))
            kernels["bu1_band_pair_kernel + bu1_band_quad_kernel"] = (
                ph["ms_side_pair"] + ph["ms_side_quad"],
                (2.0 * 9 * 9 + 18) * n * K / 2 + (2.0 * 17 * 17 + 34) * n * K / 4, SMS, None)
            kernels["bu1_band_sweep_kernel (lanes)"] = (ph["ms_side_lanes"], FLOPS_BAND_SWEEP * n * (K - k),
                                                        (P - 1) * cl[1], None)
        elif st["adjoint_band"]:
            kernels["bu1_band_prepass_kernel"] = (ph["ms_adjoint_prep"], FLOPS_BAND_PREPASS * n * (K + 1),
                                                  SMS, TRAFFIC.get("bu1_band_prepass_kernel"))
            kernels["bu1_band_sweep_kernel (lanes)"] = (ph["ms_adjoint_inhom"], FLOPS_BAND_SWEEP * n * K,
                                                        P * cl[1], None)
        if st["adjoint_band"]:
            if head == "paraexp_stepper":
                # the chain phase: bu1_band_chain4_kernel in 4 segments (four-step entries,
                # 33 taps = 66 flop per point per 4 steps) with the fill of the skipped rows
                kernels["bu1_band_chain4_kernel (chain)"] = (ph["ms_adjoint_hom"], 66.0 / 4 * n * K, cl[2],
                                                             TRAFFIC.get("bu1_band_chain4_kernel"))
        else:
            kernels["bu1c_adjoint_lanes_kernel"] = (ph["ms_adjoint_inhom"], FLOPS_RK4_ADJOINT * n * K,
                                                    P * cl[1], None)
            if head == "paraexp_stepper":
                kernels["bu1c_stepper_chain_kernel"] = (ph["ms_adjoint_hom"],
                                                        FLOPS_RK4_ADJOINT_HOM * n * k * (P - 1), cl[2], None)
        if head != "paraexp_stepper":
            kernels["bu1_magnus_chain_kernel"] = (ph["ms_adjoint_hom"], None, 1, None)
    else:
        m, sub = st["krylov_m"], st["krylov_substeps"]
        arnoldi = (8 * m + 4 * m * (m + 1) + 2 * m) * n  # operator, CGS2, norms, combine
        dense = 2 * (m ** 3) * (1 + int(np.log2(k // sub)))  # solve + squarings
        # the band chain: P - 1 links of one band product (2 flop per tap and point)
        band_flop = 2.0 * st["prop_band_taps"] * n * (P - 1)
        chain = {"band": ("ad1_band_chain_kernel", band_flop), "relpm": ("ad1_relpm_chain_kernel", None)}.get(
            head.rsplit("_", 1)[-1], ("ad1_chain_kernel", (P - 1) * sub * (arnoldi + dense)))
        chain_sms = AD1_CHAIN_CLUSTER if chain[0] == "ad1_band_chain_kernel" else 1
        kernels = {
            chain[0]: (0.5 * (ph["ms_direct_hom"] + ph["ms_adjoint_hom"]), chain[1], chain_sms,
                       TRAFFIC.get(chain[0])),
            # the lanes apply the band of M^q (lane_band_taps taps) k/q times per lane; each
            # lane is one cluster of AD1_LANE_CLUSTER CTAs
            "cn_lanes_kernel": (0.5 * (ph["ms_direct_inhom"] + ph["ms_adjoint_inhom"]),
                                FLOPS_CN_BAND_TAP * st["lane_band_taps"] * n * (k // max(st["lane_steps"], 1)) * P,
                                P * AD1_LANE_CLUSTER, TRAFFIC.get("cn_lanes_kernel")),
        }
    dom = max(kernels, key=lambda kk: kernels[kk][0])
    ms_dom, flops, sms_used, traffic = kernels[dom]
    peak_tf = FP64_PEAK_GFLOPS / 1e3
    roof = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s", "peak": peak_tf,
            "peak_kind": "nominal FP64 of GB300 (1.25 TFLOP/s; 152 SMs x 2 FP64 FMA/clk)",
            "traffic": traffic, "ms_per_launch": ms_dom, "sms_used": sms_used}
    if flops is not None and ms_dom > 0:
        ach = flops / (ms_dom * 1e-3) / 1e12
        roof.update({"achieved": ach, "frac": ach / peak_tf,
                     "frac_of_used_sms": ach / (peak_tf * sms_used / SMS),
                     "flop_per_launch": flops})
    else:
        roof.update({"achieved": None, "frac": None})
    if dom in floors:
        # serial-chain floor: FP64 instructions per step on one warp's path x 64 cycles
        roof.update({"issue_floor_ms": floors[dom], "frac_of_issue_floor": floors[dom] / ms_dom})
    roof["kernels_ms"] = {kk: v[0] for kk, v in kernels.items()}

    # kernels one graph replay (one timed gradient) launches: the kernel nodes of the
    # captured graph, as the library counted them
    launches_per_step = st["graph_kernels"] if st["graph_kernels"] > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": "gradient evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64 fields shaped like the paper's workloads)",
        "config": {"workload": w["label"], "homogeneous": head, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "variants": variants, "phases_ms": ph, "phases_source": phases_source, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "paraexp_vs_serial": comparison,
        "clocks": clk.summary(),
        "gpu_launches": None if launches_per_step is None else launches_per_step * args.steps,
    }
    ctx.close()
    return line


def run_batch_once(args, w):
    """W warm-up gradients and one more of the batched workload in each mode (Paraexp
    with the stepper's subinterval propagator applied as one band of M^(K/P), then
    serial), launched one by one with phase events, for ncu: no autotuner."""
    import torch

    from paper_2004_00546_gb300 import build, inputs as I, pxa as X

    build.build()
    X.load()
    prob = I.batch1d_problem(count=w["count"], seed=2007)
    q0 = torch.as_tensor(prob["q0"], device="cuda")
    J = torch.empty(w["count"], dtype=torch.float64, device="cuda")
    g = torch.empty_like(q0)
    out = {"once": w["label"], "warmup": args.warmup}
    for name, mode in (("paraexp", X.PARAEXP), ("serial", X.SERIAL)):
        b = X.Batch()
        b.set(prob["n"], prob["nu"], c=w["c"], T=w["T"], K=w["K"], P=w["P"])
        b.set_homogeneous(0.0)
        b.set_timing(True)  # (the one-launch schedule records only the whole gradient)
        for _ in range(args.warmup + 1):
            b.gradient(mode, q0, J, g)
        st = b.stats()
        out[name] = {k: st[k] for k in ("ms_lanes", "ms_chains", "ms_adjoint_lanes", "ms_adjoint_chains",
                                        "ms_total", "lanes_grid", "band32_max", "power_problems",
                                        "band_power_max")}
        b.close()
    return out


def run_once(args, w):
    """W warm-up gradients and one more (Paraexp, stepper propagator; for the 1D
    advection-diffusion workload as one circulant band of M^(K/P) per link), for ncu: the
    kernels of gradient W+1 are the launches after the first W of each name."""
    import torch

    from paper_2004_00546_gb300 import build, pxa as X

    build.build()
    X.load()
    inp = make_inputs(w)
    ctl = torch.as_tensor(inp["control"], device="cuda")
    ctx = make_ctx(X, w, X.PHI_STEPPER)
    if w["kind"] == "advdiff1d":
        ctx.set_propagator(X.PROP_BAND, 150)  # the fastest variant that meets the 1e-8 gate
    if w["kind"] == "burgers1d" and args.checkpoints:
        ctx.set_checkpoints(args.checkpoints)
    ctx.set_control(ctl)
    if "target" in inp:
        ctx.set_target(torch.as_tensor(inp["target"], device="cuda"))
    ctx.set_timing(True)
    grad = torch.empty(w["n"], dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.gradient(X.PARAEXP, grad)
    J = ctx.gradient(X.PARAEXP, grad)
    st = ctx.stats()
    ctx.close()
    return {"once": w["label"], "J": J, "warmup": args.warmup,
            "phases_ms": {k: st[k] for k in ("ms_direct_inhom", "ms_direct_hom", "ms_adjoint_prep",
                                             "ms_adjoint_inhom", "ms_adjoint_hom", "ms_total")},
            "clusters": [st["cluster_direct"], st["cluster_lanes"], st["cluster_chain"]]}


def run_once_2d(args, w):
    """2D advection-diffusion for ncu: W warm-up gradients and one more (Paraexp, the chain by
    the stepper propagator's power series), no graph, so every kernel is its own launch."""
    import torch

    from paper_2004_00546_gb300 import build, pxa as X

    build.build()
    X.load()
    n = args.n or w["n"]
    ctx, keep = ctx_2d(X, torch, w, n, w["P"], w["K"])
    ctx.set_propagator(X.PROP_POLY, 200)
    ctx.set_timing(True)
    grad = torch.empty(n * n, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.gradient(X.PARAEXP, grad)
    J = ctx.gradient(X.PARAEXP, grad)
    st = ctx.stats()
    ctx.close()
    del keep
    return {"once": w["label"], "J": J, "warmup": args.warmup, "degree": st["prop_degree"],
            "phases_ms": {k: st[k] for k in ("ms_direct_inhom", "ms_adjoint_inhom", "ms_adjoint_hom", "ms_total")}}


def run_once_bu2(args, w):
    """2D Burgers for ncu: W warm-up gradients and one more (K from --K to shorten the
    window), no graph, so every kernel is its own launch."""
    import torch

    from paper_2004_00546_gb300 import build, pxa as X

    build.build()
    X.load()
    ctx, keep = bu2_setup(X, torch, w)
    ctx.set_timing(True)
    grad = torch.empty(2 * w["n"] * w["n"], dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.gradient(X.PARAEXP, grad)
    J = ctx.gradient(X.PARAEXP, grad)
    st = ctx.stats()
    ctx.close()
    del keep
    return {"once": w["label"], "K": w["K"], "J": J, "warmup": args.warmup,
            "phases_ms": {k: st[k] for k in ("ms_direct_inhom", "ms_adjoint_hom", "ms_total")}}


def run_reference_batch(args, w, world):
    """The reference arm of the batched workload: the serial FP64 oracle of a bounded
    sample of the problems per step, scaled to the whole batch."""
    import oracle as O
    from paper_2004_00546_gb300 import inputs as I

    prob = I.batch1d_problem(count=w["count"], seed=2007)
    off, cnt, ns = prob["offsets"], w["count"], 4

    def step():
        for i in range(ns):
            O.ad1_cn_gradient_serial(prob["q0"][off[i]:off[i + 1]], w["c"], prob["nu"][i], w["T"], w["K"])

    for _ in range(args.warmup):
        step()
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        t.append(time.perf_counter() - t0)
    per_full = float(np.mean(t)) * cnt / ns
    value = cnt / per_full
    unit = "gradient evals/s (problems x gradients)"
    sample = (f"scaled sample: each timed step is the first {ns} of {cnt} problems (serial FP64 CN); "
              f"value = {cnt} / (sample time x {cnt}/{ns})")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(t)) * 1e3,
            "ms_per_step_kind": "measured time of one sampled step", "ms_per_batch_scaled": per_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["label"]},
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_spmv(args, w, world):
    """The reference arm of the SpMV workload: the oracle's CSR product on the first 2^21
    rows per step (bounded sample), as GB/s of the same algorithmic bytes per row."""
    import oracle as O

    n, m = w["n"], 1 << 21
    h = 2.0 * np.pi / n
    am, a0, ap = 1.0 / (2 * h) + 0.01 / h ** 2, -2 * 0.01 / h ** 2, -1.0 / (2 * h) + 0.01 / h ** 2
    i = np.arange(m)
    col = np.stack([(i - 1) % n, i, (i + 1) % n], 1).ravel().astype(np.int32)
    val = np.tile([am, a0, ap], m)
    rp = np.arange(0, 3 * m + 1, 3, dtype=np.int64)
    x = np.random.default_rng(2004).standard_normal(n)
    for _ in range(args.warmup):
        O.spmv_csr(rp, col, val, x)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.spmv_csr(rp, col, val, x)
        t.append(time.perf_counter() - t0)
    per_row = (8.0 + 12.0 * 3 + 16.0)  # bytes per row, as the GPU line counts them
    value = per_row * m / float(np.mean(t)) / 1e9
    sample = f"scaled sample: each timed step is the product of the first {m} of {n} rows"
    return {"impl": "reference", "metric": "HBM GB/s of the CSR sparse matrix-vector product", "value": value,
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(t)) * 1e3, "ms_per_step_kind": "measured time of one sampled step",
            "ms_per_product_scaled": float(np.mean(t)) * 1e3 * n / m, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": w["label"]},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_bu2(args, w, world):
    """The reference arm of the 2D Burgers workload: the serial FP64 oracle's gradient over
    the first K_s steps per timed step (the cost is linear in the number of steps), with
    the target made by the oracle from the true initial state over the same steps."""
    import oracle as O
    from paper_2004_00546_gb300 import inputs as I

    n, Ks = w["n"], 16
    p = I.burgers2d_problem(n=n)
    T_s = w["T"] * Ks / w["K"]
    sq = lambda a: (a[:n * n].reshape(n, n), a[n * n:].reshape(n, n))
    tU, tV = O.bu2_direct(*sq(p["true_ic"]), w["nu"], T_s, Ks)
    for _ in range(args.warmup):
        O.bu2_gradient_serial(*sq(p["other_ic"]), tU, tV, w["nu"], T_s, Ks)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.bu2_gradient_serial(*sq(p["other_ic"]), tU, tV, w["nu"], T_s, Ks)
        t.append(time.perf_counter() - t0)
    per_full = float(np.mean(t)) * w["K"] / Ks
    value = 1.0 / per_full
    sample = (f"scaled sample: each timed step is the first {Ks} of {w['K']} time steps (direct + adjoint); "
              f"value = 1 / (sample time x {w['K']}/{Ks})")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "gradient evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(t)) * 1e3,
            "ms_per_step_kind": "measured time of one sampled step", "ms_per_gradient_scaled": per_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["label"]},
            "cpu_baseline": {"value": value, "unit": "gradient evals/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "gradient evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args, w, rank, world):
    """The reference arm: the serial FP64 CPU oracle, timed on this host's cores."""
    if rank != 0:
        return None
    if w["kind"] == "batched1d":
        return run_reference_batch(args, w, world)
    if w["kind"] in ("lanes1d", "lanes2d"):
        return {"impl": "reference", "unavailable": "a single-kernel HBM stress measurement with no gradient; "
                                                    "the oracle has no counterpart kernel to time"}
    if w["kind"] == "spmv":
        return run_reference_spmv(args, w, world)
    if w["kind"] == "burgers2d":
        return run_reference_bu2(args, w, world)
    inp = make_inputs(w)
    # bounded sample per step: the first K_s steps of the window (direct + adjoint);
    # the cost is linear in the number of steps, so throughput scales by K_s / K
    K_s = max(w["P"], min(w["K"], 2000))
    while w["K"] % K_s:
        K_s -= 1
    for _ in range(args.warmup):
        oracle_gradient(w, inp, K_s)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_gradient(w, inp, K_s)
        t.append(time.perf_counter() - t0)
    per_full = float(np.mean(t)) * w["K"] / K_s
    value = 1.0 / per_full
    sample = (f"scaled sample: each timed step is the first {K_s} of {w['K']} time steps (direct + adjoint); "
              f"value = 1 / (sample time x {w['K']}/{K_s}), the cost being linear in the steps")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "gradient evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(t)) * 1e3, "ms_per_step_kind": "measured time of one sampled step",
            "ms_per_gradient_scaled": per_full * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["label"]},
            "cpu_baseline": {"value": value, "unit": "gradient evals/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "gradient evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def inputs_2d(n):
    from paper_2004_00546_gb300 import inputs as I

    u, v = I.streamfunction_velocity(n, n, 8, 2006)
    x = I.grid1d(n)
    X, Y = np.meshgrid(x, x)
    return u, v, np.ones((n, n)), np.sin(X) * np.sin(Y)


def ctx_2d(X, torch, w, n, P, K):
    u, v, f, ft = inputs_2d(n)
    keep = [torch.as_tensor(a.reshape(-1), device="cuda") for a in (u, v, f, ft)]
    ctx = X.Context()
    ctx.set_operator_2d(n, n, keep[0], keep[1], w.get("nu", 1e-3))
    ctx.set_time(w.get("T", 1.0), K, X.RK4, P)
    ctx.set_krylov(20, 1e-10, X.PHI_STEPPER, 1)
    ctx.set_control(keep[2], 1.0)
    ctx.set_target(keep[3])
    return ctx, keep


def run_lanes2d(args, w):
    """HBM roofline of the 2D FP32 RK4 lanes kernel (TMA halo tiles) at a size far
    above L2: algorithmic bytes = lanes * n^2 * (4 read + 4 write) per step."""
    import torch

    from paper_2004_00546_gb300 import build, pxa as X

    build.build()
    n = args.n or w["n"]
    lanes, steps = w["lanes"], max(args.steps, 2)
    ctx, keep = ctx_2d(X, torch, {"nu": 1e-3, "T": 1.0}, n, 1, 1024)
    for _ in range(max(args.warmup, 1)):
        ctx.rk4_lanes_2d(lanes, 2)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms = ctx.rk4_lanes_2d(lanes, steps)
    alg = lanes * n * n * 8.0 * steps
    peak = measured_hbm_peak()
    gbs = alg / (ms * 1e-3) / 1e9
    return {"metric": "HBM GB/s of the 2D FP32 RK4 lanes kernel", "value": gbs, "unit": "GB/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": w["label"].replace("2048", str(n)), "lanes": lanes},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None, "peak_kind": "measured copy bandwidth"},
            "clocks": clk.summary(), "gpu_launches": steps}


def run_lanes1d(args, w):
    """HBM roofline of the 1D FP32 CN band lanes kernel with its states in global memory,
    at a size far above L2: algorithmic bytes = lanes * n * (4 read + 4 write) per step.
    c = 1, nu = 1e-6, dt = h/8: the CN band then holds 21 taps, like the 1D
    advection-diffusion workload's (n = 256, nu = 0.01, dt = 1/4096)."""
    import torch

    from paper_2004_00546_gb300 import build, inputs as I, pxa as X

    build.build()
    X.load()
    n, lanes, steps = w["n"], w["lanes"], max(args.steps, 2)
    h = 2.0 * np.pi / n
    K = 1024
    ctx = X.Context()
    ctx.set_operator(X.ADVDIFF_1D, n, c=1.0, nu=1e-6)
    ctx.set_time(K * 0.125 * h, K, X.CN, 1)
    q0 = torch.as_tensor(I.grf_k2(n, 5), device="cuda")
    ctx.set_control(q0)
    for _ in range(max(args.warmup, 1)):
        ctx.cn_lanes_1d(lanes, 2)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms = ctx.cn_lanes_1d(lanes, steps)
    alg = lanes * n * 8.0 * steps
    peak = measured_hbm_peak()
    gbs = alg / (ms * 1e-3) / 1e9
    return {"metric": "HBM GB/s of the 1D FP32 CN band lanes kernel", "value": gbs, "unit": "GB/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": w["label"], "lanes": lanes},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None, "peak_kind": "measured copy bandwidth"},
            "clocks": clk.summary(), "gpu_launches": steps}


def run_spmv(args, w):
    """HBM roofline of the CSR sparse matrix-vector product at a size far above L2 (2 GB
    per product): algorithmic bytes = row pointers 8 (n + 1) + entries 12 nnz (int32
    column, FP64 value) + x 8 n (read once) + y 8 n. Sampled rows are checked against the
    oracle's definition, and the oracle is timed on the first 2^21 rows."""
    import torch

    import oracle as O
    from paper_2004_00546_gb300 import build, pxa as X

    build.build()
    X.load()
    n, c, nu = w["n"], 1.0, 0.01
    h = 2.0 * np.pi / n
    am, a0, ap = c / (2 * h) + nu / h ** 2, -2 * nu / h ** 2, -c / (2 * h) + nu / h ** 2
    i = torch.arange(n, device="cuda", dtype=torch.int64)
    col = torch.stack([(i - 1) % n, i, (i + 1) % n], 1).reshape(-1).to(torch.int32)
    val = torch.tensor([am, a0, ap], device="cuda", dtype=torch.float64).repeat(n)
    rp = torch.arange(0, 3 * n + 1, 3, device="cuda", dtype=torch.int64)
    gen = torch.Generator(device="cuda").manual_seed(2004)
    x = torch.randn(n, device="cuda", dtype=torch.float64, generator=gen)
    y = torch.empty_like(x)
    del i
    for _ in range(max(args.warmup, 3)):
        X.spmv_csr(rp, col, val, x, y)
    steps = max(args.steps, 3)
    times = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for _ in range(steps):  # the 2 GB operands do not fit in L2
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            X.spmv_csr(rp, col, val, x, y)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    nnz = 3 * n
    alg = 8.0 * (n + 1) + 12.0 * nnz + 16.0 * n
    gbs = alg / (ms * 1e-3) / 1e9
    peak = measured_hbm_peak()
    # parity on sampled rows and the oracle's time on a bounded sample
    xh, yh = x.cpu().numpy(), y.cpu().numpy()
    m = 1 << 21
    rph, colh, valh = rp[: m + 1].cpu().numpy(), col[: 3 * m].cpu().numpy(), val[: 3 * m].cpu().numpy()
    t0 = time.perf_counter()
    ref = O.spmv_csr(rph, colh, valh, xh)
    dt_cpu = time.perf_counter() - t0
    err = float(np.max(np.abs(yh[:m] - ref) / (np.abs(valh.reshape(m, 3)).sum(1) * np.abs(xh).max())))
    cpu = {"value": alg * m / n / dt_cpu / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"first {m} of {n} rows ({dt_cpu:.2f} s), the same bytes per row"}
    return {"metric": "HBM GB/s of the CSR sparse matrix-vector product", "value": gbs, "unit": "GB/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded normal x; the stencil's coefficients)",
            "config": {"workload": w["label"], "l2": "operands 2 GB, far above L2"},
            "rel_err_max_sampled": err,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "traffic": TRAFFIC.get("spmv_csr_kernel"), "peak_kind": "measured copy bandwidth",
                         "bytes_per_product": alg},
            "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": steps}


def measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def run_2d(args, w, rank, world):
    """2D advection-diffusion: serial FP32 stepping vs the hybrid Paraexp adjoint."""
    import torch

    from paper_2004_00546_gb300 import build, pxa as X

    build.build()
    n = args.n or w["n"]
    grad = torch.empty(n * n, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    variants, grads = {}, {}
    for name, mode, prop in (("paraexp_stepper", X.PARAEXP, None), ("paraexp_poly", X.PARAEXP, X.PROP_POLY),
                             ("serial", X.SERIAL, None)):
        ctx, keep = ctx_2d(X, torch, w, n, w["P"], w["K"])
        if prop is not None:
            ctx.set_propagator(prop, 200)
        times, _, g = time_mode(X, torch, ctx, mode, max(3, min(args.steps, 5)), 3, flush)
        variants[name] = {"ms_per_step": float(np.mean(times)), "mode": name}
        if prop is not None:
            st = ctx.stats()
            variants[name].update(degree=st["prop_degree"], segments_per_subinterval=st["prop_substeps"],
                                  tail_bound=st["prop_tail"])
        grads[name] = g.detach().cpu().numpy()
        ctx.close()
        del keep
    for name in ("paraexp_stepper", "paraexp_poly"):
        variants[name]["rel_diff_vs_gpu_serial"] = rel_err(grads[name], grads["serial"])
    ok = [k for k in ("paraexp_stepper", "paraexp_poly") if variants[k]["rel_diff_vs_gpu_serial"] <= 1e-4]
    head = min(ok, key=lambda k: variants[k]["ms_per_step"]) if ok else "paraexp_stepper"
    ctx, keep = ctx_2d(X, torch, w, n, w["P"], w["K"])
    if head == "paraexp_poly":
        ctx.set_propagator(X.PROP_POLY, 200)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        times, _, _ = time_mode(X, torch, ctx, X.PARAEXP, args.steps, args.warmup, flush)
    _, phases, _ = time_mode(X, torch, ctx, X.PARAEXP, 3, 1, flush, timing=True)
    ctx.set_timing(False)
    total_ms = float(sum(times))
    ph = {k: float(np.mean([p[k] for p in phases])) for k in
          ("ms_direct_inhom", "ms_direct_hom", "ms_adjoint_inhom", "ms_adjoint_hom", "ms_side_lanes")}
    # end to end through the host-buffer entry point: H2D of the forcing, D2H of the gradient
    u0, v0, f0, ft0 = inputs_2d(n)
    fh = np.ascontiguousarray(f0.reshape(-1))
    gh = np.empty(n * n)
    ctx.gradient_host(X.PARAEXP, fh, gh)
    te = []
    for _ in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.gradient_host(X.PARAEXP, fh, gh)
        te.append(time.perf_counter() - t0)
    e2e = {"value": world / float(np.mean(te)), "unit": "gradient evals/s", "h2d_bytes_per_step": 8 * n * n,
           "d2h_bytes_per_step": 8 * n * n + 8}
    # roofline of the dominant kernel, the serial direct's tile step (one launch per step):
    # algorithmic bytes per point and step = the state read and written and the stored
    # trajectory row (12 B); the state (1 MB at 512^2) is L2-resident, so this is latency-
    # bound work reported against HBM for reference
    K = w["K"]
    bytes_launch = 12.0 * n * n
    ms_launch = ph["ms_direct_inhom"] / K
    ach = bytes_launch / (ms_launch * 1e-3) / 1e9 if ms_launch > 0 else None
    peak = measured_hbm_peak()
    roof = {"bound": "hbm", "kernel": "ad2_rk4_kernel (serial direct, one RK4 step per launch)",
            "unit": "GB/s", "achieved": ach, "peak": peak, "frac": (ach / peak) if ach else None,
            "traffic": None, "bytes_per_launch": bytes_launch, "ms_per_launch": ms_launch,
            "peak_kind": "measured copy bandwidth",
            "note": "L2-resident state: latency-bound (290 tiles of 56 x 18, about two 8-warp blocks per SM); see the profiles"}
    cpu = {}
    if rank == 0:
        import oracle as O

        u, v, f, ft = inputs_2d(n)
        Ks = 16
        t0 = time.perf_counter()
        O.ad2_gradient_serial(f, ft, u, v, w["nu"], w["T"] * Ks / w["K"], Ks, omega=1.0)
        dt_cpu = (time.perf_counter() - t0) * w["K"] / Ks
        cpu = {"value": 1.0 / dt_cpu, "unit": "gradient evals/s", "cores": 1, "kind": "oracle",
               "sample": f"first {Ks} of {w['K']} steps (direct + adjoint), scaled by {Ks}/{w['K']}"}
    return {"metric": METRIC, "value": args.steps / (total_ms / 1e3), "unit": "gradient evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 stepping, f64 accumulation", "data": "synthetic",
            "config": {"workload": w["label"].replace("512x512", f"{n}x{n}"), "homogeneous": head,
                       "l2": "flushed between steps"},
            "variants": variants, "phases_ms": ph, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": (ctx.stats()["graph_kernels"] * args.steps) or None}


def run_batch(args, w, rank, world):
    """Many independent problems of uneven size (every phase one launch over the whole
    batch): Paraexp and serial stepping through pxa_batch_*, graph replay, L2 flushed."""
    import torch

    import oracle as O
    from paper_2004_00546_gb300 import build, inputs as I, pxa as X

    build.build()
    X.load()
    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    prob = I.batch1d_problem(count=w["count"], seed=2007)
    cnt, K, P = w["count"], w["K"], w["P"]
    q0 = torch.as_tensor(prob["q0"], device="cuda")
    J = torch.empty(cnt, dtype=torch.float64, device="cuda")
    g = torch.empty_like(q0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    off = prob["offsets"]
    # sample problems for the accuracy check: the four largest grids and four stiff ones
    order = np.argsort(-prob["n"])
    stiff = np.argsort(-(prob["nu"] * prob["n"] ** 2))
    sample = list(dict.fromkeys(list(order[:4]) + list(stiff[:4])))

    def timed(b, mode, steps, warmup):
        for _ in range(warmup):
            b.gradient(mode, q0, J, g)
        t = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            b.gradient_async(mode, q0, J, g)
            e1.record()
            torch.cuda.synchronize()
            b.sync()
            t.append(e0.elapsed_time(e1))
        return t

    variants, errs, bats = {}, {}, {}
    # Paraexp with the stepper's subinterval propagator as one band of M^(K/P) (default),
    # Paraexp with K/P CN steps per link instead, and serial stepping
    for name, mode, power, sched in (("paraexp", X.PARAEXP, True, 1), ("paraexp_phases", X.PARAEXP, True, 0),
                                     ("paraexp_stepped_links", X.PARAEXP, False, 1), ("serial", X.SERIAL, True, 1)):
        b = X.Batch()
        b.set(prob["n"], prob["nu"], c=w["c"], T=w["T"], K=K, P=P)
        b.set_power(power)
        b.set_schedule(sched)
        best = b.autotune(mode, q0, J, g) if mode == X.PARAEXP else None
        with ClockSampler(dev_index) as clk:
            t = timed(b, mode, args.steps, args.warmup)
        st = b.stats()
        Jh, gh = J.cpu().numpy(), g.cpu().numpy()
        e = []
        for i in sample:
            q = prob["q0"][off[i]:off[i + 1]]
            if mode == X.SERIAL:
                Jo, go, _ = O.ad1_cn_gradient_serial(q, w["c"], prob["nu"][i], w["T"], K)
            else:
                Jo, go, _ = O.ad1_cn_gradient_paraexp(q, w["c"], prob["nu"][i], w["T"], K, P, O.PHI_EXP)
            e.append(max(abs(Jh[i] - Jo) / Jo, float(np.linalg.norm(gh[off[i]:off[i + 1]] - go)
                                                      / np.linalg.norm(go))))
        variants[name] = {"ms_per_step": float(np.mean(t)), "min_ms": float(np.min(t)),
                          "rel_err_max_sampled": float(max(e)), "autotune_best_ms": best,
                          "krylov_m": st["krylov_m"], "krylov_reach": st["krylov_reach"],
                          "hom_ratio": st["hom_ratio"], "krylov_problems": st["krylov_problems"],
                          "substeps_max": st["substeps_max"], "lanes_grid": st["lanes_grid"],
                          "band32_max": st["band32_max"], "power_problems": st["power_problems"],
                          "band_power_max": st["band_power_max"], "lane_steps": st["lane_steps"],
                          "one_launch": st["one_launch"], "flow_grid": st["flow_grid"],
                          "clocks": clk.summary()}
        # kernels per gradient: sources, lanes, superposition, adjoint lanes, gradient, and
        # per direction one chain launch for each kind of homogeneous propagation in use
        kinds = sum(1 for c in (st["krylov_problems"], st["power_problems"],
                                cnt - st["krylov_problems"] - st["power_problems"]) if c > 0)
        variants[name]["kernels_per_step"] = (st["graph_kernels"] if st["graph_kernels"] > 0 else
                                              4 if mode == X.SERIAL else 1 if st["one_launch"] else 5 + 2 * kinds)
        bats[name] = b
    head = "paraexp"
    ms = variants[head]["ms_per_step"]
    value = whole_job_rate(cnt * args.steps, world, reduce_max(ms * args.steps))
    # roofline of the headline's dominant kernel, the Paraexp lanes: P x count lanes of
    # K/P CN steps taken as K/(P q) applications of the band of M^q, 2 flop per tap of
    # that band, point and application, i.e. 2 (K/q) sum_i n_i taps_i per direction. Its
    # duration comes from the phase events around the direct lanes' launch (with the
    # 0.03 ms source pass before it), in launches after the timed region.
    w32, _, _ = bats[head].problem_info()
    q = bats[head].stats()["lane_steps"]
    flop = 2.0 * 2.0 * (K / q) * float(np.sum(np.asarray(prob["n"], dtype=np.float64) * np.asarray(w32)))
    bp = bats["paraexp_phases"]
    bp.set_timing(True)
    lanes_ms = []
    for _ in range(3):
        flush.zero_()
        bp.gradient(X.PARAEXP, q0, J, g)
        lanes_ms.append(float(bp.stats()["ms_lanes"]))
    bp.set_timing(False)
    ms_lanes = float(np.median(lanes_ms))
    # the method's work: one CN step of every point of every lane, FLOPS_CN_STEP flop per
    # point and step; the P lanes of a problem take K/P steps each, K steps in all
    method_flop = FLOPS_CN_STEP * K * float(np.sum(np.asarray(prob["n"], dtype=np.float64)))
    achieved = method_flop / (ms_lanes / 1e3) / 1e12
    impl = 0.5 * flop / (ms_lanes / 1e3) / 1e12
    ms_ser = variants["serial"]["ms_per_step"]
    roof = {"bound": "alu", "kernel": "batch_cn_lanes_kernel (Paraexp lanes, one direction)",
            "unit": "TFLOP/s", "peak": FP32_PEAK_TFLOPS,
            "peak_kind": "FP32 from unit counts and clocks (152 SMs x 128 lanes x 2 flop x 2.07 GHz)",
            "achieved": achieved, "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
            "flop_per_launch": method_flop,
            "flop_kind": f"method flops: {FLOPS_CN_STEP:g} per point per CN step (tridiagonal right-hand side "
                         "and periodic tridiagonal solve), K steps per problem",
            "implementation_tflops": impl,
            "implementation_flop_kind": "2 flop per tap of the band of M^q per point and application",
            "ms_per_launch": ms_lanes, "cn_steps_per_band": q,
            "serial_lanes_tflops_implementation": flop / (ms_ser / 1e3) / 1e12}
    # end to end: pinned host q0 -> device, gradient, J and gradient back to pinned host
    qh = torch.as_tensor(prob["q0"]).pin_memory()
    gh = torch.empty(q0.numel(), dtype=torch.float64).pin_memory()
    Jhh = torch.empty(cnt, dtype=torch.float64).pin_memory()
    te = []
    for _ in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q0.copy_(qh, non_blocking=True)
        bp.gradient_async(X.PARAEXP, q0, J, g)
        gh.copy_(g, non_blocking=True)
        Jhh.copy_(J, non_blocking=True)
        torch.cuda.synchronize()
        bp.sync()
        te.append(time.perf_counter() - t0)
    for bb in bats.values():
        bb.close()
    cpu = {}
    if rank == 0:
        t0 = time.perf_counter()
        ns = 16
        for i in range(ns):
            O.ad1_cn_gradient_serial(prob["q0"][off[i]:off[i + 1]], w["c"], prob["nu"][i], w["T"], K)
        dt_cpu = (time.perf_counter() - t0) * cnt / ns
        cpu = {"value": cnt / dt_cpu, "unit": "gradient evals/s (problems x gradients)", "cores": 1,
               "kind": "oracle", "sample": f"first {ns} of {cnt} problems (serial FP64 CN), scaled by {cnt}/{ns}"}
    return {"metric": METRIC, "value": value, "unit": "gradient evals/s (problems x gradients)",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 stepping, f64 Krylov and superposition", "data": "synthetic",
            "config": {"workload": w["label"], "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "variants": variants, "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * cnt / float(np.mean(te)), "unit": "gradient evals/s (problems x gradients)",
                    "h2d_bytes_per_step": 8 * int(q0.numel()),
                    "d2h_bytes_per_step": 8 * int(q0.numel()) + 8 * cnt},
            "clocks": variants[head]["clocks"], "gpu_launches": variants[head]["kernels_per_step"] * args.steps}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        line = run_reference(args, w, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.once and w["kind"] in ("burgers1d", "advdiff1d"):
        if args.K:
            w = dict(w, K=args.K, T=w["T"] * args.K / w["K"])
        line = run_once(args, w)
    elif args.once and w["kind"] == "advdiff2d":
        line = run_once_2d(args, w)
    elif args.once and w["kind"] == "burgers2d":
        if args.K:
            w = dict(w, K=args.K, T=w["T"] * args.K / w["K"], P=min(w["P"], args.K))
        line = run_once_bu2(args, w)
    elif args.once and w["kind"] == "batched1d":
        line = run_batch_once(args, w)
    elif w["kind"] == "lanes2d":
        line = run_lanes2d(args, w)
    elif w["kind"] == "lanes1d":
        line = run_lanes1d(args, w)
    elif w["kind"] == "spmv":
        line = run_spmv(args, w)
    elif w["kind"] == "advdiff2d":
        line = run_2d(args, w, rank, world)
    elif w["kind"] == "batched1d":
        line = run_batch(args, w, rank, world)
    elif w["kind"] == "burgers2d":
        line = run_bu2(args, w, rank, world)
    else:
        line = run_ours(args, w, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
