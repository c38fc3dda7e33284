#!/usr/bin/env python3
"""Benchmark of the Line-DG hot path on GB300.

One step = one implicit BDF2 time level of the 2-D isentropic-vortex
workload (64 x 64 perturbed periodic quads on [0,10]^2, p = 4, Euler with
Roe flux, dt = 0.05) solved by Newton-GMRES(30) with the element-block
ILU(0) preconditioner to ||G|| <= 1e-8 ||G(U^n)||, with the Jacobian and
preconditioner rebuilt every step: every stage of the hot path (residual,
Jacobian assembly, preconditioner build, split matvec, ILU apply, GMRES
orthogonalisation, Newton update) runs in each step. The workload's stated
precision is FP64; the mixed-precision step (FP32 Jacobian/ILU/Krylov,
FP64 residual/update/refinement) is timed on the same data beside it.

value = DOF advanced per second over the whole job (all ranks).
Beside it (rank 0, one GPU): the paper's DIRK3 step on the same workload;
the 32^3, p=3 Navier-Stokes Taylor-Green vortex and the 64x32x32, p=4
walled channel at full size (kernels against the HBM roofline, one BDF2
level in mixed precision and in FP64); the learned Newton guess at 16^3.
`--impl reference` times the CPU oracle (the only other implementation of
the method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "residual+Jacobian DOF/s; implicit-step time mixed+learned vs FP64 @1e-8 res"
WORKLOAD = "euler2d_vortex_64x64_p4_bdf2_dt0.05_newton_gmres30_ilu0"
EQ = {"kind": "euler", "gamma": 1.4, "flux": "roe"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


FP64_NOMINAL_TFLOPS = 1.25   # nominal GB300 FP64 rate (context only; the roofline uses the measured rate)


def fp64_peak(torch, ldg, burst_reps=5, sustain_s=1.0):
    """Measured FP64 FMA rate of this GPU (ldg_fp64_fma_probe: FMA chains
    with no memory traffic, 4 blocks of 256 threads per SM), timed with CUDA
    events on the launching stream: `burst` = best of a few launches of
    about 5 ms, `sustained` = launches back to back for about a second.
    TFLOP/s at 2 FLOPs per FMA."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(4 * sms, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    ldg.ldg_fp64_fma_probe(64, sink)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, ms = 256, 0.0
    while True:   # size one launch to about 5 ms
        e0.record(st)
        fmas = ldg.ldg_fp64_fma_probe(iters, sink)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if ms > 4.0 or iters >= 1 << 20:
            break
        iters *= 2
    best = ms
    for _ in range(burst_reps):
        e0.record(st)
        ldg.ldg_fp64_fma_probe(iters, sink)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    n = max(2, int(sustain_s * 1e3 / best))
    e0.record(st)
    for _ in range(n):
        ldg.ldg_fp64_fma_probe(iters, sink)
    e1.record(st)
    e1.synchronize()
    sus = e0.elapsed_time(e1) / n
    return {"burst_tflops": 2 * fmas / (best * 1e-3) / 1e12, "sustained_tflops": 2 * fmas / (sus * 1e-3) / 1e12,
            "fmas_per_launch": fmas, "burst_ms": best, "sustained_launches": n,
            "how": "ldg_fp64_fma_probe: 16 independent FMA chains per thread, 4 x 256 threads per SM, no memory "
                   "traffic; CUDA events; burst = best of 5 launches of ~5 ms, sustained = back to back ~1 s"}


# ---------------------------------------------------------------------------
# algorithmic work per launch
# ---------------------------------------------------------------------------
def euler_residual_flops(D, p, nc, E):
    """FP64 operations of one first-order residual (divisions and square
    roots counted as one): per line interpolation, Gauss-point flux,
    contraction with M^-1 dPhi^T W, two Roe fluxes and their lifting."""
    N, NQ, NL = p + 1, (3 * p + 2) // 2, (p + 1) ** (D - 1)
    f_e = 7 * D + 7
    f_roe = 45 * D + 80
    per_line = NQ * nc * (2 * N - 1) + NQ * f_e + NQ * N * nc * 2 + 2 * (f_roe + N * nc * 2)
    return E * (D * NL * per_line + (p + 1) ** D * nc * (D + 1))


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# the timed kernels from one ncu capture of the unchanged kernels on this
# workload, every launch of one timed FP64 step (for the Gram-Schmidt
# sweeps, whose size varies with the basis: the mean over their launches);
# set to None when a kernel changes until it is captured again.
TRAFFIC = {"precond_apply": 121.47e6, "jacvec": 188.40e6, "gram_schmidt": 37.28e6}


def jac_bytes(h, esz):
    """Compulsory HBM bytes of one Jacobian assembly: the K11 (+K12) values
    written plus the state read."""
    return h.ntiles * 32 * (h.nk11 + h.nk12) * esz + h.ndof * 8


def jacvec_bytes(h, esz, vsz):
    """One split matvec: matrix values read once, x read, y written."""
    return h.ntiles * 32 * (h.nk11 + h.nk12) * esz + 2 * h.ndof * vsz


def apply_bytes(h, esz, vsz):
    """ILU(0) apply: the Dp off-diagonal factor blocks of every row and the
    inverted diagonal block read (the stored diagonal U blocks are not),
    r read, z written."""
    W = h.D * h.p + 1
    return h.E * h.npe * W * h.nc * h.nc * esz + 2 * h.ndof * vsz


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def _nvtx(torch, name):
    """Open (name) or close (None) the NVTX range that marks the timed FP64
    steps, so that ncu --nvtx-include can restrict a launch list to them."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def job_rate(ms_local, units_local, ws, device=None):
    """Whole-job step time and throughput of ws replicas: each rank advances
    units_local per step, the job's step time is the slowest rank's (max
    over ranks), and the job advances units_local * ws per step."""
    ms = float(ms_local)
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_local * ws / (ms * 1e-3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
def gpu_arm(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        from paper_1204_1533_gb300 import build
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_1204_1533_gb300 import inputs as I
    from paper_1204_1533_gb300 import ldg

    m = I.vortex_mesh(args.n, args.p)
    U0 = I.vortex_state(m)
    h = ldg.ldg_setup(m, EQ)
    st = torch.cuda.current_stream()
    dt = 0.05
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    timed_launches = {}   # library kernel launches inside the timed steps, per mode

    def run(mode, K, W, e2e=False, live=False):
        """W warm-up + K timed BDF2 levels; returns per-step ms and stats.
        With live=True the apply and matvec launches of the K timed levels
        are bracketed by CUDA events on their stream (ldg_kernel_timer)."""
        Un = torch.from_numpy(U0).cuda()
        U1 = torch.empty_like(Un)
        ldg.ldg_newton_step(h, U1, Un, None, None, dt, ldg.solver_opts(mode=mode, first_step=True))
        Unm1, Un = Un, U1
        hostbuf = None
        if e2e:
            hostbuf = [torch.empty(h.ndof, dtype=torch.float64).pin_memory() for _ in range(3)]
            hostbuf[0].copy_(Un.view(-1).cpu())
            hostbuf[1].copy_(Unm1.view(-1).cpu())
        times, stats = [], []
        timed_launches[mode] = 0
        for it in range(W + K):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            Unext = torch.empty_like(Un)
            l0 = ldg.ldg_launch_count()
            e0.record(st)
            if e2e:
                Un_d = torch.empty_like(Un)
                Unm1_d = torch.empty_like(Un)
                Un_d.view(-1).copy_(hostbuf[0], non_blocking=True)
                Unm1_d.view(-1).copy_(hostbuf[1], non_blocking=True)
                s = ldg.ldg_newton_step(h, Unext, Un_d, Unm1_d, None, dt,
                                        ldg.solver_opts(mode=mode, force_rebuild=True))
                hostbuf[2].copy_(Unext.view(-1), non_blocking=True)
            else:
                s = ldg.ldg_newton_step(h, Unext, Un, Unm1, None, dt,
                                        ldg.solver_opts(mode=mode, force_rebuild=True))
            e1.record(st)
            e1.synchronize()
            if live and it == W - 1:
                ldg.ldg_kernel_timer(True)
                _nvtx(torch, "timed_fp64")
            if it >= W:
                times.append(e0.elapsed_time(e1))
                stats.append(s)
                timed_launches[mode] += ldg.ldg_launch_count() - l0
            if e2e:
                hostbuf[0], hostbuf[1], hostbuf[2] = hostbuf[2], hostbuf[0], hostbuf[1]
            else:
                Unm1, Un = Un, Unext
        if live:
            _nvtx(torch, None)
        return times, stats

    def kernel_ms(fn, reps=20):
        for _ in range(3):
            fn()
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    # ---- timed FP64 steps (the workload's precision) ----------------------
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    t64, s64 = run(ldg.MODE_FP64, args.steps, args.warmup)
    launches = timed_launches[ldg.MODE_FP64]
    clocks = clk.stop()
    torch.cuda.synchronize()
    ms, value = job_rate(np.mean(t64), h.ndof, ws, "cuda")
    launches_per_step = launches / args.steps
    # the same steps again with every apply, matvec and Gram-Schmidt launch
    # bracketed by CUDA events on its stream (the brackets cost about 1 ms a
    # step, so these steps are not the ones `value` is taken from): device
    # time and algorithmic work, (launches, ms, bytes, FLOPs) summed over the
    # timed launches
    run(ldg.MODE_FP64, args.steps, args.warmup, live=True)
    torch.cuda.synchronize()
    live = {name: ldg.ldg_kernel_timer_read(k, ldg.PREC_FP64)
            for name, k in (("precond_apply", ldg.KT_APPLY), ("jacvec", ldg.KT_JACVEC),
                            ("gram_schmidt", ldg.KT_ORTHO))}
    ldg.ldg_kernel_timer(False)

    # ---- mixed-precision steps on the same data ----------------------------
    tmx, smx = run(ldg.MODE_MIXED, args.steps, args.warmup)
    ms_mx, value_mx = job_rate(np.mean(tmx), h.ndof, ws, "cuda")

    # ---- end to end through the public API with host buffers ----------------
    # the same time levels as the device-resident run (same Newton and GMRES
    # work per step), with the inputs copied in and the result copied out
    te2e, _ = run(ldg.MODE_FP64, args.steps, args.warmup, e2e=True)
    ms_e2e, value_e2e = job_rate(np.mean(te2e), h.ndof, ws, "cuda")

    # ---- the paper's own integrator: DIRK3 on the same workload -------------
    dirk = {}
    for name, opts in (("fp64", ldg.solver_opts(mode=ldg.MODE_FP64, force_rebuild=False)),
                       ("mixed", ldg.solver_opts(mode=ldg.MODE_MIXED, force_rebuild=False)),
                       ("fp64_paper_policy", ldg.paper_policy_opts(mode=ldg.MODE_FP64))):
        U = torch.from_numpy(U0).cuda()
        Un = U
        U = torch.empty_like(Un)
        ldg.ldg_dirk3_step(h, U, Un, dt, opts)           # warm-up step (builds the Jacobian)
        tt, ss = [], []
        for _ in range(2):
            Un, U = U, torch.empty_like(U)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            s = ldg.ldg_dirk3_step(h, U, Un, dt, opts)
            e1.record(st)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1))
            ss.append(s)
        dirk[name] = {"ms_per_step": float(np.mean(tt)), "newton_its": float(np.mean([s["newton_its"] for s in ss])),
                      "gmres_its": float(np.mean([s["gmres_its"] for s in ss])),
                      "jac_builds": float(np.mean([s["jac_builds"] for s in ss]))}

    # ---- per-kernel timings on the launching stream -------------------------
    Ut = torch.from_numpy(U0).cuda()
    R = torch.empty_like(Ut)
    t_res = kernel_ms(lambda: ldg.ldg_residual(h, Ut, R))
    J64 = ldg.ldg_jacobian(h, Ut, ldg.PREC_FP64)
    J32 = ldg.ldg_jacobian(h, Ut, ldg.PREC_FP32)
    t_j64 = kernel_ms(lambda: ldg.ldg_jacobian(h, Ut, ldg.PREC_FP64, J64))
    t_j32 = kernel_ms(lambda: ldg.ldg_jacobian(h, Ut, ldg.PREC_FP32, J32))
    x64 = torch.randn(h.ndof, dtype=torch.float64, device="cuda")
    y64 = torch.empty_like(x64)
    x32, y32 = x64.float(), torch.empty(h.ndof, dtype=torch.float32, device="cuda")
    t_mv64 = kernel_ms(lambda: ldg.ldg_jacvec(h, J64, 1.0, -0.033, x64, y64, ldg.PREC_FP64))
    t_mv32 = kernel_ms(lambda: ldg.ldg_jacvec(h, J32, 1.0, -0.033, x32, y32, ldg.PREC_FP32))
    P64 = ldg.ldg_precond(h, J64, 1.0, -0.033)
    P32 = ldg.ldg_precond(h, J32, 1.0, -0.033)
    t_pc64 = kernel_ms(lambda: ldg.ldg_precond(h, J64, 1.0, -0.033, P64), reps=5)
    t_pc32 = kernel_ms(lambda: ldg.ldg_precond(h, J32, 1.0, -0.033, P32), reps=5)
    t_ap64 = kernel_ms(lambda: ldg.ldg_precond_apply(h, P64, x64, y64, ldg.PREC_FP64))
    t_ap32 = kernel_ms(lambda: ldg.ldg_precond_apply(h, P32, x32, y32, ldg.PREC_FP32))

    fp64pk = fp64_peak(torch, ldg)
    FP64_PEAK = fp64pk["burst_tflops"]
    # phase shares of the FP64 step (CUDA-event phase timers inside the step)
    ph = {k: float(np.mean([s[k] for s in s64])) for k in
          ("t_residual_ms", "t_jacobian_ms", "t_precond_ms", "t_linear_ms")}
    hbm, src = _peaks()
    res_fl = euler_residual_flops(h.D, h.p, h.nc, h.E)
    kernels = {
        "residual_fp64": {"ms": t_res, "dof_s": h.ndof / (t_res * 1e-3),
                          "tflops": res_fl / (t_res * 1e-3) / 1e12},
        "jacobian_fp64": {"ms": t_j64, "dof_s": h.ndof / (t_j64 * 1e-3)},
        "jacobian_fp32": {"ms": t_j32, "dof_s": h.ndof / (t_j32 * 1e-3),
                          "gbs": jac_bytes(h, 4) / (t_j32 * 1e-3) / 1e9},
        "jacvec_fp64": {"ms": t_mv64, "gbs": jacvec_bytes(h, 8, 8) / (t_mv64 * 1e-3) / 1e9},
        "jacvec_fp32": {"ms": t_mv32, "gbs": jacvec_bytes(h, 4, 4) / (t_mv32 * 1e-3) / 1e9},
        "precond_build_fp64": {"ms": t_pc64}, "precond_build_fp32": {"ms": t_pc32},
        "precond_apply_fp64": {"ms": t_ap64, "gbs": apply_bytes(h, 8, 8) / (t_ap64 * 1e-3) / 1e9},
        "precond_apply_fp32": {"ms": t_ap32, "gbs": apply_bytes(h, 4, 4) / (t_ap32 * 1e-3) / 1e9},
    }
    # dominant kernel of the step: of the timed Krylov kernels (the ncu
    # launch list under profiles/ gives the shares of all kernels) the one
    # with the largest device time inside the timed FP64 steps. Achieved =
    # its algorithmic bytes (or FP64 FLOPs) per launch over its mean launch
    # time from the live CUDA events; the bound is the roofline it is closer to.
    names = {"precond_apply": "k_precond_apply (element ILU(0) apply, FP64)",
             "jacvec": "k_jacvec (split matvec K11 x, FP64)",
             "gram_schmidt": "k_ortho (fused classical Gram-Schmidt sweeps of GMRES, FP64)"}
    per_kernel = {}
    for kname, (n_l, ms_l, by_l, fl_l) in live.items():
        if n_l == 0 or ms_l <= 0:
            continue
        sec = ms_l * 1e-3
        per_kernel[kname] = {"launches": n_l, "ms_per_launch": ms_l / n_l, "gbs": by_l / sec / 1e9,
                             "tflops": fl_l / sec / 1e12, "frac_hbm": by_l / sec / 1e9 / hbm,
                             "frac_fp64": fl_l / sec / 1e12 / FP64_PEAK,
                             "share_of_step": ms_l / (ms * args.steps),
                             "bytes_per_launch": by_l / n_l, "flops_per_launch": fl_l / n_l}
    kname = max(per_kernel, key=lambda k: per_kernel[k]["ms_per_launch"] * per_kernel[k]["launches"])
    pk = per_kernel[kname]
    if pk["frac_fp64"] > pk["frac_hbm"]:
        roof = {"kernel": names[kname], "bound": "alu", "achieved": pk["tflops"], "peak": FP64_PEAK,
                "unit": "TFLOP/s", "frac": pk["frac_fp64"], "traffic": TRAFFIC.get(kname),
                "flops_per_launch": pk["flops_per_launch"],
                "peak_source": "measured: FP64 FMA burst rate of this GPU in this run (ldg_fp64_fma_probe), "
                               "of measured"}
    else:
        roof = {"kernel": names[kname], "bound": "hbm", "achieved": pk["gbs"], "peak": hbm, "unit": "GB/s",
                "frac": pk["frac_hbm"], "traffic": TRAFFIC.get(kname), "bytes_per_launch": pk["bytes_per_launch"],
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs, of measured)"}
    roof.update({"launches_timed": pk["launches"], "ms_per_launch": pk["ms_per_launch"], "live": per_kernel})
    kernels["residual_fp64"]["alu_frac_of_measured_fp64"] = res_fl / (t_res * 1e-3) / 1e12 / FP64_PEAK
    out = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": h.E, "p": h.p, "dof": h.ndof,
                   "newton_rtol": 1e-8, "linear": "GMRES(30) + element-block ILU(0), eta=1e-3, classical Gram-Schmidt with "
                             "a second pass where one shrinks the column more than 10x",
                   "jacobian": "rebuilt every step", "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas x{ws}"},
        "newton_its": float(np.mean([s["newton_its"] for s in s64])),
        "gmres_its": float(np.mean([s["gmres_its"] for s in s64])),
        "reorth_its": float(np.mean([s["reorth_its"] for s in s64])),
        "phases_ms_fp64": ph,
        "mixed": {"ms_per_step": ms_mx, "value": value_mx,
                  "speedup_vs_fp64": ms / ms_mx,
                  "newton_its": float(np.mean([s["newton_its"] for s in smx])),
                  "gmres_its": float(np.mean([s["gmres_its"] for s in smx])),
                  "reorth_its": float(np.mean([s["reorth_its"] for s in smx])),
                  "phases_ms": {k: float(np.mean([s[k] for s in smx])) for k in ph}},
        "kernels": kernels,
        "dirk3": dict(dirk, note="one step of the paper's three-stage DIRK on the same workload and dt, "
                                 "Jacobian re-used across stages and steps (the paper's policy)"),
        "roofline": roof,
        "hbm_peak_gbs": hbm, "hbm_peak_source": src,
        "fp64_peak": dict(fp64pk, nominal_tflops=FP64_NOMINAL_TFLOPS),
        "e2e": {"value": value_e2e, "unit": "DOF/s",
                "h2d_bytes_per_step": 2 * h.ndof * 8, "d2h_bytes_per_step": h.ndof * 8},
        "gpu_launches": launches,
        "gpu_launches_per_step": launches_per_step,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_tgv:
        out["tgv"] = tgv_section(args, hbm)
    if rank == 0 and ws == 1 and not args.no_learned:
        out["learned"] = learned_section(args)
    if rank == 0 and ws == 1 and not args.no_channel:
        out["channel"] = channel_section(args, hbm)
    if rank == 0 and ws == 1 and not args.no_stabilized:
        out["stabilized"] = stabilized_section(args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _oracle_step(n_sample, p):
    """One oracle BDF2 level (Newton-GMRES with the oracle's complex-step
    Jacobian and ILU(0)) on an n_sample x n_sample patch of the workload."""
    import numpy as np

    from oracle import jacobian as JAC
    from oracle import solvers as S
    from oracle.residual import Discretization, full_residual
    from paper_1204_1533_gb300 import inputs as I
    L = 10.0 * n_sample / 64.0
    m = I.vortex_mesh(n_sample, p, L=L)
    disc = Discretization(m, EQ)
    U0 = I.vortex_state(m, x0=L / 2, y0=L / 2)
    pat = S.line_pattern(disc.D, disc.p)

    def pc(K, shift, scale):
        Fct = S.ilu0(S.masked_blocks(disc, K[0], shift, scale), pat)
        return lambda v: S.ilu_apply(Fct, pat, v.reshape(U0.shape)).ravel()
    F = lambda X: full_residual(disc, X)
    jac = lambda X: (JAC.K11(disc, X), None, None)
    t0 = time.perf_counter()
    U1, st = S.newton_bdf2(F, jac, U0, U0, 0.05, first=False, rtol=1e-8, gmres_tol=1e-3,
                           restart=30, reuse=15, precond_builder=pc)
    return time.perf_counter() - t0, disc.ndof, st


NS_EQ = {"kind": "ns", "gamma": 1.4, "mu": 1.0 / 1600.0, "Pr": 0.72, "flux": "roe"}


def _kernel_ms(torch, flush, fn, reps):
    fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps


def tgv_section(args, hbm):
    """3-D Navier-Stokes Taylor-Green vortex, 32^3 curved hexes, p = 3
    (10.5M DOF): the hot-path kernels at full size against the HBM roofline
    and one BDF2 level (dt = 0.05) in mixed precision and in FP64, with the
    relative difference of the two solutions."""
    import torch

    from paper_1204_1533_gb300 import inputs as I
    from paper_1204_1533_gb300 import ldg
    n, dt = args.tgv_n, args.tgv_dt
    m = I.tgv_mesh(n, 3)
    U0 = I.tgv_state(m)
    t0 = time.perf_counter()
    h = ldg.ldg_setup(m, NS_EQ)
    t_setup = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    Ut = torch.from_numpy(U0).cuda()
    R = torch.empty_like(Ut)
    out = {"workload": f"ns3d_tgv_{n}^3_p3_bdf2_dt{dt}", "dof": h.ndof, "setup_s": t_setup}
    k = {}
    _nvtx(torch, "tgv_kernels")
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_residual(h, Ut, R), 5)
    k["residual_fp64"] = {"ms": t, "dof_s": h.ndof / (t * 1e-3)}
    J = ldg.ldg_jacobian(h, Ut, ldg.PREC_FP32)
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_jacobian(h, Ut, ldg.PREC_FP32, J), 3)
    jb = jac_bytes(h, 4)
    k["jacobian_fp32"] = {"ms": t, "dof_s": h.ndof / (t * 1e-3), "gbs": jb / (t * 1e-3) / 1e9,
                          "frac_hbm": jb / (t * 1e-3) / 1e9 / hbm}
    x = torch.randn(h.ndof, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_jacvec(h, J, 1.0, -dt, x, y, ldg.PREC_FP32), 5)
    vb = jacvec_bytes(h, 4, 4)
    k["jacvec_fp32"] = {"ms": t, "gbs": vb / (t * 1e-3) / 1e9, "frac_hbm": vb / (t * 1e-3) / 1e9 / hbm}
    P = ldg.ldg_precond(h, J, 1.0, -2.0 / 3.0 * dt)
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_precond(h, J, 1.0, -2.0 / 3.0 * dt, P), 2)
    k["precond_build_fp32"] = {"ms": t}
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_precond_apply(h, P, x, y, ldg.PREC_FP32), 5)
    ab = apply_bytes(h, 4, 4)
    k["precond_apply_fp32"] = {"ms": t, "gbs": ab / (t * 1e-3) / 1e9, "frac_hbm": ab / (t * 1e-3) / 1e9 / hbm}
    _nvtx(torch, None)
    out["kernels"] = k
    del J, P, x, y
    torch.cuda.empty_cache()
    sol = {}
    for name, mode in (("mixed", ldg.MODE_MIXED), ("fp64", ldg.MODE_FP64)):
        Un = torch.from_numpy(U0).cuda()
        U1 = torch.empty_like(Un)
        ldg.ldg_newton_step(h, U1, Un, None, None, dt, ldg.solver_opts(mode=mode, first_step=True))
        U2 = torch.empty_like(Un)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        _nvtx(torch, f"tgv_step_{name}")
        e0.record()
        s = ldg.ldg_newton_step(h, U2, U1, Un, None, dt, ldg.solver_opts(mode=mode, force_rebuild=True))
        e1.record()
        e1.synchronize()
        _nvtx(torch, None)
        sol[name] = U2
        out[name] = {"ms_per_step": e0.elapsed_time(e1), "newton_its": s["newton_its"], "gmres_its": s["gmres_its"],
                     "res_final_rel": s["res_final"] / s["res0"],
                     "phases_ms": {q: s[q] for q in ("t_residual_ms", "t_jacobian_ms", "t_precond_ms",
                                                     "t_linear_ms")}}
        del Un, U1
        torch.cuda.empty_cache()
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["rel_diff_mixed_vs_fp64"] = float((sol["mixed"] - sol["fp64"]).norm() / sol["fp64"].norm())
    del h, sol, Ut, R
    return out


def channel_section(args, hbm):
    """3-D Navier-Stokes channel with sinusoidal bump walls (no-slip,
    adiabatic), 64 x 32 x 32 curved hexes with wall-normal stretching 1.1,
    p = 4 (41M DOF), Re = 5000, Mach 0.3: the kernels at full size, then one
    BDF2 level at CFL 50 (dt from the smallest node spacing and |u| + c) in
    mixed precision and in FP64 from the same BDF1 start level (--channel-steps
    levels each, --channel-forcing of the linear solves)."""
    import numpy as np
    import torch

    from paper_1204_1533_gb300 import inputs as I
    from paper_1204_1533_gb300 import ldg
    nx, ny, nz = args.channel
    m = I.channel_mesh(nx, ny, nz, 4)
    U0 = I.channel_state(m)
    eq = {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 1.0 / 5000.0, "Pr": 0.72, "bc": {1: "wall"}}
    t0 = time.perf_counter()
    h = ldg.ldg_setup(m, eq)
    t_setup = time.perf_counter() - t0
    Xr = m["nodes"].reshape(m["nodes"].shape[0], 5, 5, 5, 3)
    dmin = min(float(np.linalg.norm(np.diff(Xr, axis=ax), axis=-1).min()) for ax in (1, 2, 3))
    dt = args.channel_cfl * dmin / (1.0 + 1.0 / 0.3)
    del Xr
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    Ut = torch.from_numpy(U0).cuda()
    R = torch.empty_like(Ut)
    out = {"workload": f"ns3d_channel_bump_{nx}x{ny}x{nz}_p4_bdf2_cfl{args.channel_cfl:g}", "dof": h.ndof,
           "setup_s": t_setup, "dt": dt}
    k = {}
    _nvtx(torch, "channel_kernels")
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_residual(h, Ut, R), 3)
    k["residual_fp64"] = {"ms": t, "dof_s": h.ndof / (t * 1e-3)}
    J = ldg.ldg_jacobian(h, Ut, ldg.PREC_FP32)
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_jacobian(h, Ut, ldg.PREC_FP32, J), 2)
    jb = jac_bytes(h, 4)
    k["jacobian_fp32"] = {"ms": t, "dof_s": h.ndof / (t * 1e-3), "gbs": jb / (t * 1e-3) / 1e9,
                          "frac_hbm": jb / (t * 1e-3) / 1e9 / hbm}
    x = torch.randn(h.ndof, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_jacvec(h, J, 1.0, -dt, x, y, ldg.PREC_FP32), 3)
    vb = jacvec_bytes(h, 4, 4)
    k["jacvec_fp32"] = {"ms": t, "gbs": vb / (t * 1e-3) / 1e9, "frac_hbm": vb / (t * 1e-3) / 1e9 / hbm}
    P = ldg.ldg_precond(h, J, 1.0, -2.0 / 3.0 * dt)
    t = _kernel_ms(torch, flush, lambda: ldg.ldg_precond_apply(h, P, x, y, ldg.PREC_FP32), 3)
    ab = apply_bytes(h, 4, 4)
    k["precond_apply_fp32"] = {"ms": t, "gbs": ab / (t * 1e-3) / 1e9, "frac_hbm": ab / (t * 1e-3) / 1e9 / hbm}
    _nvtx(torch, None)
    out["kernels"] = k
    del J, P, x, y
    torch.cuda.empty_cache()
    Un = torch.from_numpy(U0).cuda()
    U1 = torch.empty_like(Un)
    forcing = ldg.FORCING_TARGET if args.channel_forcing == "target" else ldg.FORCING_FIXED
    s1 = ldg.ldg_newton_step(h, U1, Un, None, None, dt,
                             ldg.solver_opts(mode=ldg.MODE_MIXED, first_step=True, forcing=forcing))
    out["bdf1_start"] = {"newton_its": s1["newton_its"], "gmres_its": s1["gmres_its"]}
    out["levels"] = args.channel_steps
    out["forcing"] = args.channel_forcing
    sol = {}
    for name, mode in (("mixed", ldg.MODE_MIXED), ("fp64", ldg.MODE_FP64)):
        # args.channel_steps BDF2 levels from the same BDF1 start, each solved
        # to the 1e-8 target with the Jacobian rebuilt at its first iteration
        Um1, Uc = Un, U1
        ms, newton, gmres, res_rel = [], [], [], []
        for _ in range(args.channel_steps):
            U2 = torch.empty_like(Un)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s = ldg.ldg_newton_step(h, U2, Uc, Um1, None, dt,
                                    ldg.solver_opts(mode=mode, force_rebuild=True, forcing=forcing))
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            newton.append(s["newton_its"])
            gmres.append(s["gmres_its"])
            res_rel.append(s["res_final"] / s["res0"])
            if Um1 is not Un:
                del Um1
            Um1, Uc = Uc, U2
        sol[name] = Uc
        out[name] = {"ms_per_step": float(np.mean(ms)), "newton_its": float(np.mean(newton)),
                     "gmres_its": float(np.mean(gmres)), "res_final_rel": float(np.max(res_rel)),
                     "ms_total": float(np.sum(ms)),
                     "phases_ms": {q: s[q] for q in ("t_residual_ms", "t_jacobian_ms", "t_precond_ms",
                                                     "t_linear_ms")}}
        del Um1
        torch.cuda.empty_cache()
    out["mixed_speedup_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["rel_diff_mixed_vs_fp64"] = float((sol["mixed"] - sol["fp64"]).norm() / sol["fp64"].norm())
    del h, sol, Ut, R, Un, U1
    torch.cuda.empty_cache()
    return out


def stabilized_section(args):
    """The stabilised LDG scheme (C11 = C22 = 1/20) of Table 2's lower half on
    the 16 x 16 mapped unit square with p = 3 and the paper's manufactured
    solution and Dirichlet data (Sec. 5.1): the
    coupled (U, Q) solve with its element block-Jacobi preconditioner, the
    D(U, Q) kernel, and the errors against the manufactured solution next to
    the minimal-dissipation solve of the same mesh."""
    import numpy as np
    import torch

    from paper_1204_1533_gb300 import inputs as I
    from paper_1204_1533_gb300 import ldg
    m = I.poisson_mapped_square_mesh(16, 3)
    E, npe = m["nodes"].shape[:2]
    u_ex, gu_ex, f = I.poisson_paper_solution(m)
    out = {"workload": "poisson2d_mapped16x16_p3_paper_solution_C11_C22_0.05"}
    eq = {"kind": "poisson", "C11": 0.05, "C22": 0.05, "C11b": 1.0, "bc": {0: "dirichlet"}, "source": f,
          "gD": u_ex}
    h = ldg.ldg_setup(m, eq)
    U = torch.zeros((E, 1, npe), dtype=torch.float64, device="cuda")
    Q = torch.zeros((E, 1, 2, npe), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ldg.ldg_coupled_solve(h, U, Q, rtol=1e-10, restart=64, max_cycles=100)
    wall = time.perf_counter() - t0
    out.update({"wall_ms_first_solve": wall * 1e3, "precond_build_ms": st["t_precond_ms"],
                "gmres_ms": st["t_linear_ms"], "gmres_its": st["gmres_its"], "cycles": st["newton_its"],
                "res_final_rel": st["res_final"] / st["res0"],
                "err_u": float(np.abs(U.cpu().numpy() - u_ex).max()),
                "err_q": float(np.abs(Q.cpu().numpy() - gu_ex).max())})
    U.zero_()
    Q.zero_()
    torch.cuda.synchronize()
    _nvtx(torch, "stabilized_resolve")
    t0 = time.perf_counter()
    st = ldg.ldg_coupled_solve(h, U, Q, rtol=1e-10, restart=64, max_cycles=100)
    out["wall_ms_resolve"] = (time.perf_counter() - t0) * 1e3
    _nvtx(torch, None)
    G = torch.empty_like(Q)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out["gradient_uq_ms"] = _kernel_ms(torch, flush, lambda: ldg.ldg_gradient_uq(h, U, Q, G), 20)
    eq0 = dict(eq, C11=0.0, C22=0.0)
    h0 = ldg.ldg_setup(m, eq0)
    U0 = torch.zeros_like(U)
    ldg.ldg_steady_solve(h0, U0, 1.0, 1.0, 0, ldg.solver_opts(mode=ldg.MODE_FP64, rtol=1e-10, max_newton=30,
                                                                 restart=64))
    Q0 = torch.empty_like(Q)
    ldg.ldg_gradient(h0, U0, Q0)
    out["minimal_dissipation"] = {"err_u": float(np.abs(U0.cpu().numpy() - u_ex).max()),
                                  "err_q": float(np.abs(Q0.cpu().numpy() - gu_ex).max())}
    return out


def learned_section(args):
    """The learned Newton guess on the Taylor-Green vortex at 16^3, p = 3:
    200 trajectories of 10 levels from the implicit solver for Re ~
    U[400, 1600], 20k Adam steps on the GPU, and on the held-out Re = 1200
    the wall time per BDF2 level of FP64 + extrapolation, mixed +
    extrapolation and mixed + learned guess (residual-checked), all to the
    same 1e-8 relative residual, with the fixed and the target-aware forcing
    of the linear solves."""
    import torch

    from paper_1204_1533_gb300 import learned
    from paper_1204_1533_gb300 import ldg
    out, mlp, h = learned.experiment(n=args.learn_n, n_traj=args.learn_traj, steps=10, dt=args.learn_dt,
                                     train_steps=args.learn_train, lines=4096, eval_steps=12, verbose=False)
    # the trained network's inference (tcgen05 tensor cores, TMEM accumulators)
    # over the direction-1 lines of the 32^3, p = 3 Taylor-Green mesh
    lines = 32 ** 3 * 16
    X = torch.randn((lines, ldg.MLP_INP), device="cuda").to(torch.bfloat16)
    Y = torch.empty((lines, mlp.n_out), dtype=torch.float32, device="cuda")
    for _ in range(3):
        ldg.ldg_mlp_forward(mlp, X, Y)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(st)
    for _ in range(reps):
        ldg.ldg_mlp_forward(mlp, X, Y)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * lines * (mlp.n_in * 128 + 2 * 128 * 128 + 128 * mlp.n_out)
    byts = lines * (ldg.MLP_INP * 2 + mlp.n_out * 4)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        bf16_peak = 1900.0
    hbm, _ = _peaks()
    inference = {"kernel": "k_mlp_fwd_tc (tcgen05.mma kind::f16, TMEM accumulators)", "lines": lines, "ms": ms,
                 "tflops": flops / (ms * 1e-3) / 1e12, "frac_bf16_peak": flops / (ms * 1e-3) / 1e12 / bf16_peak,
                 "gbs": byts / (ms * 1e-3) / 1e9, "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm}
    keep = ("mesh", "p", "trajectories", "levels_per_trajectory", "dt", "samples", "train_steps", "t_generate_s",
            "t_train_s", "loss_first", "loss_last", "held_out_re", "mean_res_ratio_mlp_over_extrap",
            "mean_err_ratio_mlp_over_extrap", "mean_mlp_weight", "newton_extrap", "newton_mlp", "newton_fp64",
            "gmres_extrap", "gmres_mlp", "gmres_fp64", "ms_fp64_extrap", "ms_mixed_extrap", "ms_mixed_mlp",
            "max_rel_diff_mixed_vs_fp64")
    res = {q: out[q] for q in keep if q in out}
    res["forcing"] = out.get("forcing")
    if "ms_fp64_extrap" in res:
        res["speedup_mixed_learned_vs_fp64"] = res["ms_fp64_extrap"] / res["ms_mixed_mlp"]
        res["speedup_mixed_vs_fp64"] = res["ms_fp64_extrap"] / res["ms_mixed_extrap"]
    # the same held-out levels with the target-aware forcing (each linear
    # solve asked only for the reduction the stopping rule still needs)
    tf = out.get("forcing_target")
    if tf:
        t = {q: tf[q] for q in keep if q in tf}
        if "ms_fp64_extrap" in t:
            t["speedup_mixed_learned_vs_fp64"] = t["ms_fp64_extrap"] / t["ms_mixed_mlp"]
            t["speedup_mixed_learned_vs_mixed_extrap"] = t["ms_mixed_extrap"] / t["ms_mixed_mlp"]
        res["forcing_target"] = t
    res["inference_32cubed"] = inference
    return res


def _oracle_suite(cfg):
    """The oracle, as it stands, on bounded samples of the workloads (one
    process, one thread): seconds and DOF of (i) its residual on a 6 x 6
    patch of the vortex (p = 4), a 3^3 Taylor-Green box (p = 3) and a
    3 x 2 x 3 walled channel (p = 4), each repeated for about a second,
    (ii) its Jacobian (complex-step K11, graph-coloured) of the vortex patch,
    (iii) one BDF2 level of the vortex patch (the metric's unit)."""
    import numpy as np

    from oracle import jacobian as JAC
    from oracle.residual import Discretization, full_residual
    from paper_1204_1533_gb300 import inputs as I
    n_sample, p = cfg
    out = {}
    L = 10.0 * n_sample / 64.0
    mv = I.vortex_mesh(n_sample, p, L=L)
    samples = (("residual_vortex", mv, EQ, I.vortex_state(mv, x0=L / 2, y0=L / 2)),
               ("residual_tgv", I.tgv_mesh(3, 3), NS_EQ, None),
               ("residual_channel", I.channel_mesh(3, 2, 3, 4),
                {"kind": "ns", "gamma": 1.4, "flux": "roe", "mu": 1.0 / 5000.0, "Pr": 0.72, "bc": {1: "wall"}}, None))
    for name, m, eq, U in samples:
        if U is None:
            U = I.tgv_state(m) if name == "residual_tgv" else I.channel_state(m)
        disc = Discretization(m, eq)
        full_residual(disc, U)
        k, t0 = 0, time.perf_counter()
        while True:
            full_residual(disc, U)
            k += 1
            el = time.perf_counter() - t0
            if el > 1.0:
                break
        out[name] = (el / k, disc.ndof)
    disc = Discretization(mv, EQ)
    Uv = samples[0][3]
    t0 = time.perf_counter()
    JAC.K11(disc, Uv)
    out["jacobian_vortex"] = (time.perf_counter() - t0, disc.ndof)
    secs, dof, _ = _oracle_step(n_sample, p)
    out["bdf2_level_vortex"] = (secs, dof)
    return out


def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_runs(args, nproc):
    """_oracle_suite in nproc spawned single-threaded processes at once (a
    pool started with spawn: this process has already used the GPU)."""
    import multiprocessing as mp
    _single_thread_env()
    with mp.get_context("spawn").Pool(nproc) as pool:
        return pool.map(_oracle_suite, [(args.cpu_sample, args.p)] * nproc)


def cpu_baseline(args):
    """The oracle on the host cores: DOF/s of each timed quantity on one
    core, and on all cores as one replica per core (the sum of the replicas'
    rates while they ran together)."""
    ncores = os.cpu_count() or 1
    one = _oracle_runs(args, 1)[0]
    many = _oracle_runs(args, ncores)
    per = {}
    for k in one:
        per[k] = {"dof": one[k][1], "dof_s_1core": one[k][1] / one[k][0],
                  "dof_s_all_cores": sum(r[k][1] / r[k][0] for r in many)}
    v = per["bdf2_level_vortex"]
    return {"value": v["dof_s_all_cores"], "unit": "DOF/s", "cores": ncores, "kind": "oracle",
            "value_1core": v["dof_s_1core"],
            "sample": f"one BDF2 level (Newton-GMRES(30), ILU(0), complex-step Jacobian) on a "
                      f"{args.cpu_sample}x{args.cpu_sample}-element patch of the p={args.p} vortex "
                      f"({v['dof']} DOF), one single-threaded replica per host core ({ncores}); "
                      f"per_kernel: residual samples (vortex patch, 3^3 Taylor-Green box, 3x2x3 channel), "
                      f"the Jacobian of the vortex patch",
            "per_kernel": per}


def reference_arm(args):
    """The oracle's BDF2 level on a bounded sample of the workload, one
    single-threaded replica per host core, DOF/s summed over the replicas."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import multiprocessing as mp
    _single_thread_env()
    ncores = os.cpu_count() or 1
    times = []
    dof = 0
    with mp.get_context("spawn").Pool(ncores) as pool:
        for it in range(args.warmup + args.steps):
            res = pool.map(_oracle_step_secs, [(args.cpu_sample, args.p)] * ncores)
            if it >= args.warmup:
                times.append(res)
            dof = res[0][1]
    rates = [sum(dof / r[0] for r in step) for step in times]
    v = sum(rates) / len(rates)
    ms = dof * ncores / v * 1e3
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_elements": args.cpu_sample ** 2},
        "cpu_baseline": {"value": v, "unit": "DOF/s", "cores": ncores, "kind": "oracle",
                         "sample": f"{args.cpu_sample}x{args.cpu_sample}-element patch, one BDF2 level per "
                                   f"step in each of {ncores} single-threaded replicas"},
        "e2e": {"value": v, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def _oracle_step_secs(cfg):
    secs, dof, _ = _oracle_step(*cfg)
    return secs, dof


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--cpu-sample", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tgv", action="store_true", help="skip the 3-D Taylor-Green section")
    ap.add_argument("--tgv-n", type=int, default=32)
    ap.add_argument("--tgv-dt", type=float, default=0.05)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-guess section")
    ap.add_argument("--no-channel", action="store_true", help="skip the 3-D walled channel section")
    ap.add_argument("--channel", type=int, nargs=3, default=[64, 32, 32])
    ap.add_argument("--no-stabilized", action="store_true", help="skip the stabilised-LDG Poisson section")
    ap.add_argument("--channel-cfl", type=float, default=50.0)
    ap.add_argument("--channel-steps", type=int, default=1, help="BDF2 levels of the channel per precision")
    ap.add_argument("--channel-forcing", default="fixed", choices=["fixed", "target"])
    ap.add_argument("--learn-n", type=int, default=16)
    ap.add_argument("--learn-dt", type=float, default=0.03)
    ap.add_argument("--learn-traj", type=int, default=200)
    ap.add_argument("--learn-train", type=int, default=20000)
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
