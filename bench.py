"""Throughput benchmark of the discrete-DtN ABC time-stepper on GB300.

Default workload: the large batched mean field -- 96^3 interior grid, h = 0.35,
128 orbitals (seeded Gaussian-modulated plane waves, orthonormalised), density-
dependent potential V = a rho + b rho^(1+alpha) (a = -1, b = 0.8, alpha = 1/6)
rebuilt from the state before every step, first-order ABC interpolated at s1 = 1
(n_Gamma = 54152), dt = 0.004 -- in its complex64 form with the boundary
contraction on the tensor cores.  A "step" is one time step: the mean-field
potential, then 4 Horner stages, each a forward boundary transform, the boundary
DtN contraction, the back transform and the fused stencil / potential / integrator
kernel.  The step loop is replayed as a CUDA graph.

metric: orbital*gridpoint*steps/s (b * N^3 * steps / time), higher is better.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload N]

N > 1 is launched by torchrun: every rank runs an independent replica on its own
GPU (the path has no exchange step), timing is max over ranks and ``value`` is the
sum of all ranks' units over that time ("weak" scaling).  ``--impl reference`` times
the FP64 CPU oracle on the same workload (a bounded sample of steps) instead.
``--workload 2`` gives the single-orbital harmonic-well line (its own roofline on the
one-orbital contraction); the default line also carries that workload's figures.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "orbital*gridpoint*steps/s"
WORKLOAD_NUMBER = 5
SINGLE_ORBITAL_WORKLOAD = 2
L2_BYTES = 129 << 20
L2_FLUSH_BYTES = 256 << 20          # written before every timed step when the state fits in L2
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense tensor-core rates (TF32 / BF16)
FP64_CUBLAS_TFLOPS = 1.10           # torch.matmul FP64 4096^3 on this GPU model (library probe)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: the workload's own count)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU form")
    ap.add_argument("--no-extra", action="store_true", help="skip the single-orbital figures on the default line")
    ap.add_argument("--reuse-tuning", action="store_true",
                    help="take the autotuner's cached choice when there is one (profiling runs)")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default knobs (profiling runs)")
    ap.add_argument("--knob", action="append", default=[], metavar="NAME=VALUE",
                    help="set a tuning knob (abc.TUNE_<NAME>) after tuning, e.g. BACK_MULTI=1 (profiling runs)")
    ap.add_argument("--workload", type=int, default=WORKLOAD_NUMBER,
                    help="5 (default) or 2 give a full line; 1, 3, 4, 6-10 a line of their own")
    return ap.parse_args()


# ----------------------------------------------------------------------
# distributed plumbing (replicas; the only collective is the timing reduction)
# ----------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(units: float, seconds: float, group=None):
    """(total units over ranks, max seconds over ranks) -- all ranks get the result."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units, seconds
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    s = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(s, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(s.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ----------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ----------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ----------------------------------------------------------------------
def host_threads():
    """What the host BLAS and OpenMP may use: nproc, OMP_NUM_THREADS, BLAS threads."""
    nproc = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    blas = None
    try:
        from threadpoolctl import threadpool_info
        blas = max((i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"), default=None)
    except Exception:
        blas = os.environ.get("OPENBLAS_NUM_THREADS")
    return {"nproc": nproc, "omp_num_threads": os.environ.get("OMP_NUM_THREADS"),
            "blas_threads": int(blas) if blas else nproc}


def mem_available_bytes():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def cpu_oracle_sample(w, steps: int, budget_s: float = 20.0):
    """Time the FP64 oracle's time step on the workload's full grid and orbital count.
    Its DtN set-up at this size (a dense n_Gamma^2 complex solve) takes far longer than
    a benchmark allows, so B is a seeded complex stand-in of the same size and A the
    diagonal of the order-1 ABC; the step's cost does not depend on their values.  If
    the host cannot hold the dense stand-in, the 64^3 x 32 mean-field workload is
    timed instead and the sample says so."""
    import scipy.sparse as sp

    from oracle.lattice import Box, n_gamma
    from oracle.propagate import System
    from paper_1908_02456_gb300 import inputs

    note = ""
    ng = n_gamma(w.shape, 1)
    if 16.0 * ng * ng * 1.3 + 24e9 > mem_available_bytes():
        note = (f"host memory cannot hold the dense {ng}^2 complex128 stand-in of {w.name}; "
                f"timed on the 64^3 x 32 mean-field workload instead; ")
        w = inputs.WORKLOADS[3]
        ng = n_gamma(w.shape, 1)
    psi0, V = inputs.make_inputs(w)
    box = Box(w.shape, w.h)
    B = np.empty((ng, ng), dtype=np.complex128)
    rows = 256
    blk = np.random.default_rng(1).standard_normal((rows, 2 * ng)).view(np.complex128) * 1e-3
    for i in range(0, ng, rows):
        B[i:i + rows] = blk[:min(rows, ng - i)]
    A = sp.diags(np.full(ng, -1j / (4 * w.h ** 4)))
    sysm = System(box, V_ext=V.reshape(-1), coeffs={"order": 1, "A": A, "B": B, "Q": None},
                  meanfield=w.meanfield)
    phi = psi0.reshape(w.n_orb if w.meanfield else 1, -1)
    f = np.zeros((phi.shape[0], ng), np.complex128)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        phi, f = sysm.step(phi, f, w.dt)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    sec = time.perf_counter() - t0
    th = host_threads()
    return {"value": phi.shape[0] * box.n * done / sec, "unit": METRIC, "cores": th["blas_threads"],
            "kind": "oracle", "nproc": th["nproc"], "omp_num_threads": th["omp_num_threads"],
            "blas_threads": th["blas_threads"],
            "sample": note + f"{done} step(s) of the oracle's Taylor step on the full {w.n}^3 grid with "
                             f"{phi.shape[0]} orbital(s) (sparse stencil + dense {ng}x{ng} complex128 B "
                             f"stand-in{', mean-field potential' if w.meanfield else ''}), {sec:.1f} s"}


def config_dict(w):
    """The workload as both arms name it."""
    state = w.n_orb * w.n ** 3 * 8
    if state > 2 * L2_BYTES:
        l2 = f"inputs larger than L2: each state array {state / 1e6:.0f} MB (L2 129 MB); no flush"
    else:
        l2 = f"L2 flushed before every timed step ({L2_FLUSH_BYTES >> 20} MiB write; L2 is 129 MB)"
    pot = {"none": "0", "harmonic_bumps": "0.5*0.09*r^2 + 8 seeded Gaussian bumps",
           "smooth_random": "6 seeded Gaussians, max|V| = 0.3", "zero": "0"}[w.potential]
    if w.meanfield:
        a, b, al = w.meanfield
        pot = f"V_ext = {pot}; mean field a*rho + b*rho^(1+alpha), a = {a}, b = {b}, alpha = {al:.6f}"
    prec = {"c64": "complex64 state, FP32 boundary contraction, FP64 reductions",
            "tf32x3": "complex64 state, 3xTF32 tensor-core boundary contraction (FP32 accumulate), FP64 reductions",
            "fp16x3": "complex64 state, split-FP16 tensor-core boundary contraction (power-of-two scaled hi + lo, "
                      "three products, FP32 accumulate), FP64 reductions",
            "fp64": "complex128 throughout"}[w.precision]
    return {"workload": w.name, "grid": list(w.shape), "h": w.h, "n_orb": w.n_orb, "order": w.order, "s1": w.s,
            "dt": w.dt, "potential": pot, "precision": prec, "l2": l2}


def reference_arm(args, w):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    steps = args.steps if args.steps is not None else w.steps
    cb = cpu_oracle_sample(w, steps=max(1, steps), budget_s=25.0)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def peaks():
    pk = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        pk = json.load(open(p))
    src = "measured" if "hbm_gbs" in pk else "fallback"
    return {"hbm_gbs": pk.get("hbm_gbs", 6800.0), "bf16_tflops": pk.get("bf16_tflops", 1900.0),
            "bf16_tflops_sustained": pk.get("bf16_tflops_sustained", 1700.0), "source": src}


def cublas_tf32_tflops(dev):
    """Context only: a cuBLAS TF32 GEMM (8192^3, best of 5) on this GPU."""
    import torch
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    a = torch.randn(8192, 8192, device=dev)
    b = torch.randn(8192, 8192, device=dev)
    for _ in range(2):
        a @ b
    best = 1e9
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    torch.backends.cuda.matmul.allow_tf32 = old
    del a, b
    return 2 * 8192 ** 3 / best / 1e12


# ----------------------------------------------------------------------
# native arm: a full line for the 96^3 x 128-orbital mean-field workload (default) or the
# 64^3 single-orbital one
# ----------------------------------------------------------------------
def measure(args, w, rank, world, dev, extra_lines=True):
    import torch

    from paper_1908_02456_gb300 import abc
    steps = args.steps if args.steps is not None else w.steps
    psi0, V = inputs_for(w)
    ctx = abc.Context(w.shape, w.h, w.order, w.s, precision=w.precision, max_orbitals=w.n_orb)
    psi = torch.from_numpy(psi0).to(dev, ctx.complex_dtype)
    aux = ctx.new_aux(w.n_orb)
    Vt = torch.from_numpy(V).to(dev, ctx.real_dtype)
    stream = torch.cuda.current_stream()
    mf = w.meanfield
    units = float(w.n_orb) * np.prod(w.shape) * steps
    state_bytes = w.n_orb * np.prod(w.shape) * 8
    big = state_bytes > 2 * L2_BYTES

    # per-shape kernel choices (untimed set-up, on a copy of the state)
    from paper_1908_02456_gb300 import tune
    if args.no_tune:
        tuned = {"setting": {}, "sweep": None}
    elif args.reuse_tuning:
        tuned = tune.tune(ctx, psi, aux, Vt, w.dt, meanfield=mf, use_cache=True)
    else:
        tuned = tune.tune(ctx, psi, aux, Vt, w.dt, meanfield=mf, use_cache=False)
        tune.tune(ctx, psi, aux, Vt, w.dt, meanfield=mf, use_cache=True, fresh=tuned)
    if args.knob:
        tuned = dict(tuned, knobs=apply_knobs(ctx, args.knob))
    # warm-up (also captures the CUDA graph)
    ctx.run(psi, aux, Vt, w.dt, max(args.warmup, 1), meanfield=mf)
    torch.cuda.synchronize()
    flush = None if big else torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    launches0 = ctx.launches()
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        torch.cuda.synchronize()
        if big:
            # every array is many times L2: the steps run back to back as one replay
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.run(psi, aux, Vt, w.dt, steps, meanfield=mf)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
        else:
            # the boundary tiles alone fit in L2: flush before every step, each step timed
            # by its own event pair on the launching stream, the flush outside the pairs
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for i in range(steps):
                flush.fill_(float(i & 7))
                ev[i][0].record(stream)
                ctx.run(psi, aux, Vt, w.dt, 1, meanfield=mf)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            sec = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
        barrier()
    gpu_launches = ctx.launches() - launches0
    tot_units, max_sec = aggregate(units, sec)
    out = {"value": tot_units / max_sec, "ms_per_step": max_sec / steps * 1e3, "steps": steps,
           "clocks": clk.summary(), "gpu_launches": gpu_launches,
           "tuning": {"setting": tune.describe(tuned.get("setting", {})), "sweep_ms_per_step": tuned.get("sweep"),
                      "knobs": tuned.get("knobs")}}

    # dominant kernels: live CUDA-event timing of every launch over eager steps on the
    # launching stream (no graph), the same flush policy as the timed steps
    nprof = min(steps, 10 if big else 500)
    # the stencil runs after the boundary chain in these steps (placement 2), so that each
    # event pair times its kernel alone, not beside another stage's kernels
    placement = ctx.get_tuning(abc.TUNE_STENCIL)
    ctx.set_tuning(abc.TUNE_STENCIL, 2)
    ctx.profile(True)
    torch.cuda._sleep(40_000_000)          # the host queues the launches ahead of the GPU
    for i in range(nprof):
        if flush is not None:
            flush.fill_(float(i & 7))
        ctx.run(psi, aux, Vt, w.dt, 1, meanfield=mf)
    ms_c, n_c = ctx.profile_read(abc.KERNEL_CONTRACTION)
    ms_s, n_s = ctx.profile_read(abc.KERNEL_STENCIL)
    ms_p, n_p = ctx.profile_read(abc.KERNEL_PACK)
    per = ctx.profile_durations(abc.KERNEL_CONTRACTION)
    ctx.profile(False)
    ctx.set_tuning(abc.TUNE_STENCIL, placement)
    pk = peaks()
    hbm = pk["hbm_gbs"]
    bytes_c = ctx.kernel_bytes(abc.KERNEL_CONTRACTION, w.n_orb)
    bytes_s = ctx.kernel_bytes(abc.KERNEL_STENCIL, w.n_orb)
    useful, issued = ctx.kernel_flops(abc.KERNEL_CONTRACTION, w.n_orb)
    avg_c = ms_c / n_c * 1e-3
    avg_s = ms_s / n_s * 1e-3
    ach_s = bytes_s / avg_s / 1e9
    fused = ctx.get_tuning(abc.TUNE_FUSED) == 1 or (ctx.get_tuning(abc.TUNE_FUSED) == -1 and w.n_orb >= 2)
    kz = ctx.get_tuning(abc.TUNE_STENCIL_KZ)
    form = ("stencil_stage_x2z2" if w.n_orb == 1 else
            "stencil_stage_x2_bulk" if ctx.get_tuning(abc.TUNE_STENCIL_STAGED) == 1 else
            "stencil_stage_x2_lb<8>" if kz == 1 else "stencil_stage_x2" if kz == 0 else f"stencil_stage_x2zk<{kz}>")
    sname = ("stencil_bulk4 (the four Horner stages' interior fused in time)" if fused else
             f"{form} (fused stencil + potential + Horner stage)")
    stencil = {"bound": "hbm", "kernel": sname,
               "achieved": round(ach_s, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach_s / hbm, 4),
               "avg_launch_us": round(avg_s * 1e6, 2), "bytes_per_launch": bytes_s, "launches_timed": n_s,
               "timing": "CUDA events around each launch in eager steps with the kernels serialised"}
    traffic = traffic_for(w)
    if w.n_orb > 1 and w.precision in ("tf32x3", "fp16x3"):
        if w.precision == "tf32x3":
            peak = pk["bf16_tflops_sustained"] * TF32_PER_BF16
            peak_note = (f"TF32: the {pk['source']} sustained bf16 peak {pk['bf16_tflops_sustained']} TFLOP/s x "
                         f"1.1/2.25 (nominal dense TF32/BF16 ratio); the kernel runs inside a seconds-long loop")
            kern = "gemm_tc (tcgen05 kind::tf32, 3xTF32 boundary DtN contraction)"
        else:
            peak = pk["bf16_tflops_sustained"]
            peak_note = (f"FP16: the {pk['source']} sustained bf16 peak (same nominal dense rate); the kernel runs "
                         f"inside a seconds-long loop")
            kern = "gemm_tc (tcgen05 kind::f16, split-FP16 boundary DtN contraction)"
        ach = issued / avg_c / 1e12
        roofline = {"bound": "tensor", "kernel": kern, "achieved": round(ach, 1), "peak": round(peak, 1),
                    "unit": "TFLOP/s", "frac": round(ach / peak, 4), "peak_source": pk["source"],
                    "peak_note": peak_note, "traffic": traffic,
                    "flops_issued_per_launch": issued, "flops_useful_per_launch": useful,
                    "useful_tflops": round(useful / avg_c / 1e12, 1), "bytes_per_launch": bytes_c,
                    "hbm_frac_of_bytes": round(bytes_c / avg_c / 1e9 / hbm, 4),
                    "avg_launch_us": round(avg_c * 1e6, 2), "launches_timed": n_c,
                    "frac_of_burst": round(ach / (pk["bf16_tflops"] * (TF32_PER_BF16 if w.precision == "tf32x3"
                                                                        else 1.0)), 4),
                    "pack_avg_launch_us": round(ms_p / max(n_p, 1) * 1e3, 2),
                    "stencil": stencil}
        try:
            roofline["cublas_tf32_tflops_context"] = round(cublas_tf32_tflops(dev), 1)
        except Exception:
            pass
    else:
        ach = bytes_c / avg_c / 1e9
        cold_ms = float(np.mean(per[0::4])) if len(per) >= 4 else None   # first stage after the flush
        warm_ms = float(np.mean(np.concatenate([per[1::4], per[2::4], per[3::4]]))) if len(per) >= 4 else None
        roofline = {"bound": "hbm", "kernel": "sym_gemv_tiles (boundary DtN contraction)", "achieved": round(ach, 1),
                    "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4), "peak_source": pk["source"],
                    "traffic": traffic, "bytes_per_launch": bytes_c, "avg_launch_us": round(avg_c * 1e6, 2),
                    "launches_timed": n_c,
                    "cold_launch_us": round(cold_ms * 1e3, 2) if cold_ms else None,
                    "cold_frac": round(bytes_c / (cold_ms * 1e-3) / 1e9 / hbm, 4) if cold_ms else None,
                    "warm_launch_us": round(warm_ms * 1e3, 2) if warm_ms else None,
                    "cold_warm_note": "cold = first stage after the L2 flush (tiles from HBM); warm = stages 2-4 "
                                      "(tiles resident in L2 from the previous stage)",
                    "stencil": dict(stencil, note="state is L2-resident at b = 1 (2 MB per array)")}
    out["roofline"] = roofline

    # end to end through the C ABI on pinned host buffers
    psi_h = torch.from_numpy(psi0.astype(np.complex64)).pin_memory()
    aux_h = torch.zeros((ctx.n_gamma, w.n_orb), dtype=torch.complex64).pin_memory()
    V_h = torch.from_numpy(V.astype(np.float32)).pin_memory()
    # warm-up call (untimed): the context's device copies of the state are allocated and
    # the step graph for them captured on the first call, as for any caller that steps
    # repeatedly; then the inputs are restored
    ctx.run_host(psi_h, aux_h, V_h, w.dt, max(args.warmup, 1), meanfield=mf)
    psi_h.copy_(torch.from_numpy(psi0.astype(np.complex64)))
    aux_h.zero_()
    if flush is not None:
        flush.fill_(1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.run_host(psi_h, aux_h, V_h, w.dt, steps, meanfield=mf)
    e2e_sec = time.perf_counter() - t0
    del flush
    tot_e2e, max_e2e = aggregate(units, e2e_sec)
    h2d = psi_h.numel() * 8 + aux_h.numel() * 8 + V_h.numel() * 4
    d2h = psi_h.numel() * 8 + aux_h.numel() * 8
    out["e2e"] = {"value": tot_e2e / max_e2e, "unit": METRIC, "h2d_bytes_per_step": h2d / steps,
                  "d2h_bytes_per_step": d2h / steps,
                  "call": "abc_run_host: copy psi, f, V in from pinned host memory; run the steps; copy psi, f out"}

    # the 3xTF32 tensor-core form of the same workload (context for the split-FP16 GEMM)
    if w.precision == "fp16x3" and not args.no_fp64:
        ctx_t = abc.Context(w.shape, w.h, w.order, w.s, precision="tf32x3", max_orbitals=w.n_orb)
        pt = torch.from_numpy(psi0).to(dev, torch.complex64)
        at = ctx_t.new_aux(w.n_orb)
        ctx_t.run(pt, at, Vt, w.dt, 2, meanfield=mf)
        nt = min(steps, 50)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        g0.record(stream)
        ctx_t.run(pt, at, Vt, w.dt, nt, meanfield=mf)
        g1.record(stream)
        torch.cuda.synchronize()
        st_ = g0.elapsed_time(g1) * 1e-3
        ctx_t.profile(True)
        ctx_t.run(pt, at, Vt, w.dt, 2, meanfield=mf)
        ms_t, n_t = ctx_t.profile_read(abc.KERNEL_CONTRACTION)
        ctx_t.profile(False)
        out["tf32x3_form"] = {"value": w.n_orb * np.prod(w.shape) * nt / st_, "ms_per_step": st_ / nt * 1e3,
                              "gemm_avg_launch_us": round(ms_t / n_t * 1e3, 2),
                              "gemm_tflops_issued": round(issued / (ms_t / n_t * 1e-3) / 1e12, 1)}
        ctx_t.close()

    # plain FP64 GPU form on the same inputs, and the reduced form's distance from it
    if not args.no_fp64:
        ctx64 = abc.Context(w.shape, w.h, w.order, w.s, precision="fp64", max_orbitals=w.n_orb)
        p64 = torch.from_numpy(psi0).to(dev)
        a64 = ctx64.new_aux(w.n_orb)
        V64 = torch.from_numpy(V).to(dev)
        p32 = torch.from_numpy(psi0).to(dev, torch.complex64)
        a32 = ctx.new_aux(w.n_orb)
        n64 = min(steps, 3 if big else 400)
        ctx64.run(p64, a64, V64, w.dt, 1, meanfield=mf)
        ctx.run(p32, a32, Vt, w.dt, 1, meanfield=mf)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ctx64.run(p64, a64, V64, w.dt, n64, meanfield=mf)
        f1.record(stream)
        ctx.run(p32, a32, Vt, w.dt, n64, meanfield=mf)
        torch.cuda.synchronize()
        s64 = f0.elapsed_time(f1) * 1e-3
        err = float(torch.linalg.norm(p32.to(torch.complex128) - p64) / torch.linalg.norm(p64))
        ferr = float(torch.linalg.norm(a32.to(torch.complex128) - a64) / torch.linalg.norm(a64))
        # the FP64 contraction's own rate, against the cuBLAS FP64 GEMM of this part
        ctx64.profile(True)
        ctx64.run(p64, a64, V64, w.dt, 1, meanfield=mf)
        ms64, n64c = ctx64.profile_read(abc.KERNEL_CONTRACTION)
        ctx64.profile(False)
        _, iss64 = ctx64.kernel_flops(abc.KERNEL_CONTRACTION, w.n_orb)
        fp64_gemm = {"avg_launch_ms": round(ms64 / n64c, 3),
                     "tflops": round(iss64 / (ms64 / n64c * 1e-3) / 1e12, 3),
                     "frac_of_cublas_fp64": round(iss64 / (ms64 / n64c * 1e-3) / 1e12 / FP64_CUBLAS_TFLOPS, 3)}
        out["fp64_form"] = {"value": w.n_orb * np.prod(w.shape) * n64 / s64, "ms_per_step": s64 / n64 * 1e3,
                            "steps": n64 + 1, "psi_rel_l2_vs_fp64": err, "aux_rel_l2_vs_fp64": ferr, "dtype": "f64",
                            "contraction": fp64_gemm,
                            "fp64_peak_note": f"cuBLAS FP64 GEMM measured {FP64_CUBLAS_TFLOPS} TFLOP/s on this part"}
        ctx64.close()
    ctx.close()
    return out


def traffic_for(w):
    """DRAM bytes per launch of the dominant kernel from a committed ncu capture, if the
    kernel source has not changed since."""
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tr_path):
        return None
    key = "contraction_c64_64cube" if w.n_orb == 1 else f"gemm_tc_{w.name}_{w.precision}"
    tr = json.load(open(tr_path)).get(key)
    if tr and tr.get("kernel_stamp") == ctx_stamp(tr.get("kernel_file", "sym_gemv.cuh")):
        return tr["bytes_per_launch"]
    return None


def inputs_for(w):
    from paper_1908_02456_gb300 import inputs
    return inputs.make_inputs(w)


def apply_knobs(ctx, knobs):
    """Set the --knob NAME=VALUE tuning knobs on a context; returns them as a dict."""
    from paper_1908_02456_gb300 import abc
    out = {}
    for kv in knobs:
        name, value = kv.split("=")
        ctx.set_tuning(getattr(abc, "TUNE_" + name.strip().upper()), int(value))
        out[name.strip().upper()] = int(value)
    return out


def other_workload(args, w):
    """One line for a workload without a full line: K time steps (mean-field workloads:
    the potential is rebuilt from the density every step) or, for the adjoint workload,
    one forward + reverse sweep of K steps; the oracle is not timed."""
    import torch
    from paper_1908_02456_gb300 import abc
    from paper_1908_02456_gb300 import build as nbuild
    nbuild.build()
    steps = args.steps if args.steps is not None else w.steps
    dev = torch.device("cuda", torch.cuda.current_device())
    psi0, V = inputs_for(w)
    ctx = abc.Context(w.shape, w.h, w.order, w.interp, precision=w.precision, max_orbitals=w.n_orb,
                      fit1=w.fit1, s1b=w.s1b, radius=w.radius)
    psi = torch.from_numpy(psi0).to(dev, ctx.complex_dtype)
    aux = ctx.new_aux(w.n_orb) if w.order == 1 else ctx.init_aux(psi) if w.order == 2 else None
    Vt = torch.from_numpy(V).to(dev, ctx.real_dtype)
    knobs = apply_knobs(ctx, args.knob)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    units = float(w.n_orb) * np.prod(w.shape) * steps
    if w.number == 4:
        ctx.adjoint(psi, Vt, w.dt, max(args.warmup, 1), ckpt_every=50)
        flush.fill_(0.0)
        torch.cuda.synchronize()
        launches0 = ctx.launches()
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            ctx.adjoint(psi, Vt, w.dt, steps, ckpt_every=50)
            e1.record(stream)
            torch.cuda.synchronize()
        what = "forward sweep + checkpointed reverse sweep (abc_adjoint_run), L2 flushed before the call"
    else:
        ctx.run(psi, aux, Vt, w.dt, max(args.warmup, 1), meanfield=w.meanfield)
        flush.fill_(0.0)
        torch.cuda.synchronize()
        launches0 = ctx.launches()
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            ctx.run(psi, aux, Vt, w.dt, steps, meanfield=w.meanfield)
            e1.record(stream)
            torch.cuda.synchronize()
        what = "graph-replayed steps, L2 flushed once before the timed run"
    sec = e0.elapsed_time(e1) * 1e-3
    launches = ctx.launches() - launches0
    # contraction timing over a short profiled run
    nprof = min(steps, 50)
    ctx.profile(True)
    if w.number == 4:
        ctx.run(psi, aux, Vt, w.dt, nprof)
    else:
        ctx.run(psi, aux, Vt, w.dt, nprof, meanfield=w.meanfield)
    ms_c, n_c = ctx.profile_read(abc.KERNEL_CONTRACTION)
    ctx.profile(False)
    bytes_c = ctx.kernel_bytes(abc.KERNEL_CONTRACTION, w.n_orb)
    line = {"metric": METRIC, "value": units / sec, "unit": METRIC, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": sec / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w.precision == "fp64" else "c64",
            "data": "synthetic", "config": {"workload": w.name, "grid": list(w.shape), "h": w.h, "n_orb": w.n_orb,
                                           "order": w.order, "s": w.interp, "fit1": w.fit1, "s1b": w.s1b,
                                           "radius": w.radius,
                                           "dt": w.dt, "meanfield": w.meanfield,
                                           "precision": w.precision, "what": what},
            "contraction": {"avg_launch_us": round(ms_c / n_c * 1e3, 2), "bytes_per_launch": bytes_c,
                            "achieved_gbs": round(bytes_c / (ms_c / n_c * 1e-3) / 1e9, 1)},
            "clocks": clk.summary(), "gpu_launches": launches, "knobs": knobs}
    print(json.dumps(line))
    ctx.close()


def main():
    args = parse()
    from paper_1908_02456_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        return reference_arm(args, w)
    if args.workload not in (WORKLOAD_NUMBER, SINGLE_ORBITAL_WORKLOAD):
        return other_workload(args, w)

    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1908_02456_gb300 import build as nbuild
    nbuild.build()

    res = measure(args, w, rank, world, dev)
    single = None
    if w.number == WORKLOAD_NUMBER and not args.no_extra:
        # the single-orbital harmonic-well workload (64^3, b = 1), its own flushed steps
        w2 = inputs.WORKLOADS[SINGLE_ORBITAL_WORKLOAD]
        a2 = argparse.Namespace(**vars(args))
        a2.steps, a2.no_fp64 = 200, True
        r2 = measure(a2, w2, rank, world, dev)
        single = {"config": config_dict(w2), "value": r2["value"], "ms_per_step": r2["ms_per_step"],
                  "steps": r2["steps"], "roofline": r2["roofline"], "e2e": r2["e2e"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w, steps=100, budget_s=20.0)

    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": METRIC, "n_gpus": world, "steps": res["steps"],
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
                "config": config_dict(w), "roofline": res["roofline"], "cpu_baseline": cpu, "e2e": res["e2e"],
                "clocks": res["clocks"], "gpu_launches": res["gpu_launches"], "fp64_form": res.get("fp64_form"),
                "tf32x3_form": res.get("tf32x3_form"), "tuning": res.get("tuning"),
                "single_orbital": single, "parallelism": "replicas" if world > 1 else "single"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def ctx_stamp(source="sym_gemv.cuh"):
    """Hash of the source of the kernel a traffic figure was measured on."""
    import hashlib
    h = hashlib.sha256()
    p = os.path.join(ROOT, "paper_1908_02456_gb300", "csrc", source)
    h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
