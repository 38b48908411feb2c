"""Throughput benchmark of the discrete-DtN ABC time-stepper on GB300.

Workload: the single-orbital harmonic-well case -- 64^3 interior grid, h = 0.4,
first-order ABC interpolated at s1 = 1, V = 0.5*0.3^2 r^2 + 8 seeded Gaussian bumps,
one Gaussian packet (|k| = 2), dt = 0.005 -- in the complex64 form (FP32 arithmetic,
FP32 boundary contraction).  A "step" is one time step: 4 Horner stages, each a
boundary DtN contraction plus the fused stencil / potential / integrator kernel.

metric: orbital*gridpoint*steps/s (b * N^3 * steps / time), higher is better.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 is launched by torchrun: every rank runs an independent replica on its own
GPU (the path has no exchange step), timing is max over ranks and ``value`` is the
sum of all ranks' units over that time ("weak" scaling).  ``--impl reference`` times
the FP64 CPU oracle on the same workload (a bounded sample of steps) instead.
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
WORKLOAD_NUMBER = 2
L2_FLUSH_BYTES = 256 << 20          # written before every timed step (L2 is 129 MB)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU form")
    ap.add_argument("--workload", type=int, default=WORKLOAD_NUMBER,
                    help="1-5; the default (2) is the benchmark line, the others print a line of their own")
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
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ----------------------------------------------------------------------
def cpu_oracle_sample(w, steps: int, budget_s: float = 20.0):
    """Time the FP64 oracle's step on the full workload grid.  Its DtN matrix setup at
    this size (a dense 23816^2 complex solve) takes far longer than a benchmark allows,
    so B is a seeded complex stand-in of the same size and A the diagonal of the
    order-1 ABC; the step's cost does not depend on their values."""
    import scipy.sparse as sp

    from oracle.lattice import Box, n_gamma
    from oracle.propagate import System
    from paper_1908_02456_gb300 import inputs

    psi0, V = inputs.make_inputs(w)
    box = Box(w.shape, w.h)
    ng = n_gamma(w.shape, 1)
    rng = np.random.default_rng(1)
    B = np.empty((ng, ng), dtype=np.complex128)
    for i in range(0, ng, 2048):
        blk = rng.standard_normal((min(2048, ng - i), ng * 2))
        B[i:i + blk.shape[0]] = (blk[:, 0::2] + 1j * blk[:, 1::2]) * 1e-3
    A = sp.diags(np.full(ng, -1j / (4 * w.h ** 4)))
    sysm = System(box, V_ext=V.reshape(-1), coeffs={"order": 1, "A": A, "B": B, "Q": None})
    phi = psi0.reshape(1, -1)
    f = np.zeros((1, ng), np.complex128)
    phi, f = sysm.step(phi, f, w.dt)          # warm-up
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        phi, f = sysm.step(phi, f, w.dt)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    sec = time.perf_counter() - t0
    threads = os.environ.get("OMP_NUM_THREADS") or os.environ.get("OPENBLAS_NUM_THREADS") or str(os.cpu_count())
    return {"value": w.n_orb * box.n * done / sec, "unit": METRIC, "cores": int(threads), "kind": "oracle",
            "sample": f"{done} steps of the oracle's Taylor step on the full {w.n}^3 grid "
                      f"(sparse stencil + dense {ng}x{ng} complex128 B stand-in), {sec:.1f} s"}


def reference_arm(args, w):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    cb = cpu_oracle_sample(w, steps=max(1, args.steps), budget_s=25.0)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_dict(w, matrix_mb=None):
    l2 = f"L2 flushed before every timed step ({L2_FLUSH_BYTES >> 20} MiB write; L2 is 129 MB)"
    l2 += f"; packed boundary tiles {matrix_mb:.0f} MB" if matrix_mb else ""
    return {"workload": w.name, "grid": list(w.shape), "h": w.h, "n_orb": w.n_orb, "order": w.order,
            "s1": w.s, "dt": w.dt, "potential": "0.5*0.09*r^2 + 8 seeded Gaussian bumps",
            "precision": "complex64 state, FP32 boundary contraction, FP64 reductions", "l2": l2}


# ----------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------
def other_workload(args, w):
    """One line for a workload other than the benchmark one: K time steps (mean-field
    workloads: the potential is rebuilt from the density every step) or, for the
    adjoint workload, one forward + reverse sweep of K steps; the oracle is not timed."""
    import torch
    from paper_1908_02456_gb300 import abc
    from paper_1908_02456_gb300 import build as nbuild
    nbuild.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    psi0, V = inputs_for(w)
    ctx = abc.Context(w.shape, w.h, w.order, w.interp, precision=w.precision, max_orbitals=w.n_orb,
                      fit1=w.fit1, s1b=w.s1b, radius=w.radius)
    psi = torch.from_numpy(psi0).to(dev, ctx.complex_dtype)
    aux = ctx.new_aux(w.n_orb) if w.order == 1 else ctx.init_aux(psi) if w.order == 2 else None
    Vt = torch.from_numpy(V).to(dev, ctx.real_dtype)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    units = float(w.n_orb) * np.prod(w.shape) * args.steps
    if w.number == 4:
        ctx.adjoint(psi, Vt, w.dt, max(args.warmup, 1), ckpt_every=50)
        flush.fill_(0.0)
        torch.cuda.synchronize()
        launches0 = ctx.launches()
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            J, g = ctx.adjoint(psi, Vt, w.dt, args.steps, ckpt_every=50)
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
            ctx.run(psi, aux, Vt, w.dt, args.steps, meanfield=w.meanfield)
            e1.record(stream)
            torch.cuda.synchronize()
        what = "graph-replayed steps, L2 flushed once before the timed run"
    sec = e0.elapsed_time(e1) * 1e-3
    launches = ctx.launches() - launches0
    # contraction timing over a short profiled run
    nprof = min(args.steps, 50)
    ctx.profile(True)
    if w.number == 4:
        ctx.run(psi, aux, Vt, w.dt, nprof)
    else:
        ctx.run(psi, aux, Vt, w.dt, nprof, meanfield=w.meanfield)
    ms_c, n_c = ctx.profile_read(abc.KERNEL_CONTRACTION)
    ctx.profile(False)
    bytes_c = ctx.kernel_bytes(abc.KERNEL_CONTRACTION, w.n_orb)
    line = {"metric": METRIC, "value": units / sec, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w.precision == "fp64" else "c64",
            "data": "synthetic", "config": {"workload": w.name, "grid": list(w.shape), "h": w.h, "n_orb": w.n_orb,
                                           "order": w.order, "s": w.interp, "fit1": w.fit1, "s1b": w.s1b,
                                           "radius": w.radius,
                                           "dt": w.dt, "meanfield": w.meanfield,
                                           "precision": w.precision, "what": what},
            "contraction": {"avg_launch_us": round(ms_c / n_c * 1e3, 2), "bytes_per_launch": bytes_c,
                            "achieved_gbs": round(bytes_c / (ms_c / n_c * 1e-3) / 1e9, 1)},
            "clocks": clk.summary(), "gpu_launches": launches}
    print(json.dumps(line))
    ctx.close()


def inputs_for(w):
    from paper_1908_02456_gb300 import inputs
    return inputs.make_inputs(w)


def main():
    args = parse()
    from paper_1908_02456_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        return reference_arm(args, w)
    if args.workload != WORKLOAD_NUMBER:
        return other_workload(args, w)

    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1908_02456_gb300 import abc
    from paper_1908_02456_gb300 import build as nbuild
    nbuild.build()
    psi0, V = inputs.make_inputs(w)
    ctx = abc.Context(w.shape, w.h, w.order, w.s, precision="c64", max_orbitals=w.n_orb)
    psi = torch.from_numpy(psi0).to(dev, torch.complex64)
    aux = ctx.new_aux(w.n_orb)
    Vt = torch.from_numpy(V).to(dev, torch.float32)
    stream = torch.cuda.current_stream()

    # warm-up (also captures the CUDA graph)
    ctx.run(psi, aux, Vt, w.dt, max(args.warmup, 1))
    torch.cuda.synchronize()
    # L2 is flushed before every timed step by writing a buffer twice its size (the
    # boundary tiles alone fit in L2); each step is timed by its own event pair on
    # the launching stream and the flush stays outside the pairs
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = ctx.launches()
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i & 7))
            ev[i][0].record(stream)
            ctx.run(psi, aux, Vt, w.dt, 1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
    sec = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    gpu_launches = ctx.launches() - launches0
    units = float(w.n_orb) * np.prod(w.shape) * args.steps
    tot_units, max_sec = aggregate(units, sec)
    value = tot_units / max_sec

    # steady state for context: the same steps as one graph-replayed run, no flush
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.run(psi, aux, Vt, w.dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    warm_sec = e0.elapsed_time(e1) * 1e-3
    steady = {"value": units / warm_sec, "ms_per_step": warm_sec / args.steps * 1e3,
              "note": "one run of the same number of steps, L2 not flushed between steps"}

    # dominant kernel: live CUDA-event timing of every contraction launch over the
    # same flushed steps on the launching stream (eager launches, no graph)
    nprof = min(args.steps, 500)
    ctx.profile(True)
    # a ~20 ms spin first, so the host queues the profiled launches ahead of the GPU and
    # each event pair times its kernel, not the host's launch latency
    torch.cuda._sleep(40_000_000)
    for i in range(nprof):
        flush.fill_(float(i & 7))
        ctx.run(psi, aux, Vt, w.dt, 1)
    ms_c, n_c = ctx.profile_read(abc.KERNEL_CONTRACTION)
    ms_s, n_s = ctx.profile_read(abc.KERNEL_STENCIL)
    per = ctx.profile_durations(abc.KERNEL_CONTRACTION)
    ctx.profile(False)
    cold_ms = float(np.mean(per[0::4])) if len(per) >= 4 else None   # first stage after the flush
    warm_ms = float(np.mean(np.concatenate([per[1::4], per[2::4], per[3::4]]))) if len(per) >= 4 else None
    bytes_c = ctx.kernel_bytes(abc.KERNEL_CONTRACTION, w.n_orb)
    bytes_s = ctx.kernel_bytes(abc.KERNEL_STENCIL, w.n_orb)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    ach_c = bytes_c / (ms_c / n_c * 1e-3) / 1e9
    ach_s = bytes_s / (ms_s / n_s * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        tr = json.load(open(tr_path)).get("contraction_c64_64cube")
        if tr and tr.get("kernel_stamp") == ctx_stamp():
            traffic = tr["bytes_per_launch"]
    roofline = {"bound": "hbm", "kernel": "sym_gemv_tiles (boundary DtN contraction)",
                "achieved": round(ach_c, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(ach_c / hbm_peak, 4),
                "peak_source": peak_src, "traffic": traffic,
                "bytes_per_launch": bytes_c, "avg_launch_us": round(ms_c / n_c * 1e3, 2), "launches_timed": n_c,
                "cold_launch_us": round(cold_ms * 1e3, 2) if cold_ms else None,
                "cold_frac": round(bytes_c / (cold_ms * 1e-3) / 1e9 / hbm_peak, 4) if cold_ms else None,
                "warm_launch_us": round(warm_ms * 1e3, 2) if warm_ms else None,
                "cold_warm_note": "cold = first stage after the L2 flush (tiles from HBM); warm = stages 2-4 "
                                  "(tiles resident in L2 from the previous stage)",
                "stencil": {"achieved": round(ach_s, 1), "frac": round(ach_s / hbm_peak, 4),
                            "avg_launch_us": round(ms_s / n_s * 1e3, 2), "bytes_per_launch": bytes_s,
                            "note": "state is L2-resident at b = 1 (2 MB per array)"}}

    # end to end through the C ABI on pinned host buffers
    psi_h = torch.from_numpy(psi0.astype(np.complex64)).pin_memory()
    aux_h = torch.zeros((ctx.n_gamma, w.n_orb), dtype=torch.complex64).pin_memory()
    V_h = torch.from_numpy(V.astype(np.float32)).pin_memory()
    flush.fill_(1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.run_host(psi_h, aux_h, V_h, w.dt, args.steps)
    e2e_sec = time.perf_counter() - t0
    del flush
    tot_e2e, max_e2e = aggregate(units, e2e_sec)
    h2d = psi_h.numel() * 8 + aux_h.numel() * 8 + V_h.numel() * 4
    d2h = psi_h.numel() * 8 + aux_h.numel() * 8
    e2e = {"value": tot_e2e / max_e2e, "unit": METRIC, "h2d_bytes_per_step": h2d / args.steps,
           "d2h_bytes_per_step": d2h / args.steps,
           "call": "abc_run_host: copy psi, f, V in; run the steps; copy psi, f out (L2 flushed before the call)"}

    # plain FP64 GPU form on the same inputs
    fp64 = None
    if not args.no_fp64:
        ctx64 = abc.Context(w.shape, w.h, w.order, w.s, precision="fp64", max_orbitals=w.n_orb)
        p64 = torch.from_numpy(psi0).to(dev)
        a64 = ctx64.new_aux(w.n_orb)
        V64 = torch.from_numpy(V).to(dev)
        p32 = torch.from_numpy(psi0).to(dev, torch.complex64)
        a32 = ctx.new_aux(w.n_orb)
        n64 = min(args.steps, 400)
        ctx64.run(p64, a64, V64, w.dt, 2)
        ctx.run(p32, a32, Vt, w.dt, 2)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ctx64.run(p64, a64, V64, w.dt, n64)
        f1.record(stream)
        ctx.run(p32, a32, Vt, w.dt, n64)
        torch.cuda.synchronize()
        s64 = f0.elapsed_time(f1) * 1e-3
        err = float(torch.linalg.norm(p32.to(torch.complex128) - p64) / torch.linalg.norm(p64))
        fp64 = {"value": w.n_orb * np.prod(w.shape) * n64 / s64, "ms_per_step": s64 / n64 * 1e3, "steps": n64,
                "c64_vs_fp64_rel_l2": err, "dtype": "f64"}
        ctx64.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w, steps=100, budget_s=20.0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_sec / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
                "config": config_dict(w, bytes_c / 1e6), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk.summary(), "gpu_launches": gpu_launches, "fp64_form": fp64, "steady_state": steady,
                "parallelism": "replicas" if world > 1 else "single"}
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def ctx_stamp():
    """Hash of the source of the dominant kernel the traffic figure was measured on."""
    import hashlib
    h = hashlib.sha256()
    p = os.path.join(ROOT, "paper_1908_02456_gb300", "csrc", "sym_gemv.cuh")
    h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
