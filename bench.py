"""Benchmark of the fused thermocapillary phase-field LBM step on GB300.

Workload: the 512^3 periodic throughput lattice (64 seeded droplets, R in
[8, 20], weak gradient dT/dx = 1e-4), D3Q15 phase field, D3Q27 central-moment
hydrodynamics, D3Q7 thermal LB, PDFs in FP32 (shifted storage).  A step is
one full time step of all three LB sweeps (one fused kernel launch).  The
state (52.6 GB) is far larger than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  With --impl reference it times the FP64
oracle on the host cores instead (bounded crop of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused step MLUPS FP32 vs FP64 at stated error, % HBM roofline; adjoint/fwd cost"
STORE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2}
FIELD_BYTES = {"fp64": 8, "fp32": 4, "fp16": 4}
# Field values moved per cell and step by the RK schedules: RK2 = step kernel
# (T read, u and S1 written) + final stage (S1, u, T read, T written) = 11;
# RK4 = step kernel (T read; u, S1, acc written) + two middle stages (stage
# field, u, T read; next stage field written; acc read and written) + final
# stage (S3, u, T, acc read; T written) = 29.
RK_FIELDS = {"RK2": 11, "RK4": 29}


# Of those, the step kernel itself moves: RK2 T read, u (3) and S1 written = 5;
# RK4 the same plus acc written = 6 (the rest belongs to the stage kernels).
RK_FIELDS_STEP_KERNEL = {"RK2": 5, "RK4": 6}


def bytes_per_cell(precision: str, thermal: str, q_phase: int = 15) -> int:
    """Algorithmic bytes per cell update of a whole step: every PDF read once
    and written once, plus the stage fields of the RK energy solvers; halo
    re-reads (L2) and derived fields (phi, T, u computed in the kernel) are
    not counted."""
    qf = int(thermal[3:]) if thermal.startswith("D3Q") else 0
    pdf = 2 * (q_phase + 27 + qf) * STORE_BYTES[precision]
    return pdf + RK_FIELDS.get(thermal, 0) * FIELD_BYTES[precision]


def step_kernel_bytes_per_cell(precision: str, thermal: str, q_phase: int = 15) -> int:
    """Algorithmic bytes per cell of the step kernel alone (the RK stage
    kernels' field traffic excluded)."""
    qf = int(thermal[3:]) if thermal.startswith("D3Q") else 0
    pdf = 2 * (q_phase + 27 + qf) * STORE_BYTES[precision]
    return pdf + RK_FIELDS_STEP_KERNEL.get(thermal, 0) * FIELD_BYTES[precision]
FALLBACK_HBM_GBS = 6800.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Sources of the step kernels (step_kernel, step_bulk_kernel, step_skew_kernel):
# the headers they are built from and their instantiation units.  The other
# kernels (ghost fill, RK stages, in-place layout, adjoint) live in headers of
# their own and do not change the step kernels' code.
STEP_KERNEL_SOURCES = ("lbm_device.cuh", "lbm_cell.cuh", "lbm_step.cuh", "lbm_bulk.cuh", "lbm_skew.cuh",
                       "inst_step.cuh")


def kernel_source_sha() -> str:
    """Hash of the step kernels' device-code sources (the ncu counters in
    profiles/ are valid while it matches)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2401_03041_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in STEP_KERNEL_SOURCES or (name.startswith("inst_fp") and name.endswith(".cu")):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def timed_launch_count(kernel: str, thermal: str, steps: int, warmup: int) -> int:
    """Kernel launches of `steps` timed steps after `warmup` steps from the
    initial state (level 0): the step kernel, + the ghost fill after it with
    the tiled kernels (the generic one wraps its reads); in place, the (phi, T)
    pass + the step, + a ghost refresh and a fold around the tiled steps from
    even levels; + the RK stages of the finite-difference energy solvers."""
    rk_stages = 0 if thermal.startswith("D3Q") else (1 if thermal == "RK2" else 3)
    if kernel in ("skew", "bulk", "aa"):
        return steps * (2 + rk_stages)
    if kernel == "aa_tiled":
        n_even = (warmup + steps + 1) // 2 - (warmup + 1) // 2   # levels warmup .. warmup + steps - 1
        return steps * (2 + rk_stages) + 2 * n_even
    return steps * (1 + rk_stages)


# What each step-kernel choice of lbm_kernel_info is, for the roofline record.
KERNEL_NAMES = {
    "skew": "lbm::step_skew_kernel (fused h/g/f stream-collide, tensor-TMA staging, two threads per cell "
            "one plane apart)",
    "bulk": "lbm::step_bulk_kernel (fused h/g/f stream-collide, tensor-TMA staging, two threads per cell)",
    "generic": "lbm::step_kernel (fused, generic tiles)",
    "aa_tiled": "lbm::aa_moments_kernel + lbm::step_skew_kernel in place (tensor-TMA tiles) per step",
    "aa": "lbm::aa_moments_kernel + lbm::aa_step_kernel (in place, generic tiles) per step",
}


# FP64 peak of the GB300 (nominal): 152 SMs x 2 FP64 FMA lanes per cycle x 2 FLOP
# per FMA x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def counters_record(precision: str, thermal: str):
    """The committed ncu counters of one step-kernel launch for this precision
    and thermal option (profiles/step_kernel_counters.json), or None if the
    kernel sources changed since they were taken."""
    path = os.path.join(ROOT, "profiles", "step_kernel_counters.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("source_sha") != kernel_source_sha():
        return None
    for r in d.get("records", []):
        if (r.get("precision"), r.get("thermal")) == (precision, thermal):
            return r
    return None


def traffic_per_cell(precision: str, thermal: str):
    """DRAM bytes per cell update of the step kernel from the committed ncu
    record, with the lattice edge it was captured at, or None if the kernel
    sources changed since those counters were taken.  The capture is of a
    lattice whose state is far larger than L2 (>= 128^3), so the DRAM bytes
    per cell carry over to larger lattices of the same workload (the kernel's
    traffic is a fixed amount per cell plus per-tile halo re-reads that scale
    the same way)."""
    r = counters_record(precision, thermal)
    if not r or "dram_bytes_per_cell" not in r or int(r.get("n", 0)) < 128:
        return None
    return float(r["dram_bytes_per_cell"]), int(r["n"])


def cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the platform)."""
    import platform
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


_ORACLE_TIMER = """
import os, sys, time, json
sys.path.insert(0, {root!r})
import workloads as W
from oracle.model import build
w = W.crop(W.config4({thermal!r}, 'fp64'), {n}, {n}, {n})
o = build(w)
o.step(1)
t0 = time.perf_counter(); steps = 0
while time.perf_counter() - t0 < {seconds}:
    o.step(1); steps += 1
dt = time.perf_counter() - t0
print(json.dumps({{"mlups": w.cells * steps / dt / 1e6, "steps": steps, "seconds": dt,
                   "cells": w.cells, "name": w.name}}))
"""


def cpu_oracle_sample(seconds: float = 15.0, n: int = 48, thermal: str = "D3Q7", procs: int = 1):
    """Time the FP64 oracle, as it stands, on an n^3 crop of the throughput
    workload: ``procs`` fresh single-threaded processes (no CUDA in them) each
    step their own copy of the crop at the same time, one per host core (numpy
    runs one thread per process), like the GPU replicas.  Throughput is the
    sum over the processes of cells x steps / their own time."""
    code = _ORACLE_TIMER.format(root=ROOT, thermal=thermal, n=n, seconds=seconds)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True, env=env) for _ in range(procs)]
    outs = []
    for p in ps:
        out, err = p.communicate(timeout=600)
        if p.returncode != 0:
            raise RuntimeError("oracle timing failed: " + err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    r = dict(outs[0])
    r["mlups"] = sum(o["mlups"] for o in outs)
    r["steps"] = sum(o["steps"] for o in outs)
    r["seconds"] = max(o["seconds"] for o in outs)
    r["procs"] = procs
    return r


def max_over_ranks(v, world: int, device=None):
    """Maximum of a per-rank scalar over all ranks (the job's time is that of
    its slowest replica); device is where the collective's tensor lives
    (the rank's GPU under NCCL, the CPU under gloo)."""
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(cells_per_rank: int, steps: int, world: int, secs_max: float) -> float:
    """Whole-job throughput of N independent replicas (weak scaling): every
    rank updates cells_per_rank cells per step; the job takes as long as the
    slowest rank."""
    return cells_per_rank * steps * world / secs_max / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # each reference step is one oracle step on a 32^3 crop of the workload
    import workloads as W
    from oracle.model import build
    n = 32
    w = W.crop(W.config4(args.thermal, "fp64"), n, n, n)
    o = build(w)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    mlups = w.cells * args.steps / dt / 1e6
    sample = f"{w.name}: {n}^3 crop of the 512^3 workload, {args.steps} oracle steps (numpy FP64)"
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cfg4_512cube_periodic_64drops (oracle on a 32^3 crop)",
                       "thermal": args.thermal, "precision": "fp64"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512, help="lattice edge (default 512)")
    ap.add_argument("--thermal", default="D3Q7")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-cost leg")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the thermal option x storage sweep (kernel-only timing of each)")
    ap.add_argument("--sweep-steps", type=int, default=8)
    ap.add_argument("--no-aa", action="store_true", help="skip the in-place (AA) layout leg")
    ap.add_argument("--aa-large-n", type=int, default=1024,
                    help="edge of the large lattice run in the in-place layout (0: skip)")
    ap.add_argument("--layout", default="two_grid", choices=["two_grid", "aa"],
                    help="PDF layout of the main leg (aa: the in-place layout; for profiling it)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time the step kernel only (no CPU, e2e, FP64, sweep or error legs; for profiling)")
    args = ap.parse_args()
    if args.kernel_only:
        args.no_cpu = args.no_fp64 = args.no_adjoint = args.no_sweep = args.no_aa = True
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import workloads as W
    from paper_2401_03041_gb300 import build as B
    from paper_2401_03041_gb300 import lbm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def reduce_max(v):
        return max_over_ranks(v, world, dev)

    # CPU baseline first (spawned subprocess; no CUDA in it)
    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu:
        try:
            cpu = cpu_oracle_sample(seconds=12.0, n=48, thermal=args.thermal)
        except Exception as e:  # reported, not fatal
            cpu = {"error": str(e)[:300]}
        try:
            cpu_all = cpu_oracle_sample(seconds=12.0, n=48, thermal=args.thermal,
                                        procs=max(1, os.cpu_count() or 1))
        except Exception as e:
            cpu_all = {"error": str(e)[:300]}

    w = W.config4(args.thermal, args.precision, n=args.n)

    def make_domain(prec):
        d = lbm.Domain(w.nx, w.ny, w.nz, prec, w.thermal, w.q_phase, device=dev, layout=args.layout)
        d.set_params(w.params)
        d.init_droplets(w.droplets)
        return d

    def timed_steps(d, steps, warmup, sampler=None):
        # the clock sampler starts before the warm-up: nvidia-smi's start-up
        # must not fall inside the timed region (it stalls kernel launches)
        if sampler:
            sampler.start()
            time.sleep(1.5)
        d.step(warmup)
        torch.cuda.synchronize(dev)
        barrier()
        st = d.stream
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        d.profile_read()            # discard launches timed before this region
        d.profile_steps(True)
        e0.record(st)
        d.step(steps)
        e1.record(st)
        torch.cuda.synchronize(dev)
        d.profile_steps(False)
        kms, kn = d.profile_read()  # step-kernel launches alone (events on the same stream)
        clk = sampler.stop() if sampler else None
        barrier()
        return e0.elapsed_time(e1) / 1e3, clk, (kms / kn / 1e3 if kn else None)

    # ---------------- headline: FP32 (or --precision) fused step
    d = make_domain(args.precision)
    kinfo = d.kernel_info()
    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").isdigit() else local)
    secs, clocks, kernel_secs = timed_steps(d, args.steps, args.warmup, sampler)
    secs = reduce_max(secs)
    kernel_secs = reduce_max(kernel_secs) if kernel_secs else None
    cells = w.cells
    mlups = job_mlups(cells, args.steps, world, secs)
    per_step = secs / args.steps
    timed_launches = timed_launch_count(kinfo["kernel"], w.thermal, args.steps, args.warmup)

    # ---------------- e2e: a job through the C ABI with host buffers
    # init from the host droplet table, K steps each returning FP64
    # diagnostics to the host, final phi field copied to host memory.
    e2e = None
    if not args.kernel_only:
        host_phi = torch.empty((1, w.nz, w.ny, w.nx), dtype=torch.float32, pin_memory=True)
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        d.init_droplets(w.droplets)
        for _ in range(args.steps):
            d.step_diagnostics(1)
        d.fields(lbm.FIELD_PHI, dtype="f32", out=host_phi)
        torch.cuda.synchronize(dev)
        e2e_secs = reduce_max(time.perf_counter() - t0)
        barrier()
        e2e = {"value": cells * args.steps * world / e2e_secs / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": len(w.droplets) * 7 * 8 / args.steps,
               "d2h_bytes_per_step": (args.steps * 64 + 4 * cells) / args.steps,
               "what": "lbm_init_droplets from host table + K x lbm_step_diagnostics(1) "
                       "(FP64 diagnostics to host each step) + final phi to pinned host"}
    diag_final = d.diagnostics()
    del d
    torch.cuda.empty_cache()

    # ---------------- FP64 leg (same workload, fewer steps)
    fp64 = None
    if not args.no_fp64 and args.precision != "fp64":
        d64 = make_domain("fp64")
        s64, _, k64 = timed_steps(d64, args.fp64_steps, 3)
        s64 = reduce_max(s64)
        k64 = reduce_max(k64) if k64 else None
        fp64 = {"mlups": cells * args.fp64_steps * world / s64 / 1e6,
                "ms_per_step": s64 / args.fp64_steps * 1e3, "steps": args.fp64_steps,
                "kernel_ms_per_launch": k64 * 1e3 if k64 else None}
        rec = counters_record("fp64", w.thermal)
        if rec and k64:
            # FP64 is bound by the FP64 pipe: FLOPs and FP64 instructions per
            # cell from the ncu record, against the pipe's nominal rate
            flop = rec["fp64_flop_per_cell"]
            inst = rec["fp64_inst_per_cell"]
            fp64["roofline"] = {
                "bound": "alu", "unit": "TFLOP/s",
                "achieved": flop * cells / k64 / 1e12, "peak": FP64_PEAK_TFLOPS,
                "frac": flop * cells / k64 / 1e12 / FP64_PEAK_TFLOPS,
                "fp64_inst_frac": inst * cells / k64 / (FP64_PEAK_TFLOPS * 1e12 / 2),
                "flop_per_cell": flop, "fp64_inst_per_cell": inst,
                "source": f"ncu FP64 instruction counters of one step-kernel launch at {rec['n']}^3 "
                          f"(profiles/step_kernel_counters.json)",
                "peak_kind": "nominal: 152 SMs x 2 FP64 FMA lanes per cycle x 2 FLOP x 2.07 GHz "
                             "(no measured FP64 peak on this pool)"}
        del d64
        torch.cuda.empty_cache()

    # ---------------- adjoint cost: gradient of the droplet-capture objective
    # (64^3, 2000 steps, checkpoints every 100) vs the same forward steps
    adj = None
    if rank == 0 and not args.no_adjoint:
        c5 = W.config5(n=64)

        def c5_domain():
            dd = lbm.Domain(c5.nx, c5.ny, c5.nz, "fp64", c5.thermal, c5.q_phase, device=dev)
            dd.set_params(c5.params)
            pt = c5.patches
            dd.set_heater_patches(pt.z, pt.sx, pt.sy, pt.x0, pt.y0, pt.intensity)
            dd.init_droplets(c5.droplets)
            return dd

        dd = c5_domain()
        dd.step(3)
        dd.close()
        dd = c5_domain()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        dd.step(c5.steps)
        dd.diagnostics()            # synchronises; the J evaluation of a forward run
        t_fwd = time.perf_counter() - t0
        dd.close()
        dd = c5_domain()
        t0 = time.perf_counter()
        J5, g5 = dd.adjoint_run(c5.steps, 100, c5.target, normal_cap=30.0)
        t_adj = time.perf_counter() - t0
        dd.close()
        dd = c5_domain()
        t0 = time.perf_counter()
        _, g5x = dd.adjoint_run(c5.steps, 100, c5.target, normal_cap=0.0)
        t_adj_x = time.perf_counter() - t0
        dd.close()
        adj = {"workload": c5.name, "steps": c5.steps, "ckpt_every": 100, "normal_cap": 30.0,
               "forward_s": t_fwd, "adjoint_run_s": t_adj, "cost_ratio": t_adj / t_fwd,
               "exact_adjoint_run_s": t_adj_x, "exact_cost_ratio": t_adj_x / t_fwd,
               "what": "lbm_adjoint_run (forward with checkpoints + replay + adjoint steps) wall time "
                       "over the plain forward run of the same steps; FP64; normal cap 30 and exact (cap 0)",
               "J": J5, "grad_inf": float(np.abs(g5).max()), "exact_grad_inf": float(np.abs(g5x).max())}

    # ---------------- stated error: FP32 and FP16 storage vs FP64 on a bulk-kernel
    # lattice of the same workload (128^3, 8 droplets, 200 steps); the FP64
    # bulk kernel equals the oracle to <= 1e-11 over 200 steps (parity tests)
    err = None
    if rank == 0 and not args.kernel_only:
        ce = W.config4(args.thermal, "fp64", n=128, n_droplets=8)
        esteps = 200
        res = {}
        for prec in ("fp64", "fp32", "fp16"):
            dd = lbm.Domain(ce.nx, ce.ny, ce.nz, prec, ce.thermal, ce.q_phase, device=dev)
            dd.set_params(ce.params)
            dd.init_droplets(ce.droplets)
            kern = dd.kernel_info()["kernel"]
            dd.step(esteps)
            f = dd.fields(dtype="f64")
            res[prec] = ({k: v.detach().cpu().numpy() for k, v in f.items()}, dd.diagnostics(), kern)
            dd.close()
        b, db, kb = res["fp64"]
        err = {"workload": f"{ce.name}, {esteps} steps, {ce.thermal}; reduced storage vs the FP64 "
                           f"GPU run (FP64 bulk kernel = oracle to <= 1e-11 over 200 steps)",
               "kernel_fp64": kb}
        for prec in ("fp32", "fp16"):
            a, da, ka = res[prec]
            du = a["u"] - b["u"]
            err[prec] = {"kernel": ka,
                         "phi_linf": float(np.abs(a["phi"] - b["phi"]).max()),
                         "u_l2_rel": float(math.sqrt((du ** 2).sum() / (b["u"] ** 2).sum())),
                         "T_linf": float(np.abs(a["T"] - b["T"]).max()),
                         "mass_rel": abs(da["mass"] - db["mass"]) / db["mass"],
                         "centroid_abs": max(abs(x - y) for x, y in zip(da["centroid"], db["centroid"]))}

    # ---------------- sweep: every thermal option x storage precision at the
    # headline lattice, step kernel timed alone (CUDA events around each launch)
    sweep = None
    if not args.no_sweep:
        sweep = []
        peak_s, _ = peaks()
        for prec in ("fp32", "fp16", "fp64"):
            for th in ("D3Q7", "D3Q15", "D3Q19", "D3Q27", "RK2", "RK4"):
                ws = W.config4(th, prec, n=args.n)
                nst = args.sweep_steps if prec != "fp64" else 2
                ds = lbm.Domain(ws.nx, ws.ny, ws.nz, prec, ws.thermal, ws.q_phase, device=dev)
                ds.set_params(ws.params)
                ds.init_droplets(ws.droplets)
                ssecs, _, kser = timed_steps(ds, nst, 3)
                ssecs = reduce_max(ssecs)
                kser = reduce_max(kser) if kser else None
                bpc_s = bytes_per_cell(prec, th, ws.q_phase)
                bpk = step_kernel_bytes_per_cell(prec, th, ws.q_phase)
                ach = bpk * ws.cells / kser / 1e9 if kser else None
                step_gbs = bpc_s * ws.cells * nst / ssecs / 1e9
                sweep.append({"precision": prec, "thermal": th, "kernel": ds.kernel_info()["kernel"],
                              "mlups": job_mlups(ws.cells, nst, world, ssecs),
                              "step_ms": ssecs / nst * 1e3,
                              "kernel_ms": kser * 1e3 if kser else None,
                              "bytes_per_cell": bpc_s, "step_kernel_bytes_per_cell": bpk,
                              "achieved_gbs": ach, "frac": ach / peak_s if ach else None,
                              "step_frac": step_gbs / peak_s, "steps": nst})
                ds.close()
                del ds
                torch.cuda.empty_cache()

    # ---------------- in-place (AA) layout: the headline workload, then a
    # lattice the two-grid layout cannot hold on this GPU
    aa = None
    if not args.no_aa:
        aa = []
        peak_a, _ = peaks()
        free_b, total_b = torch.cuda.mem_get_info(dev)
        for n_aa, nst in ((args.n, args.sweep_steps), (args.aa_large_n, 3)):
            if n_aa <= 0:
                continue
            wa = W.config4(args.thermal, args.precision, n=n_aa)
            two = lbm.lib().lbm_workspace_bytes_layout(n_aa, n_aa, n_aa, lbm.PRECISION[args.precision],
                                                       lbm.THERMAL[wa.thermal], wa.q_phase, 0)
            one = lbm.lib().lbm_workspace_bytes_layout(n_aa, n_aa, n_aa, lbm.PRECISION[args.precision],
                                                       lbm.THERMAL[wa.thermal], wa.q_phase, 1)
            rec = {"n": n_aa, "workspace_gb": one / 1e9, "two_grid_workspace_gb": two / 1e9,
                   "gpu_memory_gb": total_b / 1e9, "two_grid_fits": two < free_b}
            if one >= free_b:
                rec["skipped"] = "does not fit"
                aa.append(rec)
                continue
            da = lbm.Domain(wa.nx, wa.ny, wa.nz, args.precision, wa.thermal, wa.q_phase, device=dev, layout="aa")
            da.set_params(wa.params)
            da.init_droplets(wa.droplets)
            asecs, _, aker = timed_steps(da, nst, 3)
            asecs = reduce_max(asecs)
            aker = reduce_max(aker) if aker else None
            bpa = step_kernel_bytes_per_cell(args.precision, wa.thermal, wa.q_phase)
            rec.update({"kernel": da.kernel_info()["kernel"], "steps": nst,
                        "mlups": job_mlups(wa.cells, nst, world, asecs), "step_ms": asecs / nst * 1e3,
                        "kernels_ms": aker * 1e3 if aker else None,
                        "frac": bpa * wa.cells / aker / 1e9 / peak_a if aker else None,
                        "what": "(phi, T) pass + in-place step (+ ghost refresh before and fold after "
                                "the steps from even levels), kernels_ms per step; frac from the "
                                "algorithmic bytes of the two-grid step"})
            da.close()
            del da
            torch.cuda.empty_cache()
            aa.append(rec)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    peak, peak_kind = peaks()
    bpc = step_kernel_bytes_per_cell(args.precision, w.thermal, w.q_phase)
    # the dominant kernel's own average launch time (CUDA events around each
    # step-kernel launch on the domain's stream, inside the timed region)
    achieved = bpc * cells / kernel_secs / 1e9 if (bpc and kernel_secs) else None
    tr = traffic_per_cell(args.precision, w.thermal) if args.layout == "two_grid" else None
    tpc, tr_n = tr if tr else (None, None)
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else ("f64" if args.precision == "fp64" else "f16-store/f32"),
        "data": "synthetic (seeded droplets, workloads.config4)",
        "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "precision": args.precision,
                   "layout": args.layout, "kernel": kinfo,
                   "thermal": w.thermal, "q_phase": w.q_phase, "hydro": "D3Q27 central moment",
                   "l2": "state 52.6 GB >> 129 MB L2: no flush needed",
                   "parallelism": f"replicas x{world} (independent lattices, no collective)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                     "bytes_per_cell": bpc,
                     "kernel_ms_per_launch": kernel_secs * 1e3 if kernel_secs else None,
                     "step_ms": per_step * 1e3,
                     "traffic": tpc * cells if tpc else None,
                     "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one step-kernel "
                                        f"launch at {tr_n}^3 (profiles/step_kernel_counters.json): "
                                        f"{tpc:.1f} B/cell, scaled by the cell count"
                                        if tpc else "no ncu record for the current kernel sources"),
                     "kernel": KERNEL_NAMES.get(kinfo["kernel"], kinfo["kernel"])},
        "cpu_baseline": ({"value": cpu["mlups"], "unit": "MLUPS", "cores": 1, "kind": "oracle",
                          "sample": f"{cpu['name']}: {cpu['steps']} FP64 numpy oracle steps in "
                                    f"{cpu['seconds']:.1f} s, single thread",
                          "cpu_model": cpu_model(),
                          "all_cores": ({"value": cpu_all["mlups"], "unit": "MLUPS", "cores": cpu_all["procs"],
                                         "sample": f"{cpu_all['procs']} single-threaded oracle processes, each "
                                                   f"on its own copy of {cpu_all['name']}, at the same time: "
                                                   f"{cpu_all['steps']} steps in {cpu_all['seconds']:.1f} s"}
                                        if cpu_all and "mlups" in cpu_all else cpu_all)}
                         if cpu and "mlups" in cpu else cpu),
        "e2e": e2e,
        "gpu_launches": timed_launches,
        "adjoint": adj,
        "fp64": fp64,
        "fp32_vs_fp64": fp64 and {"speedup": mlups / fp64["mlups"]},
        "error_vs_fp64": err,
        "sweep": sweep,
        "aa_layout": aa,
        "final_diag": {"mass": diag_final["mass"], "level": diag_final["level"]},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
