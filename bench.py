#!/usr/bin/env python
"""Throughput benchmark of the implicit-smoothing hot path (forward + adjoint solve per mesh).

One step = assemble A = M(V) + tL(V), solve A U = M B, solve the adjoint A Lambda = U - T and
gather dl/dV, for one mesh with 3 right-hand-side columns. The default workload is the 1024 x 1024
height-field grid (1,048,576 vertices, 2,093,058 faces, t = h^2, B ~ U[-1,1]) in FP64, solved to a
relative residual of 1e-10. With torchrun (N > 1) every rank solves its own mesh (weak scaling,
no collective on the data path); the timed region is bracketed by barriers and the slowest rank
sets the time.

Printed: one JSON line on rank 0 (see the keys below). `--impl reference` times the CPU oracle
(plain FP64 C, single thread) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint Laplacian solves/s, % HBM roofline, p50/p99 latency vs plain"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid1024",
                    help="grid1024 (default), ico3, grid4096x2048, or any gridS / gridXxY of the same family")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed", "mixed32"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--launch", default="graph", choices=["graph", "host"],
                    help="graph: device-side solver loop (default); host: one launch per kernel")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel timing pass")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other workloads (mixed grid, largest mesh, 256-mesh batch, serving)")
    ap.add_argument("--serve-requests", type=int, default=600,
                    help="requests in the bounded sample of the serving stream")
    ap.add_argument("--variants", default="small,mixed,largest,batch,fairing,eigs,rgd,serve",
                    help="comma list of the extra workloads to run")
    ap.add_argument("--fma-peak", action="store_true",
                    help="measure the FP64 and FP32 FMA throughput of this GPU (ig_measure_fma_peak) with the SM "
                         "clock sampled during it; prints one JSON line")
    ap.add_argument("--oracle-timings", action="store_true",
                    help="time the CPU oracle alone (single thread) on the ico3 and grid1024 configurations in "
                         "full and on the 4096x2048 grid and the 256-mesh batch once each; prints one JSON line")
    return ap.parse_args()


def make_problem(name, seed):
    from paper_2602_12105_gb300 import meshgen as mg
    if name == "grid1024":
        return mg.config_grid1024(seed)
    if name == "grid4096x2048":
        return mg.config_grid4096x2048(seed)
    if name == "ico3":
        return mg.config_ico3(seed)
    m = re.fullmatch(r"grid(\d+)(?:x(\d+))?", name)
    if not m:
        raise SystemExit(f"unknown workload {name}")
    sx = int(m.group(1))
    sy = int(m.group(2)) if m.group(2) else sx
    return mg.config_grid(sx, sy, seed)


def workload_desc(p, precision, tol):
    return (f"{p.name}: {p.n} vertices, {p.m} faces, k={p.B.shape[1]} RHS, t={p.t:.3e}, "
            f"{precision}, forward + adjoint to relative residual {tol:g}, dl/dV gathered")


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    _count = 0

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        ClockSampler._count += 1
        self.path = os.path.join("/tmp", f"ig_clocks_{os.getpid()}_{ClockSampler._count}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": float(np.median(power)) if power else None}


# ------------------------------------------------------------------------------- roofline
def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_12105_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


def measured_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary (profiles/traffic.txt), or None when
    the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
            return float(parts[3]) if parts[2] == cur else None
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def algorithmic(kernel, n, m, nnz, k, prec, idx32=4):
    """(flops, bytes) one launch of `kernel` must do / move (vectors [k][n], p and z rows padded to
    kp). FP64 path (pcg_*): two kernels per iteration. The SpMV gathers z = D^-1 r, forms
    p = z + beta p and q = A z + beta q (the recurrence q = A p) and the sum p.q; the update writes
    x, r and z. Mixed path (pcg32_*): 4-byte values and vectors, three kernels per iteration (SpMV
    q = A p, update, p-update reading D^-1 and r), and the SpMV reads idx32-byte column indices
    (2 where every slice of 32 rows keeps its columns as 16-bit offsets, as on the grid
    workloads)."""
    kp = 4 if k == 3 else k
    if kernel.startswith("pcg32_"):
        sv, si = 4, idx32
        kernel = kernel[len("pcg32_"):]
        if kernel == "spmv":
            return (float(2 * k * nnz + 2 * k * n),
                    float(nnz * (sv + si) + 4 * (n + 1) + sv * kp * n + sv * k * n))
        if kernel == "update":
            return float(11 * k * n), float(sv * (n + 3 * k * n + kp * n) + 2 * sv * k * n)
        if kernel == "pupdate":
            return float(3 * k * n), float(sv * (n + k * n + kp * n) + sv * kp * n)
        return None, None
    sv = 8
    if kernel == "pcg_spmv":
        flops = 2 * k * nnz + 6 * k * n
        byts = nnz * (sv + 4) + 4 * (n + 1) + sv * kp * n + 2 * sv * kp * n + 2 * sv * k * n
    elif kernel == "pcg_update":
        flops = 9 * k * n
        byts = sv * (n + kp * n + 3 * k * n) + sv * (2 * k * n + kp * n)
    elif kernel == "assemble_face":
        flops = 60 * m
        byts = 12 * m + 24 * n + 32 * m
    elif kernel == "assemble_rows":
        # incidence offsets and entries (8 B per corner), the per-face weights, row offsets and
        # diagonal slots; A (and its FP32 copy in mixed precision), M and 1/A_ii written
        flops = 0
        byts = 4 * n + 24 * m + 32 * m + 8 * n + 4 * n + 8 * nnz + 16 * n + (4 * nnz + 4 * n if prec == "mixed" else 0)
    elif kernel == "vjp_vertex":
        # Lambda, B and U per vertex; <Lambda_v, B_v - U_v> written
        flops = 4 * k * n
        byts = 3 * 8 * k * n + 8 * n
    elif kernel == "vjp_face":
        # faces, V, U and Lambda at the vertices (each once from DRAM), the per-vertex weights;
        # the per-corner gradients written
        flops = 300 * m
        byts = 12 * m + 24 * n + 2 * 8 * k * n + 8 * n + 72 * m
    elif kernel == "vjp_gather":
        # incidence offsets and entries, the per-corner gradients (24 B each), M; gV written
        flops = 0
        byts = 4 * n + 24 * m + 72 * m + 8 * n + 24 * n
    # FP32 face geometry: the split vertex passes, the FP32 face kernels and the FP32 gathers
    elif kernel == "assemble_split32":
        flops = 0
        byts = 24 * n + 32 * n
    elif kernel == "assemble_face32":
        flops = 60 * m
        byts = 12 * m + 32 * n + 16 * m
    elif kernel == "assemble_rows32":
        flops = 0
        byts = 4 * n + 24 * m + 16 * m + 8 * n + 4 * n + 4 * nnz + 8 * n + 4 * n
    elif kernel == "vjp_split32":
        flops = 0
        byts = 3 * 8 * k * n + 32 * n + 32 * n + 4 * n
    elif kernel == "vjp_face32":
        flops = 330 * m
        byts = 12 * m + 3 * 32 * n + 4 * n + 48 * m
    elif kernel == "vjp_gather32":
        flops = 0
        byts = 4 * n + 24 * m + 48 * m + 24 * n
    else:
        return None, None
    return float(flops), float(byts)


# ------------------------------------------------------------------------------- ranks
def max_over_ranks(x, world, device=None):
    """The largest value of x over all ranks (the slowest rank sets a timed region); x itself on
    one rank. Uses the process group of torch.distributed (NCCL on GPUs, gloo in the CPU tests)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, steps_per_rank, ms):
    """Whole-job throughput: every rank ran `steps_per_rank` units of its own work (weak scaling)
    inside a region of `ms` milliseconds (the max over ranks)."""
    return world * steps_per_rank / (ms / 1000.0)


def rank_seed(rank):
    """Each rank solves its own seeded mesh of the same workload family."""
    return rank


def shard(items, rank, world):
    """The independent units (meshes, requests) rank `rank` takes: every world-th one."""
    return list(items)[rank::world]


# ------------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2602_12105_gb300 import _native, api

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    precision = args.precision or "fp64"
    p = make_problem(args.workload, seed=rank_seed(rank))
    k = p.B.shape[1]
    mesh = api.Mesh(torch.from_numpy(p.F).to(dev), p.n)
    V = torch.from_numpy(p.V).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    T = torch.from_numpy(p.T).to(dev)
    U = torch.empty_like(B)
    opts = api.make_opts(rel_tol=args.tol, launch=args.launch)
    stream = torch.cuda.current_stream(dev)

    def step():
        mesh.assemble(V, p.t, precision)
        mesh.solve(B, opts=opts, out=U)
        gV, _, _ = mesh.adjoint(V, B, p.b_is_V, U, U - T, opts=opts)
        return gV

    # correctness of this very configuration (outside the timed region)
    mesh.assemble(V, p.t, precision)
    U0, finfo = mesh.solve(B, opts=opts, info=True)
    gV0, _, _, ainfo = mesh.adjoint(V, B, p.b_is_V, U0, U0 - T, opts=opts, info=True)
    if finfo["status"] != 0 or ainfo["status"] != 0:
        raise RuntimeError(f"solve failed: {finfo} {ainfo}")

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)])
    total_ms = float(evs[0].elapsed_time(evs[-1]))
    total_ms = max_over_ranks(total_ms, world, dev)
    value = aggregate_rate(world, args.steps, total_ms)

    # per-kernel device times (CUDA events around each launch, host-launched loop)
    prof = {}
    if not args.no_profile:
        _native.profile_enable(True)
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        prof = _native.profile_read()
        _native.profile_enable(False)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hV = torch.from_numpy(p.V).pin_memory()
        hB = torch.from_numpy(p.B).pin_memory()
        hT = torch.from_numpy(p.T).pin_memory()
        hG = torch.empty((p.n, 3), dtype=torch.float64).pin_memory()
        dV, dB, dT = torch.empty_like(V), torch.empty_like(B), torch.empty_like(T)

        def e2e_step():
            dV.copy_(hV, non_blocking=True)
            dB.copy_(hB, non_blocking=True)
            dT.copy_(hT, non_blocking=True)
            mesh.assemble(dV, p.t, precision)
            mesh.solve(dB, opts=opts, out=U)
            gV, _, _ = mesh.adjoint(dV, dB, p.b_is_V, U, U - dT, opts=opts)
            hG.copy_(gV, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = float(e0.elapsed_time(e1))
        ems = max_over_ranks(ems, world, dev)
        e2e = {"value": aggregate_rate(world, args.e2e_steps, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(hV.nbytes + hB.nbytes + hT.nbytes), "d2h_bytes_per_step": int(hG.nbytes)}

    if rank != 0:
        return None

    # roofline of the dominant kernel, against the ALU peaks measured on this GPU now
    alu = measure_alu_peaks(_native, local_rank, stream.cuda_stream)
    its_f, its_a = finfo["iterations"], ainfo["iterations"]
    rl_all, roofline = kernel_roofline(prof, p.n, p.m, mesh.nnz, k, precision, clocks, args.workload, alu,
                                       idx32=2 if args.workload.startswith("grid") else 4)
    step_roof = step_hbm(prof, 3, total_ms / args.steps, p.n, p.m, mesh.nnz, k, precision,
                         idx32=2 if args.workload.startswith("grid") else 4) if prof else None

    # the CPU oracle on the same workload (bounded sample)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(p, args)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded meshgen: smoothed height-field grid, B ~ U[-1,1])",
        "config": {"workload": workload_desc(p, precision, args.tol), "precision": precision,
                   "mesh": p.name, "n": p.n, "m": p.m, "nnz": mesh.nnz, "k": k,
                   "l2": f"inputs larger than L2: {mesh.device_bytes / 1e6:.0f} MB resident per mesh > 129 MB L2",
                   "iterations": {"forward": its_f, "adjoint": its_a},
                   "true_rel_residual": {"forward": max(finfo["true_rel_residual"]),
                                         "adjoint": max(ainfo["true_rel_residual"])},
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "latency_ms": {"p50": round(float(np.percentile(step_ms, 50)), 4),
                       "p99": round(float(np.percentile(step_ms, 99)), 4)},
        "clocks": clocks,
        "roofline": roofline,
        "alu_peaks": alu,
        "step_roofline": step_roof,
        "kernels": rl_all,
        "loop_iteration": loop_iteration(api, dev, mesh, p, alu, (clocks or {}).get("sm_mhz"), prof)
        if precision == "fp64" else None,
        "gpu_launches": gpu_launches(prof, args.steps, its_f, its_a, args.launch),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if world == 1 and not args.no_variants:
        out["variants"] = run_variants(args, p, U0, gV0, dev, alu)
    return out


def gpu_launches(prof, steps, its_f, its_a, launch):
    """Kernel launches of the timed region, counted from the profile pass (one host-launched
    step, every launch bracketed by events): the kernels outside the solver loops as they were
    counted, the loop bodies as 2 kernels per iteration of the two FP64 solves, in passes of two
    iterations (a solve with an odd count ends with one pass whose second half does no work)."""
    def in_graph(its):  # the graph's body holds two iterations (four launches) per pass
        return 4 * ((its + 1) // 2)
    if not prof:
        return int(steps * (2 + (2 + in_graph(its_f)) + (2 + in_graph(its_a)) + 2))
    loop = {"pcg_spmv", "pcg_update"}
    outside = sum(c for name, (c, _) in prof.items() if name not in loop)
    per_step = outside / 3.0 + in_graph(its_f) + in_graph(its_a) if launch == "graph" else \
        sum(c for c, _ in prof.values()) / 3.0
    return int(round(steps * per_step))


def measure_alu_peaks(_native, gpu_index, stream_ptr=None):
    """FP64 and FP32 fused multiply-add throughput of this GPU, measured by the library's
    ig_measure_fma_peak (8 independent FMA chains per thread, one wave of resident CTAs on every
    SM; best of 3 runs of about 0.3 s each), with the SM clock sampled while they run."""
    import torch
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.2)
    r64 = max(_native.measure_fma_peak(True, steps=80000, stream=stream_ptr)[0] for _ in range(3))
    r32 = max(_native.measure_fma_peak(False, steps=4000000, stream=stream_ptr)[0] for _ in range(3))
    clocks = sampler.stop()
    sms = torch.cuda.get_device_properties(gpu_index).multi_processor_count
    mhz = clocks.get("sm_mhz")
    out = {"fp64_tflops": round(r64 / 1e12, 4), "fp32_tflops": round(r32 / 1e12, 3), "sms": sms,
           "sm_mhz": mhz, "clocks": clocks,
           "how": "ig_measure_fma_peak: 8 independent FMA chains per thread, one wave of resident 256-thread CTAs on "
                  "every SM, CUDA events, best of 3"}
    if mhz:
        out["fp64_fma_per_clk_per_sm"] = round(r64 / 2 / sms / (mhz * 1e6), 3)
        out["fp32_fma_per_clk_per_sm"] = round(r32 / 2 / sms / (mhz * 1e6), 2)
    return out


def alu_peak_at(alu, key, sm_mhz):
    """A measured ALU peak (TFLOP/s) scaled from the SM clock it was measured at to sm_mhz (the
    median clock of the timed region): both are instruction rates proportional to the clock."""
    v = alu[key]
    if sm_mhz and alu.get("sm_mhz"):
        v = v * sm_mhz / alu["sm_mhz"]
    return v


def loop_iteration(api, dev, mesh, p, alu, sm_mhz, prof, n1=10, n2=60, reps=5):
    """Time of one FP64 Jacobi-PCG iteration as the solver runs it: inside the CUDA graph's
    conditional WHILE loop, where no event can sit between kernels. Solves of the assembled mesh
    with an unreachable tolerance run exactly n1 and n2 iterations (status NOT_CONVERGED); the
    median time difference over reps, divided by n2 - n1, is the iteration. It is compared with the
    FP64 floor of the iteration (the method's FP64 flops at the measured FP64 FMA peak, scaled to
    the timed region's SM clock) and with the per-kernel event timing of the host-launched loop,
    which adds a launch gap before each kernel."""
    import torch
    B = torch.from_numpy(p.B).to(dev)
    stream = torch.cuda.current_stream(dev)
    times = {n1: [], n2: []}
    for _ in range(reps):
        for it in (n1, n2):
            opts = api.make_opts(rel_tol=1e-300, max_iter=it, launch="graph")
            mesh.solve(B, opts=opts, info=True)  # warm (graph built, caches as in a solve)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = mesh.solve(B, opts=opts, info=True)
            e1.record(stream)
            torch.cuda.synchronize()
            assert info["iterations"] == it, info
            times[it].append(float(e0.elapsed_time(e1)))
    us = (float(np.median(times[n2])) - float(np.median(times[n1]))) * 1000.0 / (n2 - n1)
    k = p.B.shape[1]
    f_spmv, _ = algorithmic("pcg_spmv", p.n, p.m, mesh.nnz, k, "fp64")
    f_upd, _ = algorithmic("pcg_update", p.n, p.m, mesh.nnz, k, "fp64")
    peak = alu_peak_at(alu, "fp64_tflops", sm_mhz)
    floor_us = (f_spmv + f_upd) / (peak * 1e12) * 1e6
    host = None
    if prof and "pcg_spmv" in prof and "pcg_update" in prof:
        host = round(sum(prof[name][1] / prof[name][0] for name in ("pcg_spmv", "pcg_update")) * 1000.0, 2)
    return {"us_in_graph": round(us, 2), "fp64_floor_us": round(floor_us, 2),
            "frac_of_fp64_peak": round(floor_us / us, 4) if us > 0 else None,
            "us_host_launch_kernel_events": host,
            "method": f"graph-launched solves of exactly {n1} and {n2} iterations (unreachable tolerance), "
                      f"median of {reps}; floor = the method's FP64 flops per iteration "
                      f"({(f_spmv + f_upd) / 1e6:.1f} MFLOP) at the measured FP64 FMA peak"}


def kernel_roofline(prof, n, m, nnz, k, precision, clocks, workload, alu, idx32=4):
    """Per-kernel achieved rates from the profile pass ({name: (launches, total ms)}) and the
    roofline object of the kernel with the largest total time. FP64 kernels are held against the
    measured FP64 FMA peak, FP32 ones against the measured HBM copy bandwidth and the measured FP32
    FMA peak (alu: measure_alu_peaks, scaled to the timed region's median SM clock); the bound is
    whichever fraction is higher."""
    hbm_peak, peak_kind = peaks()
    sm_mhz = (clocks or {}).get("sm_mhz")
    fp64_peak_tflops = alu_peak_at(alu, "fp64_tflops", sm_mhz)
    fp32_peak_tflops = alu_peak_at(alu, "fp32_tflops", sm_mhz)
    rl_all = {}
    for name, (cnt, ms) in prof.items():
        is64 = (name.startswith(("assemble", "vjp")) and not name.endswith("32")) or \
            (name.startswith("pcg_") and precision == "fp64")
        fl, by = algorithmic(name, n, m, nnz, k, precision if name == "assemble_rows" else ("fp64" if is64 else "fp32"),
                             idx32)
        if fl is None or cnt == 0 or ms <= 0:
            continue
        avg_s = ms / cnt / 1000.0
        alu_peak = fp64_peak_tflops if is64 else fp32_peak_tflops
        rl_all[name] = {"avg_us": avg_s * 1e6, "launches": cnt, "total_ms": ms,
                        "gbs": by / avg_s / 1e9, "hbm_frac": by / avg_s / 1e9 / hbm_peak,
                        "tflops": fl / avg_s / 1e12, "alu_frac": fl / avg_s / 1e12 / alu_peak,
                        "alu_peak": alu_peak, "bytes": by}
    if not rl_all:
        return {}, None
    dom = max(rl_all.items(), key=lambda kv: kv[1]["total_ms"])[0]
    d = rl_all[dom]
    if d["alu_frac"] >= d["hbm_frac"]:
        roofline = {"bound": "alu", "achieved": round(d["tflops"], 4), "peak": round(d["alu_peak"], 4),
                    "unit": "TFLOP/s", "frac": round(d["alu_frac"], 4), "traffic": measured_traffic(dom, workload),
                    "kernel": dom,
                    "peak_source": f"measured in this run: ig_measure_fma_peak {alu['fp64_tflops']} TFLOP/s FP64 "
                                   f"({alu['fp32_tflops']} FP32) at a median {alu.get('sm_mhz')} MHz, scaled to the "
                                   f"timed region's median {sm_mhz} MHz",
                    "hbm_gbs": round(d["gbs"], 1), "hbm_frac_of_measured": round(d["hbm_frac"], 4),
                    "algorithmic_bytes_per_launch": int(d["bytes"])}
    else:
        roofline = {"bound": "hbm", "achieved": round(d["gbs"], 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(d["hbm_frac"], 4), "traffic": measured_traffic(dom, workload),
                    "kernel": dom, "peak_source": f"{peak_kind} (hbm_gbs copy bandwidth)",
                    "frac_of_nominal_7900_gbs": round(d["gbs"] / 7900.0, 4),
                    "algorithmic_bytes_per_launch": int(d["bytes"])}
    table = {kname: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in kv.items()
                     if kk not in ("alu_peak", "bytes")} for kname, kv in rl_all.items()}
    return table, roofline


def step_hbm(prof, nsteps, ms_per_step, n, m, nnz, k, precision, idx32=4):
    """The whole step against the HBM roofline: the algorithmic bytes of every profiled kernel
    that has a byte model (the solver loop, assembly and the VJP; the small init, finalize,
    gather and residual kernels are left out, so the figure is a lower bound), per step, divided
    by the step time of the timed region."""
    hbm_peak, peak_kind = peaks()
    total, counted = 0.0, []
    for name, (cnt, _) in prof.items():
        is64 = (name.startswith(("assemble", "vjp")) and not name.endswith("32")) or \
            (name.startswith("pcg_") and precision == "fp64")
        _, by = algorithmic(name, n, m, nnz, k, precision if name == "assemble_rows" else ("fp64" if is64 else "fp32"),
                            idx32)
        if by is None or cnt == 0:
            continue
        total += by * cnt / nsteps
        counted.append(name)
    if total == 0.0 or ms_per_step <= 0:
        return None
    gbs = total / (ms_per_step / 1000.0) / 1e9
    return {"bytes_per_step": int(total), "achieved_gbs": round(gbs, 1), "peak": hbm_peak,
            "peak_source": f"{peak_kind} (hbm_gbs copy bandwidth)", "frac": round(gbs / hbm_peak, 4),
            "kernels_counted": sorted(counted)}


# ------------------------------------------------------------------------------- other workloads
def _rel(a, b):
    import torch
    den = float(torch.linalg.vector_norm(b))
    return float(torch.linalg.vector_norm(a - b)) / (den if den > 0 else 1.0)


def _relmax(a, b):
    """Largest elementwise error of a against b, relative to max |b|."""
    import torch
    den = float(b.abs().max())
    return float((a - b).abs().max()) / (den if den > 0 else 1.0)


def _dev_problem(p, dev):
    import torch
    V = torch.from_numpy(np.ascontiguousarray(p.V)).to(dev)
    B = V if p.b_is_V else torch.from_numpy(np.ascontiguousarray(p.B)).to(dev)
    T = torch.from_numpy(np.ascontiguousarray(p.T)).to(dev)
    return V, B, T


def single_mesh(api, _native, dev, p, precision, tol, steps, warmup, launch="graph", profile=True, mesh=None):
    """Forward + adjoint of one mesh, timed over `steps` (CUDA events on the launching stream).
    Returns timings, solver info, the per-kernel profile and the results of the last step."""
    import torch
    stream = torch.cuda.current_stream(dev)
    if mesh is None:
        mesh = api.Mesh(torch.from_numpy(p.F).to(dev), p.n)
    V, B, T = _dev_problem(p, dev)
    U = torch.empty((p.n, B.shape[1]), dtype=torch.float64, device=dev)
    opts = api.make_opts(rel_tol=tol, launch=launch)

    def step():
        mesh.assemble(V, p.t, precision)
        mesh.solve(B, opts=opts, out=U)
        gV, _, _ = mesh.adjoint(V, B, p.b_is_V, U, U - T, opts=opts)
        return gV

    mesh.assemble(V, p.t, precision)
    U0, finfo = mesh.solve(B, opts=opts, info=True)
    gV0, _, _, ainfo = mesh.adjoint(V, B, p.b_is_V, U0, U0 - T, opts=opts, info=True)
    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = float(e0.elapsed_time(e1)) / steps
    prof = {}
    if profile:
        _native.profile_enable(True)
        step()
        torch.cuda.synchronize()
        prof = _native.profile_read()
        _native.profile_enable(False)
    return {"ms_per_step": ms, "solves_per_s": 1000.0 / ms, "finfo": finfo, "ainfo": ainfo, "U": U0, "gV": gV0,
            "prof": prof, "mesh": mesh}


def variant_mixed_grid(api, _native, dev, p, tol, steps, fp64_U, fp64_gV, clocks, alu):
    """The headline grid in mixed precision (FP32 PCG inside FP64 refinement)."""
    r = single_mesh(api, _native, dev, p, "mixed", tol, steps, 3)
    table, roof = kernel_roofline(r["prof"], p.n, p.m, r["mesh"].nnz, p.B.shape[1], "mixed", clocks, p.name + "_mixed",
                                  alu, idx32=2)
    out = {"workload": f"{p.name} mixed: FP32 Jacobi-PCG (FP32 CSR values) inside FP64 residual refinement to {tol:g}",
           "value": round(r["solves_per_s"], 3), "unit": UNIT, "ms_per_step": round(r["ms_per_step"], 4),
           "steps": steps, "iterations": {"forward": r["finfo"]["iterations"], "adjoint": r["ainfo"]["iterations"]},
           "refinements": {"forward": r["finfo"]["refinements"], "adjoint": r["ainfo"]["refinements"]},
           "true_rel_residual": {"forward": max(r["finfo"]["true_rel_residual"]),
                                 "adjoint": max(r["ainfo"]["true_rel_residual"])},
           "rel_err_vs_fp64_gpu": {"U": _rel(r["U"], fp64_U), "gV": _rel(r["gV"], fp64_gV)},
           "roofline": roof,
           "step_roofline": step_hbm(r["prof"], 1, r["ms_per_step"], p.n, p.m, r["mesh"].nnz, p.B.shape[1], "mixed",
                                     idx32=2),
           "kernels": table}
    r["mesh"].close()
    return out


def variant_small(api, _native, dev, steps=300):
    """The small single mesh of the plain FP64 configuration: the noisy level-3 icosphere (642
    vertices), B = V, loss 1/2 |U - clean sphere|^2, forward + adjoint to 1e-12; a mesh of three
    FP64 tiles, whose solves loop inside one thread-block cluster."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_ico3(0)
    r = single_mesh(api, _native, dev, p, "fp64", 1e-12, steps, 10, profile=False)
    r["mesh"].close()
    return {"workload": f"{p.name}: {p.n} vertices, {p.m} faces, B = V, FP64, forward + adjoint to 1e-12",
            "unit": UNIT, "value": round(r["solves_per_s"], 2), "ms_per_step": round(r["ms_per_step"], 4),
            "steps": steps, "iterations": {"forward": r["finfo"]["iterations"], "adjoint": r["ainfo"]["iterations"]},
            "true_rel_residual": {"forward": max(r["finfo"]["true_rel_residual"]),
                                  "adjoint": max(r["ainfo"]["true_rel_residual"])}}


def variant_largest(api, _native, dev, tol, steps, clocks, alu):
    """The largest single mesh (4096 x 2048 grid, 8.4M vertices) in mixed precision, with its HBM
    roofline, and its error against the FP64 GPU path on the same mesh."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid4096x2048(0)
    r = single_mesh(api, _native, dev, p, "mixed", tol, steps, 3)
    mesh = r["mesh"]
    table, roof = kernel_roofline(r["prof"], p.n, p.m, mesh.nnz, p.B.shape[1], "mixed", clocks, "grid4096x2048",
                                  alu, idx32=2)
    r64 = single_mesh(api, _native, dev, p, "fp64", tol, 1, 0, profile=False, mesh=mesh)
    out = {"workload": f"{p.name}: {p.n} vertices, {p.m} faces, k=3, t=h^2, mixed precision to {tol:g}",
           "value": round(r["solves_per_s"], 3), "unit": UNIT, "ms_per_step": round(r["ms_per_step"], 4),
           "steps": steps, "fp64_gpu_ms_per_step": round(r64["ms_per_step"], 4),
           "iterations": {"forward": r["finfo"]["iterations"], "adjoint": r["ainfo"]["iterations"]},
           "refinements": {"forward": r["finfo"]["refinements"], "adjoint": r["ainfo"]["refinements"]},
           "true_rel_residual": {"forward": max(r["finfo"]["true_rel_residual"]),
                                 "adjoint": max(r["ainfo"]["true_rel_residual"])},
           "rel_err_vs_fp64_gpu": {"U": _rel(r["U"], r64["U"]), "gV": _rel(r["gV"], r64["gV"])},
           "resident_mb": round(mesh.device_bytes / 1e6, 1), "roofline": roof,
           "step_roofline": step_hbm(r["prof"], 1, r["ms_per_step"], p.n, p.m, mesh.nnz, p.B.shape[1], "mixed",
                                     idx32=2),
           "kernels": table}
    # the same mesh with FP32 face geometry (FP64 for slivers): the FP32 operator solved exactly
    r32 = single_mesh(api, _native, dev, p, "mixed32", tol, steps, 3, mesh=mesh)
    table32, roof32 = kernel_roofline(r32["prof"], p.n, p.m, mesh.nnz, p.B.shape[1], "mixed", clocks,
                                      "grid4096x2048_mixed32", alu, idx32=2)
    out["fp32_geometry"] = {
        "workload": f"{p.name}, mixed precision with FP32 face geometry (cotangents, areas and the per-face "
                    f"gradient in FP32; FP64 for faces with sin(theta_min) < 1e-2), FP32 operator solved to {tol:g}",
        "value": round(r32["solves_per_s"], 3), "unit": UNIT, "ms_per_step": round(r32["ms_per_step"], 4),
        "steps": steps,
        "iterations": {"forward": r32["finfo"]["iterations"], "adjoint": r32["ainfo"]["iterations"]},
        "true_rel_residual_own_operator": {"forward": max(r32["finfo"]["true_rel_residual"]),
                                           "adjoint": max(r32["ainfo"]["true_rel_residual"])},
        "rel_err_vs_fp64_gpu": {"U": _rel(r32["U"], r64["U"]), "gV": _rel(r32["gV"], r64["gV"]),
                                "U_max_elementwise": _relmax(r32["U"], r64["U"]),
                                "gV_max_elementwise": _relmax(r32["gV"], r64["gV"])},
        "roofline": roof32,
        "step_roofline": step_hbm(r32["prof"], 1, r32["ms_per_step"], p.n, p.m, mesh.nnz, p.B.shape[1], "mixed",
                                  idx32=2),
        "kernels": table32}
    mesh.close()
    return out


def variant_batch(api, _native, dev, tol, steps):
    """The differentiation batch (256 icospheres, levels 2..6, per-mesh t): forward + adjoint of
    all meshes in shared launches, FP64 and mixed, against the plain path that runs the same
    meshes one after another in FP64."""
    import torch
    from paper_2602_12105_gb300 import meshgen as mg
    probs = mg.config_batch(seed=0, count=256)
    stream = torch.cuda.current_stream(dev)
    meshes = [api.Mesh(torch.from_numpy(q.F).to(dev), q.n) for q in probs]
    Vs = [torch.from_numpy(q.V).to(dev) for q in probs]
    Ts = [torch.from_numpy(q.T).to(dev) for q in probs]
    ts = [q.t for q in probs]
    opts = api.make_opts(rel_tol=tol)
    batch = api.Batch(meshes)

    def bstep(prec, info=False):
        batch.assemble(Vs, ts, prec)
        if info:
            Us, fi = batch.solve(Vs, opts=opts, info=True)
            gVs, _, _, ai = batch.adjoint(Vs, None, True, Us, [U - T for U, T in zip(Us, Ts)], opts=opts, info=True)
            return Us, gVs, fi, ai
        Us = batch.solve(Vs, opts=opts)
        gVs, _, _ = batch.adjoint(Vs, None, True, Us, [U - T for U, T in zip(Us, Ts)], opts=opts)
        return Us, gVs

    def pstep():
        res = []
        for m, V, T, t in zip(meshes, Vs, Ts, ts):
            m.assemble(V, t, "fp64")
            U = m.solve(V, opts=opts)
            gV, _, _ = m.adjoint(V, V, True, U, U - T, opts=opts)
            res.append((U, gV))
        return res

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return float(e0.elapsed_time(e1)) / reps

    # accuracy: every mesh's mixed result against its FP64 result (both to the same tolerance)
    U64, g64, f64i, a64i = bstep("fp64", True)
    U32, g32, f32i, a32i = bstep("mixed", True)
    errU = max(_rel(a, b) for a, b in zip(U32, U64))
    errG = max(_rel(a, b) for a, b in zip(g32, g64))
    worst = int(np.argmax([_rel(a, b) for a, b in zip(g32, g64)]))

    def its(infos):
        it = np.array([i["iterations"] for i in infos])
        return {"max": int(it.max()), "mean": round(float(it.mean()), 1),
                "row_iterations": int(sum(q.n * i["iterations"] for q, i in zip(probs, infos)))}

    def prof_step(prec):
        _native.profile_enable(True)
        bstep(prec)
        torch.cuda.synchronize()
        pr = _native.profile_read()
        _native.profile_enable(False)
        return {k: {"launches": c, "total_ms": round(ms, 3)} for k, (c, ms) in sorted(pr.items(), key=lambda kv: -kv[1][1])}
    ms64 = timed(lambda: bstep("fp64"), steps)
    ms32 = timed(lambda: bstep("mixed"), steps)
    msp = timed(pstep, max(1, steps // 2))
    prof64, prof32 = prof_step("fp64"), prof_step("mixed")
    nb = len(probs)
    batch.close()
    for m in meshes:
        m.close()
    return {"workload": f"{nb} icospheres, levels 2..6 ({min(q.n for q in probs)}..{max(q.n for q in probs)} "
                        f"vertices, {sum(q.n for q in probs)} in all), radial N(0, 0.02), t log-uniform "
                        f"[1e-4, 1e-2], B = V, forward + adjoint to {tol:g}",
            "unit": UNIT, "steps": steps,
            "batched_mixed": round(nb * 1000.0 / ms32, 2), "batched_fp64": round(nb * 1000.0 / ms64, 2),
            "plain_fp64_one_at_a_time": round(nb * 1000.0 / msp, 2),
            "ms_per_batch": {"batched_mixed": round(ms32, 3), "batched_fp64": round(ms64, 3),
                             "plain_fp64": round(msp, 3)},
            "speedup_batched_mixed_vs_plain": round(msp / ms32, 3),
            "max_rel_err_mixed_vs_fp64": {"U": errU, "gV": errG},
            "worst_gV_mesh": {"name": probs[worst].name, "n": probs[worst].n, "t": probs[worst].t},
            "iterations": {"fp64": {"forward": its(f64i), "adjoint": its(a64i)},
                           "mixed": {"forward": its(f32i), "adjoint": its(a32i)}},
            "profile_one_step_host_launch": {"fp64": prof64, "mixed": prof32}}


def variant_fairing(api, _native, dev, steps, level=7):
    """The inverse-fairing loop of §7.1 (ig_fairing_step: forward solve, M-norm objective,
    adjoint gradient with the mass term, Sobolev-preconditioned step; three solves per step) on an
    icosphere with radial noise, V starting at the targets, in FP64 and mixed precision."""
    import torch
    from paper_2602_12105_gb300 import meshgen as mg
    Vc, F = mg.icosphere(level)
    T = mg.radial_perturb(Vc, 0.02, np.random.default_rng(35))
    t, eta = 2e-3, 1.0
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"ico{level} ({T.shape[0]} vertices, {F.shape[0]} faces), radial N(0, 0.02), t = {t:g}, "
                       f"eta = {eta:g}, solves to 1e-10; one step = assemble + 3 solves + VJP + update",
           "unit": "steps/s", "steps": steps}
    for prec in ("fp64", "mixed"):
        mesh = api.Mesh(torch.from_numpy(F).to(dev), T.shape[0])
        Td = torch.from_numpy(T).to(dev)
        fair = api.InverseFairing(mesh, Td, t, eta, precision=prec)
        V = Td.clone()
        loss0, infos = fair.step(V, info=True)
        for _ in range(2):
            fair.step(V, want_loss=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fair.step(V, want_loss=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = float(e0.elapsed_time(e1)) / steps
        loss_end = fair.step(V)
        out[prec] = {"value": round(1000.0 / ms, 3), "ms_per_step": round(ms, 4),
                     "iterations_first_step": [i["iterations"] for i in infos],
                     "loss_first": loss0, f"loss_after_{steps + 4}_steps": loss_end}
        mesh.close()
    return out


def variant_eigs(api, dev, steps, level=7):
    """The lowest four eigenpairs of L u = lambda M u on a slightly perturbed unit icosphere by the
    shift-invert subspace iteration of Eq. eigiter (§5, ig_eigs): each step is a 4-column
    smoothing solve (M + tL) Y = M U to 1e-10 and the M-orthonormalization of Y. The smooth unit
    sphere's lowest eigenvalues are 0 and 2 (three times), then 6, so with t = 0.5 a step
    contracts the error by about (1 + 2t) / (1 + 6t) = 1/2."""
    import torch
    from paper_2602_12105_gb300 import meshgen as mg
    Vc, F = mg.icosphere(level)
    V = mg.radial_perturb(Vc, 0.002, np.random.default_rng(41))
    t = 0.5
    mesh = api.Mesh(torch.from_numpy(F).to(dev), V.shape[0])
    mesh.assemble(torch.from_numpy(V).to(dev), t)
    U0 = torch.from_numpy(np.random.default_rng(42).uniform(-1, 1, (V.shape[0], 4))).to(dev)
    opts = api.make_opts(rel_tol=1e-10)
    mesh.eigs(U0, 2, opts=opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U, lam, info = mesh.eigs(U0, steps, opts=opts, info=True)
    dt = time.perf_counter() - t0
    M = mesh.mass()
    G = U.T @ (M[:, None] * U)
    orth = float((G - torch.eye(4, dtype=G.dtype, device=G.device)).abs().max())
    mesh.close()
    return {"workload": f"ico{level} ({V.shape[0]} vertices), radial N(0, 0.002), t = {t:g}, k = 4, "
                        f"{steps} subspace steps, each a 4-column solve to 1e-10 and an M-orthonormalization",
            "unit": "subspace steps/s", "value": round(steps / dt, 3), "ms_per_step": round(1000.0 * dt / steps, 4),
            "pcg_iterations_last_step": info["iterations"], "eigenvalues": [float(x) for x in lam],
            "max_abs_UtMU_minus_I": orth}


def variant_rgd(api, dev, rounds, side=257):
    """Regularized geodesic distances by the ADMM of formulation eq. edelstein (ig_rgd_admm) on a
    flat square grid with the source at a corner and beta = 0, where the answer is the Euclidean
    distance: rounds/s, the primal residual of the last round and the largest error against the
    Euclidean distance (relative to the largest distance)."""
    import torch
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(side, side, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.0
    mesh = api.Mesh(torch.from_numpy(p.F).to(dev), p.n)
    Vd = torch.from_numpy(V).to(dev)
    opts = api.make_opts(rel_tol=1e-10)
    mesh.rgd_admm(Vd, [0], 10.0, 0.0, 1.0, 2, opts=opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u, y, z, st = mesh.rgd_admm(Vd, [0], 10.0, 0.0, 1.0, rounds, opts=opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    d = np.linalg.norm(V - V[0], axis=1)
    err = float(np.abs(u.cpu().numpy() - d).max() / d.max())
    mesh.close()
    return {"workload": f"flat {side} x {side} grid ({p.n} vertices), source at a corner, beta = 0, rho = 10, "
                        f"beta_k = 1, {rounds} ADMM rounds, each a constrained Laplacian solve to 1e-10",
            "unit": "ADMM rounds/s", "value": round(rounds / dt, 3), "ms_per_round": round(1000.0 * dt / rounds, 3),
            "primal_residual_last_round": st["primal"], "dual_residual_last_round": st["dual"],
            "max_rel_err_vs_euclidean_distance": err}


def variant_rgd_adjoint(api, dev, side=33, max_rounds=3000, max_iter=1000):
    """The gradient through the geodesic ADMM (ig_rgd_admm_vjp) in the setting of the paper's
    terrain design, at its mesh size (2048 faces): a smoothed height field on a side x side grid,
    the source at a corner, the loss sum over the diagonal of (u_c - u_i)^2. The forward runs the
    rounds with residual balancing to 1e-5 (at most max_rounds); the backward solves the
    fixed-point adjoint by GMRES(50) to 1e-8 (at most max_iter Arnoldi steps, each one constrained
    Laplacian solve to 1e-10). Reports both wall times and the GMRES steps/s."""
    import torch
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(side, side, seed=0, t=1.0)
    mesh = api.Mesh(torch.from_numpy(p.F).to(dev), p.n)
    Vd = torch.from_numpy(p.V).to(dev)
    opts = api.make_opts(rel_tol=1e-10)
    beta, bk = 0.1, 1.0
    mesh.rgd_admm(Vd, [0], 2.0, beta, bk, 3, opts=opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u, y, z, st = mesh.rgd_admm(Vd, [0], 2.0, beta, bk, max_rounds, tol=1e-5, adapt_rho=True, opts=opts)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    diag = torch.arange(side, device=dev) * (side + 1)
    uc = float(u[diag].mean())
    gu = torch.zeros_like(u)
    gu[diag] = -2.0 * (uc - u[diag])
    mesh.rgd_admm_vjp(Vd, [0], y, z, st["rho"], beta, bk, gu, restart=50, max_iter=3, tol=1e-8, opts=opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gV, info = mesh.rgd_admm_vjp(Vd, [0], y, z, st["rho"], beta, bk, gu, restart=50, max_iter=max_iter, tol=1e-8,
                                 opts=opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    mesh.close()
    return {"workload": f"terrain: smoothed height field on a {side} x {side} grid ({p.n} vertices, {p.F.shape[0]} "
                        f"faces), source at a corner, beta = {beta}, beta_k = {bk}, loss sum over the diagonal of "
                        f"(u_c - u_i)^2; forward rounds with rho balancing to 1e-5, backward GMRES(50) to 1e-8 on "
                        f"the fixed-point adjoint",
            # a run whose forward or GMRES stopped short of its tolerance is reported as such, not as a
            # rate; the step rate stays beside it as a cost figure
            "unit": "GMRES steps/s",
            "value": round(info["iterations"] / dt, 3) if (info["converged"] and st["converged"]) else None,
            "status": ("converged" if (info["converged"] and st["converged"]) else
                       "not converged: " + "; ".join(
                           ([f"forward stopped at {st['rounds']} rounds with primal {st['primal']:.2e} and dual "
                             f"{st['dual']:.2e} against 1e-5"] if not st["converged"] else []) +
                           ([f"GMRES stopped at {info['iterations']} steps with relative residual "
                             f"{info['rel_resid']:.2e} against 1e-8"] if not info["converged"] else []))),
            "gmres_steps_per_s": round(info["iterations"] / dt, 3),
            "forward_ms_per_round": round(1000.0 * t_fwd / max(st["rounds"], 1), 3),
            "forward_ms": round(1000.0 * t_fwd, 2), "backward_ms": round(1000.0 * dt, 2),
            "gmres_steps": info["iterations"], "gmres_rel_resid": info["rel_resid"], "converged": info["converged"],
            "forward_rounds": st["rounds"], "forward_primal": st["primal"], "forward_dual": st["dual"],
            "final_rho": st["rho"], "sum_gV_rows_rel": float(gV.sum(0).abs().max() / gV.abs().max())}


def serving_requests(count, seed=7):
    """A bounded sample of the serving stream: request sizes log-uniform in [1e3, 2e6] vertices,
    half icospheres (levels 4..8), half square grids whose side is snapped to one of 32
    log-spaced sides (so the sample's meshes are generated once), t log-uniform in [1e-4, 1e-2].
    Arrival times are for a rate of 1/s; the caller rescales them."""
    import dataclasses
    from paper_2602_12105_gb300 import meshgen as mg
    from paper_2602_12105_gb300 import serve
    stream = mg.request_stream(count, 1.0, seed=seed)
    sides = np.unique(np.round(np.exp(np.linspace(np.log(32), np.log(1414), 32))).astype(int))
    bank = {}
    reqs = []
    for rq in stream:
        size = rq.size if rq.kind == "ico" else int(sides[np.argmin(np.abs(np.log(sides) - np.log(rq.size)))])
        key = (rq.kind, size)
        if key not in bank:
            bank[key] = mg.request_problem(mg.Request(0, 0.0, rq.kind, size, 1e-3, seed * 7919 + len(bank)))
        base = bank[key]

        def make(base=base, t=rq.t, rid=rq.rid):
            return dataclasses.replace(base, t=t, name=f"req{rid}")
        reqs.append(serve.make_request(rq.rid, rq.arrival_s, make, base.n, base.m))
    return reqs


def _window_rate(done):
    """Requests completed between the first and the last arrival, per second of that window (the
    steady-state throughput, without the drain after the last arrival)."""
    if not done:
        return None
    a0 = min(r.arrival_s for r in done)
    a1 = max(r.arrival_s for r in done)
    if a1 <= a0:
        return None
    k = sum(1 for r in done if r.status == 0 and r.done_s is not None and r.done_s <= a1)
    return k / (a1 - a0)


def variant_serving(dev, tol, count, loads=(0.5, 0.8, 0.95), spot_checks=4):
    """Continuous batching (mixed precision) against the plain path (one request at a time, FP64,
    first come first served) on the same request sample: the closed-loop capacity of both servers;
    Poisson streams at 0.5, 0.8 and 0.95 x the continuous-batching capacity through the
    continuous-batching server (p50/p99 latency, throughput over the whole run and over the arrival
    window), and the 0.8 stream through the plain server; served results of a few requests
    against the CPU oracle."""
    import copy
    import oracle
    from paper_2602_12105_gb300 import serve
    reqs = serving_requests(count)
    sizes = np.array([r.n_hint for r in reqs])

    def fresh(r, arrival):
        c = copy.copy(r)
        c.arrival_s = arrival
        c.iterations = []
        return c

    # closed loop: every request waiting at t = 0 (results kept for the spot checks)
    srv = serve.Server(precision="mixed", rel_tol=tol, keep_results=True)
    t0 = time.perf_counter()
    done = srv.run([fresh(r, 0.0) for r in reqs], realtime=False)
    wall = time.perf_counter() - t0
    cap = serve.latency_summary(done, wall)
    cap["stats"] = dict(srv.stats)
    # served results against the oracle (the smallest requests: the oracle solves them in well under a second)
    checks = []
    by_id = {r.rid: r for r in done}
    for r in sorted(reqs, key=lambda q: q.n_hint)[:spot_checks]:
        d = by_id[r.rid]
        prob = r.make()
        ref = oracle.forward_adjoint(prob.V, prob.F, prob.B, prob.t, prob.T, prob.b_is_V, tol=1e-13, method="pcg")
        gV = d.gV.cpu().numpy()
        U = d.U.cpu().numpy()
        checks.append({"rid": r.rid, "n": int(prob.n), "t": prob.t,
                       "U_rel_err": float(np.linalg.norm(U - ref["U"]) / np.linalg.norm(ref["U"])),
                       "gV_rel_err": float(np.linalg.norm(gV - ref["gV"]) / np.linalg.norm(ref["gV"]))})
    for d in done:
        d.gV = d.U = None
    # closed loop of the plain server
    plain_srv = serve.PlainServer(rel_tol=tol)
    t0 = time.perf_counter()
    done_p = plain_srv.run([fresh(r, 0.0) for r in reqs], realtime=False)
    plain_cap = serve.latency_summary(done_p, time.perf_counter() - t0)
    # open-loop streams
    streams = {}
    for lf in loads:
        rate = lf * cap["solves_per_s"]
        srv = serve.Server(precision="mixed", rel_tol=tol)
        t0 = time.perf_counter()
        d_s = srv.run([fresh(r, r.arrival_s / rate) for r in reqs], realtime=True)
        summ = serve.latency_summary(d_s, time.perf_counter() - t0)
        summ["offered_rate_per_s"] = round(rate, 3)
        summ["window_solves_per_s"] = _window_rate(d_s)
        summ["stats"] = dict(srv.stats)
        streams[f"{lf:g}"] = summ
    rate = 0.8 * cap["solves_per_s"]
    plain_srv = serve.PlainServer(rel_tol=tol)
    t0 = time.perf_counter()
    d_p = plain_srv.run([fresh(r, r.arrival_s / rate) for r in reqs], realtime=True)
    plain = serve.latency_summary(d_p, time.perf_counter() - t0)
    plain["offered_rate_per_s"] = round(rate, 3)
    plain["window_solves_per_s"] = _window_rate(d_p)
    served = streams["0.8"]
    return {"workload": f"{count} requests (a bounded sample of the 10k stream, the first {count} of the same seeded "
                        f"stream: the whole stream would take about 5 min per load point of the continuous-batching "
                        f"server alone): vertex counts log-uniform [1e3, 2e6] (median {int(np.median(sizes))}), half "
                        f"icospheres (levels 4..8), half square grids, t log-uniform [1e-4, 1e-2], k=3, forward + "
                        f"adjoint to {tol:g}, 150 GB HBM budget",
            "closed_loop_capacity": cap, "plain_fifo_closed_loop_capacity": plain_cap,
            "continuous_batching_mixed": streams, "plain_fp64_fifo_at_0.8": plain,
            "oracle_spot_checks": checks,
            "capacity_ratio_vs_plain": (cap["solves_per_s"] / plain_cap["solves_per_s"])
            if plain_cap["solves_per_s"] else None,
            "p99_ratio_plain_over_served_at_0.8": (plain["p99_ms"] / served["p99_ms"])
            if served["p99_ms"] and plain["p99_ms"] else None}


def run_variants(args, p, U64, gV64, dev, alu):
    from paper_2602_12105_gb300 import _native, api
    want = set(x.strip() for x in args.variants.split(",") if x.strip())
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    out = {}
    t_start = time.perf_counter()
    clocks_guess = {"sm_mhz": None}
    if "small" in want:
        out["ico3_fp64"] = variant_small(api, _native, dev)
    if "mixed" in want:
        out["grid1024_mixed"] = variant_mixed_grid(api, _native, dev, p, args.tol, 100, U64, gV64, clocks_guess, alu)
    if "largest" in want:
        out["grid4096x2048_mixed"] = variant_largest(api, _native, dev, args.tol, 10, clocks_guess, alu)
    if "batch" in want:
        out["batch256_icospheres"] = variant_batch(api, _native, dev, args.tol, 6)
    if "fairing" in want:
        out["inverse_fairing_ico7"] = variant_fairing(api, _native, dev, 20)
    if "eigs" in want:
        out["eigs_ico7"] = variant_eigs(api, dev, 40)
    if "rgd" in want:
        out["rgd_grid257"] = variant_rgd(api, dev, 100)
        try:
            out["rgd_adjoint_terrain33"] = variant_rgd_adjoint(api, dev)
        except _native.IgError as exc:   # reported in the line, the other variants still run
            out["rgd_adjoint_terrain33"] = {"error": str(exc)}
    if "serve" in want and args.serve_requests > 0:
        out["serving"] = variant_serving(dev, args.tol, args.serve_requests)
    out["clocks"] = sampler.stop()
    out["wall_s"] = round(time.perf_counter() - t_start, 1)
    return out


def cpu_baseline(p, args):
    """The oracle as it stands (single-threaded FP64 C) on one full step of the same workload."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.forward_adjoint(p.V, p.F, p.B, p.t, p.T, p.b_is_V, tol=args.tol, method="pcg")
    dt = time.perf_counter() - t0
    del r
    return {"value": round(1.0 / dt, 5), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one full forward+adjoint step of {p.name} ({p.n} vertices) by the single-threaded "
                      f"FP64 C oracle, Jacobi-PCG to {args.tol:g}; {dt:.2f} s"}


# ------------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle as it stands (single-threaded FP64 C) on the very configuration the main arm
    names: every step is one whole forward + adjoint step of the full mesh (operator, both
    Jacobi-PCG solves to --tol, the per-face gradient), timed on the host's wall clock."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    p = make_problem(args.workload, 0)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.forward_adjoint(p.V, p.F, p.B, p.t, p.T, p.b_is_V, tol=args.tol, method="pcg")
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_step = float(np.sum(times)) / len(times)
    value = 1.0 / per_step
    cpu = {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"the full workload: {args.steps} timed steps (after {args.warmup} untimed), each one whole "
                     f"forward + adjoint step of {p.name} ({p.n} vertices) by the single-threaded FP64 C oracle; "
                     f"{len(os.sched_getaffinity(0))} host cores present, 1 used"}
    return {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(per_step * 1000, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(p, "fp64", args.tol), "mesh": p.name, "n": p.n, "m": p.m},
            "impl": "reference", "cpu_baseline": cpu,
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def oracle_timings(args):
    """The CPU oracle as it stands (single-threaded FP64 C, Jacobi-PCG to tol) on the host cores:
    one forward + adjoint step of the small icosphere and the 1024^2 grid (best of 3 and of 1), and
    one step each of the 4096 x 2048 grid and of the 256-mesh batch (the sum over its meshes)."""
    import oracle
    from paper_2602_12105_gb300 import meshgen as mg
    oracle.build()

    def step(q):
        t0 = time.perf_counter()
        oracle.forward_adjoint(q.V, q.F, q.B, q.t, q.T, q.b_is_V, tol=args.tol, method="pcg")
        return time.perf_counter() - t0

    out = {"kind": "oracle", "threads": oracle.num_threads(), "host_cores": len(os.sched_getaffinity(0)),
           "tol": args.tol, "unit": UNIT, "configs": {}}
    for name, reps in (("ico3", 3), ("grid1024", 1), ("grid4096x2048", 1)):
        q = make_problem(name, 0)
        dt = min(step(q) for _ in range(reps))
        out["configs"][name] = {"n": int(q.n), "seconds_per_step": round(dt, 4), "solves_per_s": round(1.0 / dt, 5)}
        del q
    probs = mg.config_batch(seed=0, count=256)
    dt = sum(step(q) for q in probs)
    out["configs"]["batch256_icospheres"] = {"n": int(sum(q.n for q in probs)), "meshes": len(probs),
                                             "seconds_for_all": round(dt, 3),
                                             "solves_per_s": round(len(probs) / dt, 4)}
    return out


def main():
    args = parse()
    if args.oracle_timings:
        print(json.dumps(oracle_timings(args)), flush=True)
        return
    if args.fma_peak:
        import torch

        from paper_2602_12105_gb300 import _native
        torch.cuda.set_device(0)
        print(json.dumps(measure_alu_peaks(_native, 0, torch.cuda.current_stream().cuda_stream)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_ours(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
