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
    ap.add_argument("--workload", default="grid1024", choices=["grid1024", "ico3", "grid2048", "grid4096x2048"])
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--launch", default="graph", choices=["graph", "host"],
                    help="graph: device-side solver loop (default); host: one launch per kernel")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel timing pass")
    return ap.parse_args()


def make_problem(name, seed):
    from paper_2602_12105_gb300 import meshgen as mg
    if name == "grid1024":
        return mg.config_grid1024(seed)
    if name == "grid4096x2048":
        return mg.config_grid4096x2048(seed)
    if name == "grid2048":
        return mg.config_grid(2048, 2048, seed)
    return mg.config_ico3(seed)


def workload_desc(p, precision, tol):
    return (f"{p.name}: {p.n} vertices, {p.m} faces, k={p.B.shape[1]} RHS, t={p.t:.3e}, "
            f"{precision}, forward + adjoint to relative residual {tol:g}, dl/dV gathered")


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"ig_clocks_{os.getpid()}.csv")

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


def algorithmic(kernel, n, m, nnz, k, prec):
    """(FP64-or-FP32 flops, bytes) one launch of `kernel` must do / move (vectors [n][k])."""
    sv = 8 if prec == "fp64" else 4   # value and vector element size
    kp = 4 if k == 3 else k
    if kernel == "pcg_spmv":
        flops = 2 * k * nnz + 2 * k * n
        byts = nnz * (sv + 4) + 4 * (n + 1) + sv * kp * n + sv * k * n
    elif kernel == "pcg_update":
        flops = 10 * k * n + k * n
        byts = sv * (n + 4 * k * n + kp * n - k * n) + 2 * sv * k * n
    elif kernel == "pcg_pupdate":
        flops = 3 * k * n
        byts = sv * (n + k * n + kp * n) + sv * kp * n
    elif kernel == "assemble_face":
        flops = 60 * m
        byts = 12 * m + 24 * n + 32 * m
    elif kernel == "vjp_face":
        flops = 330 * m
        byts = 12 * m + 24 * n + 3 * 8 * k * n + 72 * m
    else:
        return None, None
    return float(flops), float(byts)


# ------------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2602_12105_gb300 import _native, api

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    precision = args.precision or ("mixed" if args.workload == "grid4096x2048" else "fp64")
    p = make_problem(args.workload, seed=rank)
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
    _, _, _, ainfo = mesh.adjoint(V, B, p.b_is_V, U0, U0 - T, opts=opts, info=True)
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
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1000.0)

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
        if world > 1:
            t = torch.tensor([ems], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": world * args.e2e_steps / (ems / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(hV.nbytes + hB.nbytes + hT.nbytes), "d2h_bytes_per_step": int(hG.nbytes)}

    if rank != 0:
        return None

    # roofline of the dominant kernel
    its_f, its_a = finfo["iterations"], ainfo["iterations"]
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    hbm_peak, peak_kind = peaks()
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fp64_peak_tflops = 152 * 2 * 2 * sm_mhz * 1e6 / 1e12     # 2 FP64 FMA / clk / SM
    fp32_peak_tflops = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12   # 128 FP32 FMA / clk / SM
    rl_all = {}
    for name, (cnt, ms) in prof.items():
        fl, by = algorithmic(name, p.n, p.m, mesh.nnz, k, "fp64" if name.startswith(("assemble", "vjp")) or
                             precision == "fp64" else "fp32")
        if fl is None:
            continue
        avg_s = ms / cnt / 1000.0
        alu_peak = fp64_peak_tflops if (precision == "fp64" or name.startswith(("assemble", "vjp"))) \
            else fp32_peak_tflops
        rl_all[name] = {"avg_us": avg_s * 1e6, "launches": cnt,
                        "gbs": by / avg_s / 1e9, "hbm_frac": by / avg_s / 1e9 / hbm_peak,
                        "tflops": fl / avg_s / 1e12, "alu_frac": fl / avg_s / 1e12 / alu_peak}
    d = rl_all.get(dom)
    if d is None:
        roofline = None
    elif d["alu_frac"] >= d["hbm_frac"]:
        roofline = {"bound": "alu", "achieved": round(d["tflops"], 4), "peak": round(
            fp64_peak_tflops if precision == "fp64" or dom.startswith(("assemble", "vjp")) else fp32_peak_tflops, 4),
            "unit": "TFLOP/s", "frac": round(d["alu_frac"], 4), "traffic": measured_traffic(dom, args.workload),
            "kernel": dom, "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x median SM clock under load",
            "hbm_gbs": round(d["gbs"], 1), "hbm_frac_of_measured": round(d["hbm_frac"], 4)}
    else:
        roofline = {"bound": "hbm", "achieved": round(d["gbs"], 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(d["hbm_frac"], 4), "traffic": measured_traffic(dom, args.workload),
                    "kernel": dom, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}

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
        "kernels": {kname: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in kv.items()}
                    for kname, kv in rl_all.items()},
        "gpu_launches": int(args.steps * (2 + (2 + 3 * its_f) + (2 + 3 * its_a) + 2)),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
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
    if rank != 0:
        return None
    import oracle
    from paper_2602_12105_gb300 import meshgen as mg
    oracle.build()
    full = make_problem(args.workload, 0)
    # bounded sample per step: the same family at a side of 128 (grid) or the icosphere itself
    if args.workload.startswith("grid"):
        side = 128
        h = 1.0 / (side - 1)
        sample = mg.problem_grid(side, side, h, h * h, seed=0, name="grid128")
    else:
        sample = full
    scale = sample.n / full.n
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.forward_adjoint(sample.V, sample.F, sample.B, sample.t, sample.T, sample.b_is_V, tol=args.tol,
                               method="pcg")
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_step = float(np.sum(times)) / len(times) / scale   # seconds per full-size step, scaled by n
    value = 1.0 / per_step
    cpu = {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{sample.name} ({sample.n} vertices) per step, time scaled by vertex count to "
                     f"{full.name} ({full.n} vertices)"}
    return {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(per_step * 1000, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(full, "fp64", args.tol)}, "impl": "reference",
            "cpu_baseline": cpu, "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}


def main():
    args = parse()
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
