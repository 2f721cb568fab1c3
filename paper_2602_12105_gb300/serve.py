"""Continuous-batching server for smoothing requests (one forward + adjoint solve each).

Requests arrive over time (any mix of mesh sizes). The server admits a request as soon as it has
arrived and its device memory fits the HBM budget, uploads its topology (the pattern is built on
the device), assembles its operator and starts its forward solve. All running solves -- forward or
adjoint, at any iteration or refinement -- advance together in shared kernel launches
(ig_batch_iterate); whenever one finishes, the server moves it on (forward -> adjoint -> gradient
-> done), frees its memory and admits waiting requests, then rebuilds the batch. A request gives
the same result alone and in the mix (its reductions depend on its own tiles only).

The solver state of every request stays on the device between quanta; only done flags and the
final gradient travel back.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np
import torch

from . import _native as N
from .api import Batch, Context, Mesh, _ptr, default_context, make_opts


@dataclass
class ServeRequest:
    rid: int
    arrival_s: float                      # arrival time relative to the start of the run
    make: Callable[[], object]            # returns a meshgen.Problem (V, F, B, T, t)
    # filled by the server
    admitted_s: Optional[float] = None
    done_s: Optional[float] = None
    n: int = 0
    gV: Optional[torch.Tensor] = None
    U: Optional[torch.Tensor] = None
    status: int = 0
    iterations: List[int] = field(default_factory=list)

    @property
    def latency_s(self):
        return None if self.done_s is None else self.done_s - self.arrival_s


def estimate_bytes(n: int, m: int, k: int = 3, mixed: bool = True) -> int:
    """Device bytes one request holds: the mesh (topology, operator, solver and gradient
    workspace) and the request's own arrays, with the transient pattern-build buffers."""
    per_v = 4 * 3 + 8 * 2 + 8 * 4 * 5 + (4 + 4 * 4 * 4 if mixed else 0) + 8 * 3 * 5
    per_f = 12 + 24 + 32 + 72
    per_nz = 4 + 4 + 8 + (4 if mixed else 0)
    build = 4 * (13 * n) + 16 * m
    return int(per_v * n + per_f * m + per_nz * 8 * n + build)


class _Live:
    """A request on the device."""

    def __init__(self, req: ServeRequest, ctx: Context, precision: str, opts, stream_dev):
        p = req.make()
        dev = ctx.device

        def dev_t(a, dtype=torch.float64):
            return a.to(device=dev, dtype=dtype).contiguous() if isinstance(a, torch.Tensor) else \
                torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dtype)

        self.req, self.p = req, p
        self.mesh = Mesh(dev_t(p.F, torch.int32), p.n, ctx=ctx)
        self.V = dev_t(p.V)
        self.B = self.V if p.b_is_V else dev_t(p.B)
        self.T = dev_t(p.T)
        self.U = torch.empty((p.n, 3), dtype=torch.float64, device=dev)
        self.G = None
        self.bytes = self.mesh.device_bytes + 5 * p.n * 3 * 8
        self.stage = "fwd"
        self.k = 3
        lib = ctx.lib
        self.mesh.assemble(self.V, p.t, precision)
        ctx.check(lib.ig_solve_begin(self.mesh.h, _ptr(self.B), self.k, 1, ctypes.byref(opts)))
        req.n = p.n

    def advance(self, ctx: Context, opts) -> bool:
        """Called when the running solve finished: returns True when the request is complete."""
        lib = ctx.lib
        info = N.SolveInfo()
        if self.stage == "fwd":
            st = lib.ig_solve_end(self.mesh.h, self.k, _ptr(self.U), ctypes.byref(info))
            self.req.iterations.append(info.iterations)
            if st not in (N.IG_OK, N.IG_ERR_NOT_CONVERGED):
                ctx.check(st)
            self.req.status = max(self.req.status, st)
            self.G = (self.U - self.T).contiguous()
            ctx.check(lib.ig_solve_begin(self.mesh.h, _ptr(self.G), self.k, 0, ctypes.byref(opts)))
            self.stage = "adj"
            return False
        st = lib.ig_solve_end(self.mesh.h, self.k, None, ctypes.byref(info))
        self.req.iterations.append(info.iterations)
        if st not in (N.IG_OK, N.IG_ERR_NOT_CONVERGED):
            ctx.check(st)
        self.req.status = max(self.req.status, st)
        gV = torch.empty((self.p.n, 3), dtype=torch.float64, device=ctx.device)
        ctx.check(lib.ig_vjp(self.mesh.h, _ptr(self.V), _ptr(self.B), int(bool(self.p.b_is_V)), _ptr(self.U),
                             self.k, _ptr(gV), None, None))
        self.req.gV = gV
        self.req.U = self.U
        return True

    def close(self):
        self.mesh.close()


class Server:
    """Continuous batching under an HBM budget.

    budget_bytes: device memory the requests in flight may hold together (admission control).
    quantum: iterations per shared launch round before the server looks at the requests again
             (a round also ends as soon as one running solve finishes).
    keep_results: keep U and gV of every request (tests); otherwise they are dropped once done.
    """

    def __init__(self, ctx: Optional[Context] = None, budget_bytes: float = 150e9, precision: str = "mixed",
                 rel_tol: float = 1e-10, quantum: int = 32, max_batch: int = 256, keep_results: bool = False):
        self.ctx = ctx or default_context()
        self.budget = int(budget_bytes)
        self.precision = precision
        self.opts = make_opts(rel_tol=rel_tol, launch="host")
        self.quantum = int(quantum)
        self.max_batch = int(max_batch)
        self.keep = keep_results
        self.stats = {"admitted": 0, "rejected": 0, "rounds": 0, "rebuilds": 0, "peak_bytes": 0}

    def run(self, requests: List[ServeRequest], realtime: bool = True) -> List[ServeRequest]:
        """Serve `requests` (sorted by arrival). With realtime the arrivals follow the wall clock;
        otherwise every request is available at once (closed-loop capacity)."""
        ctx = self.ctx
        lib = ctx.lib
        pending = sorted(requests, key=lambda r: r.arrival_s)
        waiting: List[ServeRequest] = []
        live: List[_Live] = []
        used = 0
        batch: Optional[Batch] = None
        members: List[_Live] = []
        t0 = time.perf_counter()
        i_next = 0
        done: List[ServeRequest] = []
        retired: List[_Live] = []
        while i_next < len(pending) or waiting or live:
            now = time.perf_counter() - t0
            while i_next < len(pending) and (not realtime or pending[i_next].arrival_s <= now):
                waiting.append(pending[i_next])
                i_next += 1
            # admission: oldest first, while the budget and the batch size allow
            changed = False
            while waiting and len(live) < self.max_batch:
                req = waiting[0]
                est = req_bytes(req)
                if est > self.budget:
                    waiting.pop(0)
                    req.status = N.IG_ERR_OOM
                    req.done_s = time.perf_counter() - t0
                    self.stats["rejected"] += 1
                    done.append(req)
                    continue
                if used + est > self.budget and live:
                    break
                waiting.pop(0)
                req.admitted_s = time.perf_counter() - t0
                lv = _Live(req, ctx, self.precision, self.opts, None)
                lv.est = est
                used += max(est, lv.bytes)
                live.append(lv)
                self.stats["admitted"] += 1
                self.stats["peak_bytes"] = max(self.stats["peak_bytes"], used)
                changed = True
            if not live:
                if i_next < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[i_next].arrival_s - (time.perf_counter() - t0))))
                continue
            if changed or batch is None or len(members) != len(live) or any(a is not b for a, b in zip(members, live)):
                if batch is not None:
                    batch.close()
                members = list(live)
                batch = Batch([lv.mesh for lv in members], ctx=ctx)
                self.stats["rebuilds"] += 1
            flags = (ctypes.c_int * len(members))()
            ctx.sync_stream()
            ctx.check(lib.ig_batch_iterate(batch.h, 3, self.quantum, flags))
            self.stats["rounds"] += 1
            finished = [lv for lv, f in zip(members, flags) if f]
            for lv in finished:
                if lv.advance(ctx, self.opts):
                    torch.cuda.current_stream(ctx.device).synchronize()
                    lv.req.done_s = time.perf_counter() - t0
                    if not self.keep:
                        lv.req.gV = None
                        lv.req.U = None
                    live.remove(lv)
                    used -= max(lv.est, lv.bytes)
                    done.append(lv.req)
                    retired.append(lv)
            if retired and batch is not None:
                # membership changes: the batch that referenced the retired meshes goes first
                batch.close()
                batch = None
                for lv in retired:
                    lv.close()
                retired.clear()
        if batch is not None:
            batch.close()
        return done


def req_bytes(req: ServeRequest) -> int:
    n = getattr(req, "n_hint", 0)
    m = getattr(req, "m_hint", 0)
    if n <= 0:
        return 0
    return estimate_bytes(n, m)


def latency_summary(done: List[ServeRequest], wall_s: float):
    lat = np.array([r.latency_s for r in done if r.latency_s is not None and r.status in (0,)])
    ok = int(sum(1 for r in done if r.status == 0))
    vit = float(sum(r.n * sum(r.iterations) for r in done if r.status == 0))
    return {"requests": len(done), "ok": ok, "solves_per_s": ok / wall_s if wall_s > 0 else None,
            "wall_s": wall_s, "vertex_iterations_per_s": vit / wall_s if wall_s > 0 else None,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "mean_ms": float(lat.mean() * 1e3) if lat.size else None}


def make_request(rid: int, arrival_s: float, make: Callable[[], object], n: int, m: int) -> ServeRequest:
    """A request whose mesh will have n vertices and m faces (used for admission before the
    mesh exists)."""
    r = ServeRequest(rid, arrival_s, make)
    r.n_hint, r.m_hint = int(n), int(m)
    return r


class PlainServer:
    """The plain baseline: requests served one at a time, first come first served, each as a
    whole FP64 solve + adjoint on its own (no batching, no overlap)."""

    def __init__(self, ctx: Optional[Context] = None, precision: str = "fp64", rel_tol: float = 1e-10,
                 keep_results: bool = False):
        self.ctx = ctx or default_context()
        self.precision = precision
        self.opts = make_opts(rel_tol=rel_tol)
        self.keep = keep_results

    def run(self, requests: List[ServeRequest], realtime: bool = True) -> List[ServeRequest]:
        ctx = self.ctx
        pending = sorted(requests, key=lambda r: r.arrival_s)
        t0 = time.perf_counter()
        done = []
        for req in pending:
            if realtime:
                wait = req.arrival_s - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            req.admitted_s = time.perf_counter() - t0
            p = req.make()
            dev = ctx.device

            def dev_t(a, dtype=torch.float64):
                return a.to(device=dev, dtype=dtype).contiguous() if isinstance(a, torch.Tensor) else \
                    torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dtype)

            mesh = Mesh(dev_t(p.F, torch.int32), p.n, ctx=ctx)
            V = dev_t(p.V)
            B = V if p.b_is_V else dev_t(p.B)
            T = dev_t(p.T)
            mesh.assemble(V, p.t, self.precision)
            U, finfo = mesh.solve(B, opts=self.opts, info=True)
            gV, _, _, ainfo = mesh.adjoint(V, B, p.b_is_V, U, U - T, opts=self.opts, info=True)
            torch.cuda.current_stream(dev).synchronize()
            req.iterations = [finfo["iterations"], ainfo["iterations"]]
            req.status = max(finfo["status"], ainfo["status"])
            req.done_s = time.perf_counter() - t0
            req.n = p.n
            if self.keep:
                req.U, req.gV = U, gV
            mesh.close()
            done.append(req)
        return done
