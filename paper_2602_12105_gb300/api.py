"""Python API over the native library: contexts, meshes and a differentiable smoothing step.

PyTorch supplies device memory and the CUDA stream; every step of the computation runs in the
library's kernels (assemble, solve, adjoint). The differentiable entry point `smooth` follows the
paper's "differentiable linear_solve with a non-differentiable solver" pattern (§5.2): the forward
solves (M + tL) U = M B (§7.1) and the backward solves the adjoint system with the same operator.
"""
from __future__ import annotations

import ctypes
import warnings
from typing import Optional

import numpy as np
import torch

from . import _native as N

# "fp64": FP64 throughout; "mixed": FP32 iterations inside FP64 refinement against the FP64
# operator (the FP64 answer); "mixed32": also FP32 face geometry (FP64 for near-degenerate faces),
# the FP32 operator solved exactly (see IG_PRECISION_MIXED_GEOM32 in the C header)
_PREC = {"fp64": N.IG_PRECISION_FP64, "mixed": N.IG_PRECISION_MIXED, "mixed32": N.IG_PRECISION_MIXED_GEOM32}


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _require_cuda():
    if not torch.cuda.is_available():
        raise N.NativeLibraryError("a CUDA device is required: this library has no CPU path")


def make_opts(rel_tol=1e-10, max_iter=20000, launch="graph", inner_tol=1e-5, max_refine=30):
    o = N.SolveOpts()
    N.load().ig_default_opts(ctypes.byref(o))
    o.rel_tol = float(rel_tol)
    o.max_iter = int(max_iter)
    o.launch = N.IG_LAUNCH_GRAPH if launch == "graph" else N.IG_LAUNCH_HOST
    o.inner_tol = float(inner_tol)
    o.max_refine = int(max_refine)
    return o


class Context:
    """One library context on one CUDA device (work goes on torch's current stream)."""

    def __init__(self, device=None):
        _require_cuda()
        self.lib = N.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.h = ctypes.c_void_p()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        N.check(self.lib.ig_create(ctypes.byref(self.h), self.device.index, ctypes.c_void_p(stream)))

    def sync_stream(self):
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.lib.ig_set_stream(self.h, ctypes.c_void_p(stream))

    def check(self, status):
        N.check(status, self.h)

    def close(self):
        if self.h:
            self.lib.ig_destroy(self.h)
            self.h = ctypes.c_void_p()


_default_ctx: dict = {}


def default_context(device=None) -> Context:
    _require_cuda()
    idx = torch.cuda.current_device() if device is None else (torch.device(device).index or 0)
    if idx not in _default_ctx:
        _default_ctx[idx] = Context(idx)
    return _default_ctx[idx]


class Mesh:
    """A triangle mesh uploaded to the library: the CSR pattern and incidence are built once from
    F and reused by every assemble / solve / adjoint (the sparsity pattern does not change with
    the positions, §7.1)."""

    def __init__(self, F: torch.Tensor, n: int, ctx: Optional[Context] = None):
        self.ctx = ctx or default_context(F.device if F.is_cuda else None)
        F = F.to(device=self.ctx.device, dtype=torch.int32).contiguous()
        if F.dim() != 2 or F.shape[1] != 3:
            raise ValueError("F must be [m][3]")
        self.n, self.m = int(n), int(F.shape[0])
        self.h = ctypes.c_void_p()
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_mesh_upload(self.ctx.h, _ptr(F), self.m, self.n, ctypes.byref(self.h)))
        nnz, nbytes = ctypes.c_int64(), ctypes.c_int64()
        self.ctx.lib.ig_mesh_info(self.h, None, None, ctypes.byref(nnz), ctypes.byref(nbytes))
        self.nnz, self.device_bytes = nnz.value, nbytes.value
        self.t = None
        self.precision = None
        self._token = None

    # -- helpers
    def _dev(self, x: torch.Tensor, cols=None, name="array"):
        if x.device != self.ctx.device or x.dtype != torch.float64:
            raise ValueError(f"{name} must be a float64 tensor on {self.ctx.device}")
        x = x.contiguous()
        if x.dim() != 2 or x.shape[0] != self.n or (cols is not None and x.shape[1] != cols):
            raise ValueError(f"{name} must be [{self.n}][{cols or 'k'}]")
        return x

    def close(self):
        if self.h:
            self.ctx.lib.ig_mesh_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    # -- library calls
    def set_cot_clamp(self, clamp_min: Optional[float]):
        """Clamp every corner's cotangent from below at clamp_min in later assemblies (and their
        gradients), or restore the plain cotangents with None (ig_mesh_set_cot_clamp). The mesh
        must be assembled again afterwards."""
        self.ctx.sync_stream()
        on = clamp_min is not None
        self.ctx.check(self.ctx.lib.ig_mesh_set_cot_clamp(self.h, 1 if on else 0, float(clamp_min) if on else 0.0))
        self.clamp_min = clamp_min
        self._token = None
        return self

    def assemble(self, V: torch.Tensor, t: float, precision: str = "fp64"):
        V = self._dev(V, 3, "V")
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_assemble(self.h, _ptr(V), float(t), _PREC[precision]))
        self.t, self.precision = float(t), precision
        self._token = (V.data_ptr(), V._version, float(t), precision)
        self._V = V
        return self

    def check(self):
        self.ctx.check(self.ctx.lib.ig_check(self.h))

    def operator(self):
        A = torch.empty(self.nnz, dtype=torch.float64, device=self.ctx.device)
        M = torch.empty(self.n, dtype=torch.float64, device=self.ctx.device)
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_operator(self.h, _ptr(A), _ptr(M)))
        return A, M

    def operator32(self):
        """The FP32 operator of a mixed-precision assembly, on the pattern (ig_operator32)."""
        A = torch.empty(self.nnz, dtype=torch.float32, device=self.ctx.device)
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_operator32(self.h, _ptr(A)))
        return A

    def mass(self):
        """The lumped mass M [n] of the assembled operator."""
        M = torch.empty(self.n, dtype=torch.float64, device=self.ctx.device)
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_operator(self.h, None, _ptr(M)))
        return M

    def mass_vjp(self, V: torch.Tensor, w: torch.Tensor):
        """d(sum_i M_i(V) w_i)/dV [n][3] for per-vertex weights w [n] (ig_mass_vjp)."""
        V = self._dev(V, 3, "V")
        w = w.to(device=self.ctx.device, dtype=torch.float64).contiguous().reshape(-1)
        if w.numel() != self.n:
            raise ValueError(f"w must have {self.n} entries")
        gV = torch.empty((self.n, 3), dtype=torch.float64, device=self.ctx.device)
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_mass_vjp(self.h, _ptr(V), _ptr(w), _ptr(gV)))
        return gV

    def pattern(self):
        rowptr = torch.empty(self.n + 1, dtype=torch.int32, device=self.ctx.device)
        col = torch.empty(self.nnz, dtype=torch.int32, device=self.ctx.device)
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_mesh_pattern(self.h, _ptr(rowptr), _ptr(col)))
        return rowptr, col

    def solve(self, B: torch.Tensor, opts=None, info: bool = False, out: Optional[torch.Tensor] = None):
        B = self._dev(B, None, "B")
        k = B.shape[1]
        U = out if out is not None else torch.empty_like(B)
        inf = N.SolveInfo() if info else None
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_solve(self.h, _ptr(B), k, _ptr(U), ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(inf) if inf is not None else None)
        if info:
            if st not in (N.IG_OK, N.IG_ERR_NOT_CONVERGED):
                self.ctx.check(st)
            return U, inf.as_dict()
        self.ctx.check(st)
        return U

    def eigs(self, U0: torch.Tensor, iters: int, opts=None, info: bool = False):
        """The lowest k = U0.shape[1] (<= 4) eigenpairs of L u = lambda M u by the shift-invert
        subspace iteration of Eq. eigiter (§5), starting from U0 [n][k] (linearly independent
        columns), with the shift -1/t of the assembled operator (see ig_eigs). Returns (U, lam)
        with M-orthonormal, canonically signed columns; with info=True also the last solve's
        info."""
        U = self._dev(U0, None, "U0").clone()
        k = U.shape[1]
        lam = (ctypes.c_double * k)()
        inf = N.SolveInfo() if info else None
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_eigs(self.h, k, int(iters), _ptr(U), lam,
                                  ctypes.byref(opts) if opts is not None else None,
                                  ctypes.byref(inf) if inf is not None else None)
        self.ctx.check(st)
        lam_t = torch.tensor(list(lam), dtype=torch.float64)
        return (U, lam_t, inf.as_dict()) if info else (U, lam_t)

    def rgd_u_step(self, V: torch.Tensor, sources, y: torch.Tensor, z: torch.Tensor, rho: float, beta: float,
                   opts=None, info: bool = False):
        """The u-step of the regularized-geodesic ADMM (see ig_rgd_u_step): u [n] with
        L u = (m - D y + rho D z) / (beta + rho) off the sources and u = 0 on them, for per-face
        y and z [m][3]. Leaves the mesh to be assembled again before other solves."""
        V = self._dev(V, 3, "V")
        y, z = (x.to(self.ctx.device, torch.float64).contiguous() for x in (y, z))
        if y.shape != (self.m, 3) or z.shape != (self.m, 3):
            raise ValueError(f"y and z must be [{self.m}][3]")
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).ravel())
        u = torch.empty(self.n, dtype=torch.float64, device=self.ctx.device)
        inf = N.SolveInfo() if info else None
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_rgd_u_step(self.h, _ptr(V), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        int(src.size), _ptr(y), _ptr(z), float(rho), float(beta), _ptr(u),
                                        ctypes.byref(opts) if opts is not None else None,
                                        ctypes.byref(inf) if inf is not None else None)
        self._token = None
        self.t = None
        if info:
            if st not in (N.IG_OK, N.IG_ERR_NOT_CONVERGED):
                self.ctx.check(st)
            return u, inf.as_dict()
        self.ctx.check(st)
        return u

    def rgd_admm(self, V: torch.Tensor, sources, rho: float, beta: float, beta_k: float, max_rounds: int,
                 tol: float = 0.0, adapt_rho: bool = False, y: Optional[torch.Tensor] = None,
                 z: Optional[torch.Tensor] = None, opts=None):
        """Rounds of the regularized-geodesic ADMM (see ig_rgd_admm) from y and z (zeros when not
        given), at most max_rounds, stopping early at tol when tol > 0, with residual balancing of
        rho when adapt_rho. Returns (u [n], y [m][3], z [m][3], stats) with stats a dict of the
        rounds run, the last primal and dual residuals, the final rho, the rounds whose warm-started
        u already met the solver tolerance (no solve), whether the rounds met tol ("converged") and
        the worst status of the u-step solves ("solve_status": 0, or IG_ERR_NOT_CONVERGED with a
        warning; other failures raise)."""
        V = self._dev(V, 3, "V")
        dev = self.ctx.device
        y = torch.zeros((self.m, 3), dtype=torch.float64, device=dev) if y is None else \
            y.to(dev, torch.float64).contiguous().clone()
        z = torch.zeros((self.m, 3), dtype=torch.float64, device=dev) if z is None else \
            z.to(dev, torch.float64).contiguous().clone()
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).ravel())
        u = torch.empty(self.n, dtype=torch.float64, device=dev)
        stats = (ctypes.c_double * 5)()
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_rgd_admm(self.h, _ptr(V), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(src.size),
                                      float(rho), float(beta), float(beta_k), int(max_rounds), float(tol),
                                      int(bool(adapt_rho)), _ptr(u), _ptr(y), _ptr(z), stats,
                                      ctypes.byref(opts) if opts is not None else None)
        self._token = None
        self.t = None
        if st == N.IG_ERR_NOT_CONVERGED:
            warnings.warn("rgd_admm: a u-step solve stopped at max_iter above rel_tol")
        else:
            self.ctx.check(st)
        return u, y, z, {"rounds": int(stats[0]), "primal": stats[1], "dual": stats[2], "rho": stats[3],
                         "warm_rounds_without_solve": int(stats[4]),
                         "converged": bool(tol > 0.0 and stats[1] <= tol and stats[2] <= tol), "solve_status": st}

    def rgd_u_step_vjp(self, V: torch.Tensor, sources, y: torch.Tensor, z: torch.Tensor, rho: float, beta: float,
                       u: torch.Tensor, gu: torch.Tensor, opts=None):
        """Gradients (gV [n][3], gy [m][3], gz [m][3]) of a loss through the u-step, for its result
        u and the cotangent gu = dl/du (see ig_rgd_u_step_vjp)."""
        V = self._dev(V, 3, "V")
        y, z, u, gu = (x.to(self.ctx.device, torch.float64).contiguous() for x in (y, z, u, gu))
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).ravel())
        gV = torch.empty((self.n, 3), dtype=torch.float64, device=self.ctx.device)
        gy = torch.empty((self.m, 3), dtype=torch.float64, device=self.ctx.device)
        gz = torch.empty((self.m, 3), dtype=torch.float64, device=self.ctx.device)
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_rgd_u_step_vjp(self.h, _ptr(V), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                            int(src.size), _ptr(y), _ptr(z), float(rho), float(beta), _ptr(u),
                                            _ptr(gu), _ptr(gV), _ptr(gy), _ptr(gz),
                                            ctypes.byref(opts) if opts is not None else None)
        self._token = None
        self.t = None
        self.ctx.check(st)
        return gV, gy, gz

    def rgd_admm_vjp(self, V: torch.Tensor, sources, y: torch.Tensor, z: torch.Tensor, rho: float, beta: float,
                     beta_k: float, gu: torch.Tensor, restart: int = 30, max_iter: int = 300, tol: float = 1e-10,
                     strict: bool = False, return_w: bool = False, opts=None):
        """dl/dV [n][3] through the converged ADMM (see ig_rgd_admm_vjp), for its fixed point (y, z)
        and the cotangent gu = dl/du*. The adjoint system is solved by restarted GMRES; when it stops
        at max_iter above tol this warns (raises with strict=True) and returns the best iterate's
        gradient. Returns (gV, stats) with stats a dict of the Arnoldi steps, the final relative
        residual and whether tol was met, and w = (w_y, w_z) [2][m][3] as well with return_w."""
        V = self._dev(V, 3, "V")
        dev = self.ctx.device
        y, z, gu = (x.to(dev, torch.float64).contiguous() for x in (y, z, gu))
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).ravel())
        gV = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        w = torch.empty((2, self.m, 3), dtype=torch.float64, device=dev) if return_w else None
        stats = (ctypes.c_double * 3)()
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_rgd_admm_vjp(self.h, _ptr(V), src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                          int(src.size), float(rho), float(beta), float(beta_k), _ptr(y), _ptr(z),
                                          _ptr(gu), int(restart), int(max_iter), float(tol), _ptr(gV),
                                          _ptr(w) if w is not None else None, stats,
                                          ctypes.byref(opts) if opts is not None else None)
        self._token = None
        self.t = None
        info = {"iterations": int(stats[0]), "rel_resid": stats[1], "converged": bool(stats[2])}
        if st == N.IG_ERR_NOT_CONVERGED and not strict:
            warnings.warn(f"rgd_admm_vjp: GMRES stopped at max_iter with relative residual {stats[1]:.3e}",
                          RuntimeWarning)
        else:
            self.ctx.check(st)
        return (gV, info, w) if return_w else (gV, info)

    def eigs_vjp(self, V: torch.Tensor, U: torch.Tensor, gU: torch.Tensor, iters: int, opts=None):
        """dl/dV [n][3] through the eigenvector fixed point of eigs (see ig_eigs_vjp), for the
        result U of eigs at the assembled positions V and the cotangent gU = dl/dU."""
        V = self._dev(V, 3, "V")
        U = self._dev(U, None, "U")
        gU = self._dev(gU, U.shape[1], "gU")
        gV = torch.empty((self.n, 3), dtype=torch.float64, device=self.ctx.device)
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_eigs_vjp(self.h, _ptr(V), U.shape[1], int(iters), _ptr(U), _ptr(gU), _ptr(gV),
                                                ctypes.byref(opts) if opts is not None else None))
        return gV

    def adjoint(self, V, B, b_is_V, U, G, want_gB=False, want_gt=False, opts=None, info: bool = False):
        V = self._dev(V, 3, "V")
        G = self._dev(G, None, "G")
        k = G.shape[1]
        U = self._dev(U, k, "U")
        B = None if b_is_V else self._dev(B, k, "B")
        gV = torch.empty((self.n, 3), dtype=torch.float64, device=self.ctx.device)
        gB = torch.empty((self.n, k), dtype=torch.float64, device=self.ctx.device) if want_gB else None
        gt = torch.empty(1, dtype=torch.float64, device=self.ctx.device) if want_gt else None
        inf = N.SolveInfo() if info else None
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_adjoint(self.h, _ptr(V), _ptr(B), int(bool(b_is_V)), _ptr(U), _ptr(G), k, _ptr(gV),
                                     _ptr(gB), _ptr(gt), ctypes.byref(opts) if opts is not None else None,
                                     ctypes.byref(inf) if inf is not None else None)
        if info:
            if st not in (N.IG_OK, N.IG_ERR_NOT_CONVERGED):
                self.ctx.check(st)
            return gV, gB, gt, inf.as_dict()
        self.ctx.check(st)
        return gV, gB, gt


class SmoothSolve(torch.autograd.Function):
    """U = (M(V) + t L(V))^-1 M(V) B, differentiable in V, B and t (adjoint rule of §5.2)."""

    @staticmethod
    def forward(ctx, V, B, t, mesh: Mesh, precision: str, opts):
        b_is_V = B is None
        tval = float(t)
        mesh.assemble(V, tval, precision)
        U = mesh.solve(V if b_is_V else B, opts=opts)
        ctx.mesh, ctx.b_is_V, ctx.t, ctx.precision, ctx.opts = mesh, b_is_V, tval, precision, opts
        ctx.t_is_tensor = isinstance(t, torch.Tensor)
        ctx.save_for_backward(V, U, *(() if b_is_V else (B,)))
        return U

    @staticmethod
    def backward(ctx, gU):
        mesh: Mesh = ctx.mesh
        V, U = ctx.saved_tensors[:2]
        B = None if ctx.b_is_V else ctx.saved_tensors[2]
        if mesh._token != (V.data_ptr(), V._version, ctx.t, ctx.precision):
            mesh.assemble(V, ctx.t, ctx.precision)
        want_gB = (not ctx.b_is_V) and ctx.needs_input_grad[1]
        want_gt = ctx.t_is_tensor and ctx.needs_input_grad[2]
        gV, gB, gt = mesh.adjoint(V, B, ctx.b_is_V, U, gU.to(torch.float64).contiguous(), want_gB=want_gB,
                                  want_gt=want_gt, opts=ctx.opts)
        gt_out = gt.reshape(()) if want_gt else None
        return gV, gB, gt_out, None, None, None


def smooth(mesh: Mesh, V: torch.Tensor, B: Optional[torch.Tensor], t, precision: str = "fp64", opts=None):
    """Differentiable implicit smoothing step: solve (M(V) + t L(V)) U = M(V) B (B = V if None)."""
    return SmoothSolve.apply(V, B, t, mesh, precision, opts)


class EigsFn(torch.autograd.Function):
    """The lowest k eigenvectors U of L(V) u = lambda M(V) u by the shift-invert subspace
    iteration of Eq. eigiter (§5; shift -1/t), differentiable in V through the fixed point
    (ig_eigs_vjp). The eigenvalues are returned alongside, without a gradient."""

    @staticmethod
    def forward(ctx, V, mesh: Mesh, t, U0, iters, adj_iters, opts):
        mesh.assemble(V, float(t), "fp64")
        U, lam = mesh.eigs(U0, iters, opts=opts)
        ctx.mesh, ctx.t, ctx.adj_iters, ctx.opts = mesh, float(t), adj_iters, opts
        ctx.save_for_backward(V, U)
        ctx.mark_non_differentiable(lam)
        return U, lam

    @staticmethod
    def backward(ctx, gU, glam):
        mesh: Mesh = ctx.mesh
        V, U = ctx.saved_tensors
        if mesh._token != (V.data_ptr(), V._version, ctx.t, "fp64"):
            mesh.assemble(V, ctx.t, "fp64")
        gV = mesh.eigs_vjp(V, U, gU.to(torch.float64).contiguous(), ctx.adj_iters, opts=ctx.opts)
        return gV, None, None, None, None, None, None


def eigs(mesh: Mesh, V: torch.Tensor, t: float, U0: torch.Tensor, iters: int, adj_iters: Optional[int] = None,
         opts=None):
    """Differentiable lowest eigenvectors of the pencil (L(V), M(V)) (see EigsFn); adj_iters
    defaults to iters. Returns (U, lam)."""
    return EigsFn.apply(V, mesh, t, U0, iters, adj_iters if adj_iters is not None else iters, opts)


class RgdUStep(torch.autograd.Function):
    """The u-step of the regularized-geodesic ADMM (ig_rgd_u_step), differentiable in V, y and z
    (ig_rgd_u_step_vjp)."""

    @staticmethod
    def forward(ctx, V, y, z, mesh: Mesh, sources, rho, beta, opts):
        u = mesh.rgd_u_step(V, sources, y, z, rho, beta, opts=opts)
        ctx.mesh, ctx.sources, ctx.rho, ctx.beta, ctx.opts = mesh, sources, float(rho), float(beta), opts
        ctx.save_for_backward(V, y, z, u)
        return u

    @staticmethod
    def backward(ctx, gu):
        V, y, z, u = ctx.saved_tensors
        gV, gy, gz = ctx.mesh.rgd_u_step_vjp(V, ctx.sources, y, z, ctx.rho, ctx.beta, u,
                                             gu.to(torch.float64).contiguous(), opts=ctx.opts)
        return gV, gy, gz, None, None, None, None, None


def rgd_u_step(mesh: Mesh, V: torch.Tensor, y: torch.Tensor, z: torch.Tensor, sources, rho: float, beta: float,
               opts=None):
    """Differentiable u-step of the regularized-geodesic ADMM (see RgdUStep)."""
    return RgdUStep.apply(V, y, z, mesh, sources, rho, beta, opts)


class RgdAdmm(torch.autograd.Function):
    """Regularized geodesic distance u* from the ADMM run to its tolerance (ig_rgd_admm, y and z from
    zeros), differentiable in V through the fixed point of the rounds (ig_rgd_admm_vjp)."""

    @staticmethod
    def forward(ctx, V, mesh: Mesh, sources, rho, beta, beta_k, max_rounds, tol, adapt_rho, gmres, opts):
        u, y, z, st = mesh.rgd_admm(V, sources, rho, beta, beta_k, max_rounds, tol=tol, adapt_rho=adapt_rho,
                                    opts=opts)
        ctx.mesh, ctx.sources, ctx.beta, ctx.beta_k, ctx.opts = mesh, sources, float(beta), float(beta_k), opts
        ctx.rho, ctx.gmres, ctx.stats = st["rho"], dict(gmres or {}), st
        ctx.save_for_backward(V, y, z)
        return u

    @staticmethod
    def backward(ctx, gu):
        V, y, z = ctx.saved_tensors
        gV, _ = ctx.mesh.rgd_admm_vjp(V, ctx.sources, y, z, ctx.rho, ctx.beta, ctx.beta_k,
                                      gu.to(torch.float64).contiguous(), opts=ctx.opts, **ctx.gmres)
        return gV, None, None, None, None, None, None, None, None, None, None


def rgd_distance(mesh: Mesh, V: torch.Tensor, sources, rho: float, beta: float, beta_k: float = 1.0,
                 max_rounds: int = 2000, tol: float = 1e-6, adapt_rho: bool = False, gmres=None, opts=None):
    """Differentiable regularized geodesic distance (see RgdAdmm); gmres: keyword arguments of
    Mesh.rgd_admm_vjp (restart, max_iter, tol, strict)."""
    return RgdAdmm.apply(V, mesh, sources, rho, beta, beta_k, max_rounds, tol, adapt_rho, gmres, opts)


class MassFn(torch.autograd.Function):
    """The lumped mass M(V) [n] (area/3 per incident face), differentiable in V."""

    @staticmethod
    def forward(ctx, V, mesh: Mesh):
        t = mesh.t if mesh.t is not None else 0.0
        prec = mesh.precision if mesh.precision is not None else "fp64"
        if mesh._token != (V.data_ptr(), V._version, t, prec):
            mesh.assemble(V, t, prec)
        ctx.mesh = mesh
        ctx.save_for_backward(V)
        return mesh.mass()

    @staticmethod
    def backward(ctx, gM):
        (V,) = ctx.saved_tensors
        return ctx.mesh.mass_vjp(V, gM.to(torch.float64).contiguous()), None


def mass(mesh: Mesh, V: torch.Tensor):
    """Differentiable lumped mass M(V); with smooth() it forms the M-norm loss of §7.1:
    0.5 * (mass(mesh, V)[:, None] * (smooth(mesh, V, None, t) - T) ** 2).sum()."""
    return MassFn.apply(V, mesh)


class InverseFairing:
    """The inverse-fairing optimisation of §7.1, one device-side step per call (ig_fairing_step):
    g(V) = (M + tL)^-1 M V, loss = 1/2 ||T - g(V)||_M^2, and the Sobolev-preconditioned step
    V <- V - eta (M + tL)^-1 dloss/dV with the same operator."""

    def __init__(self, mesh: Mesh, T: torch.Tensor, t: float, eta: float, precision: str = "fp64", opts=None):
        self.mesh = mesh
        self.T = mesh._dev(T, 3, "T")
        self.t, self.eta, self.precision = float(t), float(eta), precision
        self.opts = opts if opts is not None else make_opts()

    def step(self, V: torch.Tensor, want_loss: bool = True, info: bool = False):
        """Update V [n][3] (float64, on the device) in place; returns the loss at the starting V
        (None unless want_loss), and with info the three solves' info dicts."""
        mesh = self.mesh
        if V.dtype != torch.float64 or not V.is_contiguous() or V.device != mesh.ctx.device:
            raise ValueError("V must be a contiguous float64 tensor on the mesh's device")
        loss = ctypes.c_double(0.0)
        infos = (N.SolveInfo * 3)() if info else None
        mesh.ctx.sync_stream()
        st = mesh.ctx.lib.ig_fairing_step(mesh.h, _ptr(V), _ptr(self.T), self.t, self.eta, _PREC[self.precision],
                                          ctypes.byref(self.opts), ctypes.byref(loss) if want_loss else None,
                                          infos)
        mesh.ctx.check(st)
        mesh.t, mesh.precision = self.t, self.precision
        mesh._token = None  # V changed after the assembly
        out = loss.value if want_loss else None
        if info:
            return out, [i.as_dict() for i in infos]
        return out


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = t.data_ptr() if t is not None else None
    return arr


class Batch:
    """Many meshes assembled, solved and differentiated by the same kernel launches (each mesh
    keeps its own t, scalars and convergence test; results equal those of the meshes alone)."""

    def __init__(self, meshes, ctx: Optional[Context] = None):
        self.meshes = list(meshes)
        self.ctx = ctx or self.meshes[0].ctx
        self.h = ctypes.c_void_p()
        handles = (ctypes.c_void_p * len(self.meshes))(*[m.h.value for m in self.meshes])
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_batch_create(self.ctx.h, handles, len(self.meshes), ctypes.byref(self.h)))
        self.ts = None
        self.precision = None

    def __len__(self):
        return len(self.meshes)

    def close(self):
        if self.h:
            self.ctx.lib.ig_batch_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def assemble(self, Vs, ts, precision: str = "fp64"):
        Vs = [m._dev(V, 3, "V") for m, V in zip(self.meshes, Vs)]
        tarr = (ctypes.c_double * len(Vs))(*[float(t) for t in ts])
        self.ctx.sync_stream()
        self.ctx.check(self.ctx.lib.ig_batch_assemble(self.h, _ptr_array(Vs), tarr, _PREC[precision]))
        self.ts, self.precision = [float(t) for t in ts], precision
        for m, V, t in zip(self.meshes, Vs, ts):
            m.t, m.precision = float(t), precision
            m._token = (V.data_ptr(), V._version, float(t), precision)
        return self

    def solve(self, Bs, opts=None, info: bool = False, outs=None):
        Bs = [m._dev(B, None, "B") for m, B in zip(self.meshes, Bs)]
        k = Bs[0].shape[1]
        Us = outs if outs is not None else [torch.empty_like(B) for B in Bs]
        infos = (N.SolveInfo * len(Bs))() if info else None
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_batch_solve(self.h, _ptr_array(Bs), k, _ptr_array(Us),
                                         ctypes.byref(opts) if opts is not None else None, infos)
        if info:
            if st not in (N.IG_OK, N.IG_ERR_NOT_CONVERGED):
                self.ctx.check(st)
            return Us, [i.as_dict() for i in infos]
        self.ctx.check(st)
        return Us

    def adjoint(self, Vs, Bs, b_is_V, Us, Gs, want_gB=False, want_gt=False, opts=None, info: bool = False):
        n = len(self.meshes)
        k = Gs[0].shape[1]
        Vs = [m._dev(V, 3, "V") for m, V in zip(self.meshes, Vs)]
        Gs = [m._dev(G, k, "G") for m, G in zip(self.meshes, Gs)]
        Us = [m._dev(U, k, "U") for m, U in zip(self.meshes, Us)]
        Bs = None if b_is_V else [m._dev(B, k, "B") for m, B in zip(self.meshes, Bs)]
        dev = self.ctx.device
        gVs = [torch.empty((m.n, 3), dtype=torch.float64, device=dev) for m in self.meshes]
        gBs = [torch.empty((m.n, k), dtype=torch.float64, device=dev) for m in self.meshes] if want_gB else None
        gt = torch.empty(n, dtype=torch.float64, device=dev) if want_gt else None
        infos = (N.SolveInfo * n)() if info else None
        self.ctx.sync_stream()
        st = self.ctx.lib.ig_batch_adjoint(self.h, _ptr_array(Vs), _ptr_array(Bs) if Bs else None, int(bool(b_is_V)),
                                           _ptr_array(Us), _ptr_array(Gs), k, _ptr_array(gVs),
                                           _ptr_array(gBs) if gBs else None, _ptr(gt),
                                           ctypes.byref(opts) if opts is not None else None, infos)
        if info:
            if st not in (N.IG_OK, N.IG_ERR_NOT_CONVERGED):
                self.ctx.check(st)
            return gVs, gBs, gt, [i.as_dict() for i in infos]
        self.ctx.check(st)
        return gVs, gBs, gt


class SmoothBatch(torch.autograd.Function):
    """U_i = (M(V_i) + t_i L(V_i))^-1 M(V_i) B_i for every mesh of a batch (B_i = V_i when no B
    is given), differentiable in the V_i (and B_i) by one batched adjoint pass."""

    @staticmethod
    def forward(ctx, batch: "Batch", ts, precision, opts, nB, *tensors):
        n = len(batch)
        Vs = list(tensors[:n])
        Bs = list(tensors[n:n + nB]) if nB else None
        batch.assemble(Vs, ts, precision)
        Us = batch.solve(Vs if Bs is None else Bs, opts=opts)
        ctx.batch, ctx.ts, ctx.precision, ctx.opts, ctx.nB = batch, list(ts), precision, opts, nB
        ctx.save_for_backward(*Vs, *(Bs or []), *Us)
        return tuple(Us)

    @staticmethod
    def backward(ctx, *gUs):
        batch: Batch = ctx.batch
        n = len(batch)
        saved = ctx.saved_tensors
        Vs = list(saved[:n])
        Bs = list(saved[n:n + ctx.nB]) if ctx.nB else None
        Us = list(saved[n + ctx.nB:])
        if any(m._token != (V.data_ptr(), V._version, t, ctx.precision)
               for m, V, t in zip(batch.meshes, Vs, ctx.ts)):
            batch.assemble(Vs, ctx.ts, ctx.precision)
        Gs = [(g if g is not None else torch.zeros_like(U)).to(torch.float64).contiguous() for g, U in zip(gUs, Us)]
        want_gB = ctx.nB > 0 and any(ctx.needs_input_grad[5 + n:5 + n + ctx.nB])
        gVs, gBs, _ = batch.adjoint(Vs, Bs, Bs is None, Us, Gs, want_gB=want_gB, opts=ctx.opts)
        return (None, None, None, None, None, *gVs, *(gBs if gBs else [None] * ctx.nB))


def smooth_batch(batch: Batch, Vs, Bs, ts, precision: str = "fp64", opts=None):
    """Differentiable batched smoothing step; returns the list of U_i."""
    nB = 0 if Bs is None else len(Bs)
    return list(SmoothBatch.apply(batch, list(ts), precision, opts, nB, *Vs, *(Bs or [])))
