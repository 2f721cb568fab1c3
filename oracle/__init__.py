"""Python access to the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU-baseline
leg use this module; the product library never does. The C source is compiled on first use
with the system C compiler (plain -O2, no fast-math) into oracle/liboracle.so.

Each wrapper names the part of the paper it follows: the forward step of inverse mean
curvature flow (§7.1, (M - tau L) v' = M v, here written A = M + t L with L positive
semidefinite) and the adjoint rule for linear solves (§5.2, built on Eq. 3 of §3.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_INDEX, ERR_DEGENERATE, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_OOM, ERR_NOT_SPD = (
    0, 1, 2, 3, 4, 5, 6, 8)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (only when missing or older than the source)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            L.orc_validate.argtypes = [i64, i64, vp]
            L.orc_face_geometry.argtypes = [i64, vp, i64, vp, vp, vp]
            L.orc_laplacian_csr.argtypes = [i64, vp, i64, vp, vp, vp, vp, i64]
            L.orc_laplacian_csr.restype = i64
            L.orc_mass.argtypes = [i64, vp, i64, vp, vp]
            L.orc_operator.argtypes = [i64, vp, vp, vp, vp, dbl, vp]
            L.orc_spmv.argtypes = [i64, vp, vp, vp, i32, vp, vp]
            L.orc_spmv.restype = None
            L.orc_dense_cholesky_solve.argtypes = [i64, vp, vp, vp, i32, vp, vp]
            L.orc_pcg_solve.argtypes = [i64, vp, vp, vp, i32, vp, vp, dbl, i32, vp, vp]
            L.orc_vjp.argtypes = [i64, vp, i64, vp, dbl, i32, vp, vp, vp, i32, vp, vp, vp]
            L.orc_laplacian_csr_clamp.argtypes = [i64, vp, i64, vp, dbl, vp, vp, vp, i64]
            L.orc_laplacian_csr_clamp.restype = i64
            L.orc_vjp_clamp.argtypes = [i64, vp, i64, vp, dbl, i32, vp, vp, vp, i32, dbl, vp, vp, vp]
            L.orc_mass_vjp.argtypes = [i64, vp, i64, vp, vp, vp]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def validate(F, n):
    F = _i32(F)
    return lib().orc_validate(n, F.shape[0], _p(F))


def face_geometry(V, F):
    """Per-face corner cotangents [m][3] and areas [m] (§7.1's L(v), M(v) ingredients)."""
    V, F = _f64(V), _i32(F)
    m = F.shape[0]
    cot = np.empty((m, 3)); area = np.empty(m)
    st = lib().orc_face_geometry(V.shape[0], _p(V), m, _p(F), _p(cot), _p(area))
    if st:
        raise OracleError(st, "face_geometry")
    return cot, area


def laplacian(V, F, clamp_min=None):
    """Cotangent Laplacian (PSD convention) as CSR: (rowptr int64[n+1], col int32, val f64).
    With clamp_min, every corner's cotangent is clamped from below first (the cotangent weights
    with a minimum of the §4 ARAP listing, read per corner)."""
    V, F = _f64(V), _i32(F)
    n, m = V.shape[0], F.shape[0]
    cap = n + 6 * m
    rowptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(cap, dtype=np.int32)
    val = np.empty(cap)
    if clamp_min is None:
        nnz = lib().orc_laplacian_csr(n, _p(V), m, _p(F), _p(rowptr), _p(col), _p(val), cap)
    else:
        nnz = lib().orc_laplacian_csr_clamp(n, _p(V), m, _p(F), float(clamp_min), _p(rowptr), _p(col), _p(val), cap)
    if nnz < 0:
        raise OracleError(-nnz, "laplacian_csr")
    return rowptr, col[:nnz].copy(), val[:nnz].copy()


def mass(V, F):
    """Barycentric lumped mass diagonal M_ii = sum of incident face areas / 3."""
    V, F = _f64(V), _i32(F)
    M = np.empty(V.shape[0])
    st = lib().orc_mass(V.shape[0], _p(V), F.shape[0], _p(F), _p(M))
    if st:
        raise OracleError(st, "mass")
    return M


def operator(V, F, t, clamp_min=None):
    """A = M + t L on L's pattern. Returns (rowptr, col, Aval, Lval, M)."""
    rowptr, col, Lval = laplacian(V, F, clamp_min)
    M = mass(V, F)
    Aval = np.empty_like(Lval)
    lib().orc_operator(M.shape[0], _p(rowptr), _p(col), _p(Lval), _p(M), float(t), _p(Aval))
    return rowptr, col, Aval, Lval, M


def spmv(rowptr, col, val, X):
    X = _f64(X)
    X2 = X.reshape(X.shape[0], -1)
    Y = np.empty_like(X2)
    lib().orc_spmv(X2.shape[0], _p(rowptr), _p(col), _p(_f64(val)), X2.shape[1], _p(X2), _p(Y))
    return Y.reshape(X.shape)


def dense_cholesky_solve(rowptr, col, Aval, R):
    R = _f64(R)
    R2 = R.reshape(R.shape[0], -1)
    X = np.empty_like(R2)
    st = lib().orc_dense_cholesky_solve(R2.shape[0], _p(rowptr), _p(col), _p(_f64(Aval)), R2.shape[1], _p(R2),
                                        _p(X))
    if st:
        raise OracleError(st, "dense_cholesky_solve")
    return X.reshape(R.shape)


def pcg_solve(rowptr, col, Aval, R, tol=1e-14, max_iter=100000):
    """Textbook Jacobi-PCG per column, x0 = 0. Returns (X, iters, true relres, status)."""
    R = _f64(R)
    R2 = R.reshape(R.shape[0], -1)
    k = R2.shape[1]
    X = np.empty_like(R2)
    iters = np.zeros(k, dtype=np.int32)
    rel = np.zeros(k)
    st = lib().orc_pcg_solve(R2.shape[0], _p(rowptr), _p(col), _p(_f64(Aval)), k, _p(R2), _p(X), float(tol),
                             int(max_iter), _p(iters), _p(rel))
    if st not in (OK, ERR_NOT_CONVERGED):
        raise OracleError(st, "pcg_solve")
    return X.reshape(R.shape), iters, rel, st


def solve(rowptr, col, Aval, R, tol=1e-14, method="auto", max_iter=100000):
    """Dense Cholesky when n <= 3000 (method 'auto' or 'dense'), else Jacobi-PCG to tol."""
    n = rowptr.shape[0] - 1
    if method == "dense" or (method == "auto" and n <= 3000):
        return dense_cholesky_solve(rowptr, col, Aval, R)
    X, _, _, st = pcg_solve(rowptr, col, Aval, R, tol=tol, max_iter=max_iter)
    return X


def vjp(V, F, t, U, Lam, B, b_is_V, clamp_min=None):
    """Closed-form per-face gradient of the loss w.r.t. V (see orc_vjp; with clamp_min, of the
    step assembled from clamped cotangents, orc_vjp_clamp). Returns (gV, gB, gt)."""
    V, F, U, Lam = _f64(V), _i32(F), _f64(U), _f64(Lam)
    n, k = U.shape
    Bc = None if b_is_V else _f64(B)
    gV = np.empty((n, 3))
    gB = None if b_is_V else np.empty((n, k))
    gt = ctypes.c_double(0.0)
    if clamp_min is None:
        st = lib().orc_vjp(n, _p(V), F.shape[0], _p(F), float(t), k, _p(U), _p(Lam), _p(Bc), int(bool(b_is_V)),
                           _p(gV), _p(gB), ctypes.byref(gt))
    else:
        st = lib().orc_vjp_clamp(n, _p(V), F.shape[0], _p(F), float(t), k, _p(U), _p(Lam), _p(Bc),
                                 int(bool(b_is_V)), float(clamp_min), _p(gV), _p(gB), ctypes.byref(gt))
    if st:
        raise OracleError(st, "vjp")
    return gV, gB, gt.value


def forward_adjoint(V, F, B, t, T, b_is_V, tol=1e-14, method="auto", clamp_min=None):
    """The whole path for loss l = 0.5 ||U - T||^2: assemble, solve A U = M B, adjoint
    A Lambda = U - T, gradient. Returns a dict with U, Lam, gV, gB, gt, loss and the operator.
    clamp_min: assemble from clamped cotangents (and differentiate that step)."""
    rowptr, col, Aval, Lval, M = operator(V, F, t, clamp_min)
    Bv = _f64(V) if b_is_V else _f64(B)
    R = M[:, None] * Bv
    U = solve(rowptr, col, Aval, R, tol=tol, method=method)
    G = U - T
    Lam = solve(rowptr, col, Aval, G, tol=tol, method=method)
    gV, gB, gt = vjp(V, F, t, U, Lam, B, b_is_V, clamp_min)
    return dict(U=U, Lam=Lam, gV=gV, gB=gB, gt=gt, loss=0.5 * float(np.sum(G * G)), rowptr=rowptr, col=col,
                Aval=Aval, Lval=Lval, M=M, R=R, G=G)


def mass_vjp(V, F, w):
    """d(sum_i M_i(V) w_i)/dV [n][3] (see orc_mass_vjp)."""
    V, F, w = _f64(V), _i32(F), _f64(w)
    gV = np.empty((V.shape[0], 3))
    st = lib().orc_mass_vjp(V.shape[0], _p(V), F.shape[0], _p(F), _p(w), _p(gV))
    if st:
        raise OracleError(st, "mass_vjp")
    return gV


def mnorm_objective(V, F, T, t, tol=1e-14, method="auto"):
    """The inverse-fairing objective of §7.1 at V: U = g(V) = (M + tL)^-1 M V and
    loss = 1/2 ||T - U||_M^2 = 1/2 sum_i M_i |T_i - U_i|^2, with its gradient by the adjoint rule
    (Eq. 3, B = V) plus the direct dependence through M. Returns a dict with U, loss, gV, G, Lam,
    w and the operator."""
    rowptr, col, Aval, Lval, M = operator(V, F, t)
    V = _f64(V)
    U = solve(rowptr, col, Aval, M[:, None] * V, tol=tol, method=method)
    D = U - _f64(T)
    G = M[:, None] * D                      # dl/dU
    w = 0.5 * np.sum(D * D, axis=1)         # l = sum_i M_i w_i
    Lam = solve(rowptr, col, Aval, G, tol=tol, method=method)
    gV, _, _ = vjp(V, F, t, U, Lam, None, True)
    gV = gV + mass_vjp(V, F, w)
    return dict(U=U, loss=float(np.sum(M * w)), gV=gV, G=G, Lam=Lam, w=w, rowptr=rowptr, col=col, Aval=Aval, M=M)


def fairing_step(V, F, T, t, eta, tol=1e-14, method="auto"):
    """One Sobolev-preconditioned gradient step of the inverse-fairing problem (§7.1): the
    gradient of mnorm_objective smoothed with the same operator, g~ = (M + tL)^-1 g, then
    V - eta g~. Returns (new V, loss at V)."""
    r = mnorm_objective(V, F, T, t, tol=tol, method=method)
    gs = solve(r["rowptr"], r["col"], r["Aval"], r["gV"], tol=tol, method=method)
    return _f64(V) - eta * gs, r["loss"]


def canonical_sign(U):
    """Flip each column so that its first entry (in vertex order) whose magnitude is within a
    relative 1e-6 of the column's largest magnitude is positive: the canonical sign that the
    orthonormalization Q of Eq. eigiter (§5) chooses, in the reading taken here. (Eigenvectors of
    symmetric meshes reach their largest magnitude at several vertices, with either sign, so the
    first such vertex is taken rather than the largest entry itself.)"""
    U = _f64(U).copy()
    A = np.abs(U)
    big = A >= (1.0 - 1e-6) * A.max(axis=0)[None, :]
    j = np.argmax(big, axis=0)
    s = np.where(U[j, np.arange(U.shape[1])] < 0.0, -1.0, 1.0)
    return U * s[None, :]


def m_orthonormalize(Y, M):
    """Q of Eq. eigiter: an M-orthonormal basis of the columns of Y in Gram-Schmidt order, Y = Q R
    with R upper triangular (the transposed Cholesky factor of the Gram matrix Y^T M Y), followed
    by the canonical sign of each column."""
    Y = _f64(Y)
    G = Y.T @ (M[:, None] * Y)
    R = np.linalg.cholesky(G).T
    Q = np.linalg.solve(R.T, Y.T).T
    return canonical_sign(Q)


def subspace_iteration(V, F, t, U0, iters, tol=1e-14, method="auto"):
    """Shift-invert subspace iteration of Eq. eigiter (§5) for the eigenpairs of L u = lambda M u
    with the shift sigma = -1/t: (L - sigma M)^-1 M = t (M + t L)^-1 M, so each step solves
    (M + t L) Y = M U with the smoothing operator of §7.1 and takes U = Q(Y). The constant t drops
    out in Q. Returns (U, lam) with lam_c = u_c^T L u_c (u_c M-normalized)."""
    rowptr, col, Aval, Lval, M = operator(V, F, t)
    U = _f64(U0)
    for _ in range(int(iters)):
        Y = solve(rowptr, col, Aval, M[:, None] * U, tol=tol, method=method)
        U = m_orthonormalize(Y, M)
    LU = spmv(rowptr, col, Lval, U)
    return U, np.sum(U * LU, axis=0)


def _phi(C):
    """Upper triangle with half the diagonal: the map X = Phi(R^-T dG R^-1) with X + X^T =
    R^-T dG R^-1 that gives dR R^-1 for the Cholesky factor (and is its own adjoint)."""
    return np.triu(C) - 0.5 * np.diag(np.diag(C))


def eigs_vjp(V, F, t, U, gU, iters, tol=1e-14, method="auto"):
    """Gradient of a loss l(U*) with respect to the positions V through the fixed point of
    Eq. eigiter (§5), U* = f(U*) = Q(S U*) with S = (M + tL)^-1 M (the factor t of the shift
    drops out in Q), by the implicit-function rule for fixed points: w = gU + J^T w with
    J = df/dU at U*, solved here by its Neumann series (iters terms; it converges at the forward
    iteration's own rate when the k lowest eigenvalues are distinct), then dl/dV = (df/dV)^T w.
    The Q step's adjoint is that of the Cholesky factor of Y^T M Y. U: the converged basis
    [n][k] (canonical signs); gU = dl/dU [n][k]. Returns gV [n][3]."""
    rowptr, col, Aval, Lval, M = operator(V, F, t)
    U, gU = _f64(U), _f64(gU)
    Y = solve(rowptr, col, Aval, M[:, None] * U, tol=tol, method=method)
    R = np.linalg.cholesky(Y.T @ (M[:, None] * Y)).T
    Ri = np.linalg.inv(R)
    Qraw = Y @ Ri
    s = np.where(np.sum(M[:, None] * Qraw * U, axis=0) < 0.0, -1.0, 1.0)

    def ybar(w):
        Qb = w * s[None, :]
        P = Ri @ _phi(Qraw.T @ Qb) @ Ri.T
        return Qb @ Ri.T - (M[:, None] * Y) @ (P + P.T), P

    w = gU
    for _ in range(int(iters)):
        Yb, _ = ybar(w)
        w = gU + M[:, None] * solve(rowptr, col, Aval, Yb, tol=tol, method=method)
    Yb, P = ybar(w)
    Lam = solve(rowptr, col, Aval, Yb, tol=tol, method=method)
    gV, _, _ = vjp(V, F, t, Y, Lam, U, False)
    wts = -np.einsum("ic,cd,id->i", Y, P, Y)
    return gV + mass_vjp(V, F, wts)


def hat_gradients(V, F):
    """Per face, the gradients of its three piecewise-linear hat functions, [m][3][3] (corner,
    coordinate), and the face areas [m]: grad phi_c = n x e_c / (2 area) with e_c the edge
    opposite corner c taken counter-clockwise (e_0 = p_2 - p_1, ...) and n the unit normal."""
    V, F = _f64(V), _i32(F)
    P = V[F]                                   # [m][3][3]
    e = np.stack([P[:, 2] - P[:, 1], P[:, 0] - P[:, 2], P[:, 1] - P[:, 0]], axis=1)
    N = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    twice = np.linalg.norm(N, axis=1)
    nhat = N / twice[:, None]
    grads = np.cross(nhat[:, None, :], e) / twice[:, None, None]
    return grads, 0.5 * twice


def face_gradient(V, F, u):
    """G u: the gradient of the piecewise-linear function u [n] on every face, [m][3]."""
    grads, _ = hat_gradients(V, F)
    return np.einsum("fcd,fc->fd", grads, _f64(u)[_i32(F)])


def divergence(V, F, Y):
    """D Y = G^T A_F Y: per vertex, the sum over its faces of area * <grad phi, Y_f> for per-face
    vectors Y [m][3]. (With this D the cotangent Laplacian is L = D G.)"""
    grads, area = hat_gradients(V, F)
    contrib = area[:, None] * np.einsum("fcd,fd->fc", grads, _f64(Y))
    out = np.zeros(_f64(V).shape[0])
    np.add.at(out, _i32(F).ravel(), contrib.ravel())
    return out


def rgd_u_step(V, F, sources, y, z, rho, beta, tol=1e-14):
    """The u-step of the ADMM scheme for regularized geodesic distances (§ geodesics, formulation
    eq. edelstein): b = m - D y + rho D z with m the lumped vertex areas, then L u = b / (beta + rho)
    on the vertices that are not sources, u = 0 on the sources (the constraint u_s = 0). Dense
    Cholesky of the reduced Laplacian for small meshes, else Jacobi-PCG to tol."""
    V, F = _f64(V), _i32(F)
    n = V.shape[0]
    rowptr, col, Lval = laplacian(V, F)
    m = mass(V, F)
    b = (m - divergence(V, F, y) + rho * divergence(V, F, z)) / (beta + rho)
    src = np.zeros(n, dtype=bool)
    src[np.asarray(sources, dtype=np.int64)] = True
    # the reduced system as a CSR matrix on all vertices: identity rows and columns at the sources
    Aval = Lval.copy()
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    Aval[src[rows] | src[col]] = 0.0
    Aval[(rows == col) & src[rows]] = 1.0
    rhs = np.where(src, 0.0, b)
    u = solve(rowptr, col, Aval, rhs[:, None], tol=tol)[:, 0]
    u[src] = 0.0
    return u


def divergence_vjp(V, F, lam, W):
    """d(lam^T D W)/dV [n][3] for per-vertex lam [n] and per-face vectors W [m][3] held fixed.
    Per face, sum_c lam_c area <grad phi_c, W_f> = n . (E x W_f) / 2 with E = sum_c lam_c e_c
    (e_c the edge opposite corner c) and n the unit normal; differentiated through E (linear in
    the positions) and through n (dn = (I - n n^T) dN / |N|, N = (p1 - p0) x (p2 - p0))."""
    V, F, lam, W = _f64(V), _i32(F), _f64(lam), _f64(W)
    P = V[F]
    lf = lam[F]                                             # [m][3]
    e = np.stack([P[:, 2] - P[:, 1], P[:, 0] - P[:, 2], P[:, 1] - P[:, 0]], axis=1)
    E = np.einsum("fc,fcd->fd", lf, e)
    a, b = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]
    N = np.cross(a, b)
    nN = np.linalg.norm(N, axis=1)
    nh = N / nN[:, None]
    g = np.zeros((F.shape[0], 3, 3))
    # through E: dE = sum_c (lam_{c+1} - lam_{c+2}) dp_c, and n . (dE x W) = dE . (W x n)
    wxn = np.cross(W, nh)
    for c in range(3):
        g[:, c] += 0.5 * (lf[:, (c + 1) % 3] - lf[:, (c + 2) % 3])[:, None] * wxn
    # through n: v = (I - n n^T)(E x W) / |N|, and v . dN = da . (b x v) + db . (v x a)
    ExW = np.cross(E, W)
    v = (ExW - np.sum(ExW * nh, axis=1)[:, None] * nh) / nN[:, None]
    ga, gb = np.cross(b, v), np.cross(v, a)
    g[:, 1] += 0.5 * ga
    g[:, 2] += 0.5 * gb
    g[:, 0] -= 0.5 * (ga + gb)
    out = np.zeros_like(V)
    np.add.at(out, F.ravel(), g.reshape(-1, 3))
    return out


def rgd_u_step_vjp(V, F, sources, y, z, rho, beta, gu, tol=1e-14):
    """Gradients of l(u) through the u-step (rgd_u_step) for gu = dl/du [n]: with
    lam = L_D^-1 gu (L_D the source-constrained Laplacian, lam = 0 on the sources),
      dl/dy_f = -area_f grad(lam)_f / (beta + rho),   dl/dz_f = rho area_f grad(lam)_f / (beta + rho),
      dl/dV = [<lam, dm> + <lam, dD (rho z - y)>] / (beta + rho) - <lam, dL u>.
    Returns (gV [n][3], gy [m][3], gz [m][3])."""
    V, F = _f64(V), _i32(F)
    n = V.shape[0]
    u = rgd_u_step(V, F, sources, y, z, rho, beta, tol=tol)
    rowptr, col, Lval = laplacian(V, F)
    src = np.zeros(n, dtype=bool)
    src[np.asarray(sources, dtype=np.int64)] = True
    Aval = Lval.copy()
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    Aval[src[rows] | src[col]] = 0.0
    Aval[(rows == col) & src[rows]] = 1.0
    lam = solve(rowptr, col, Aval, np.where(src, 0.0, _f64(gu))[:, None], tol=tol)[:, 0]
    lam[src] = 0.0
    s = 1.0 / (beta + rho)
    grads, area = hat_gradients(V, F)
    agl = area[:, None] * np.einsum("fcd,fc->fd", grads, lam[F])   # area * grad(lam) per face
    gy, gz = -s * agl, rho * s * agl
    # <lam, dm> / (beta + rho) - <lam, dL u>: the smoothing VJP with t = 1 (A = M + L), B = u + s, U = u
    gV, _, _ = vjp(V, F, 1.0, u[:, None], lam[:, None], (u + s)[:, None], False)
    gV = gV + s * divergence_vjp(V, F, lam, rho * _f64(z) - _f64(y))
    return gV, gy, gz


def rgd_admm(V, F, sources, rho, beta, beta_k, iters, y=None, z=None, tol=0.0, adapt_rho=False, solve_tol=1e-14):
    """The ADMM scheme for regularized geodesic distances (formulation eq. edelstein and its
    listing), up to `iters` rounds of: the u-step (rgd_u_step); the z-step z = P(y / rho + G u), P
    the projection of each face's vector onto the unit ball; the dual step
    y += rho (beta_k G u + (1 - beta_k) z_old - z). Residuals of a round: primal = max_f |G u - z|,
    dual = rho max_i |(D (z - z_old))_i| / m_i over the non-source vertices. With tol > 0 the
    rounds stop once both are <= tol; with adapt_rho, rho doubles when primal > 10 dual and halves
    when dual > 10 primal (residual balancing). y and z start at 0 unless given.
    Returns (u, y, z, stats) with stats = (rounds, primal, dual, rho)."""
    V, F = _f64(V), _i32(F)
    m = F.shape[0]
    y = np.zeros((m, 3)) if y is None else _f64(y).copy()
    z = np.zeros((m, 3)) if z is None else _f64(z).copy()
    M = mass(V, F)
    free = np.ones(V.shape[0], dtype=bool)
    free[np.asarray(sources, dtype=np.int64)] = False
    u, primal, dual, rounds = None, 0.0, 0.0, 0
    for it in range(int(iters)):
        u = rgd_u_step(V, F, sources, y, z, rho, beta, tol=solve_tol)
        g = face_gradient(V, F, u)
        zn = y / rho + g
        zn = zn / np.maximum(np.linalg.norm(zn, axis=1), 1.0)[:, None]
        y = y + rho * (beta_k * g + (1.0 - beta_k) * z - zn)
        primal = float(np.linalg.norm(g - zn, axis=1).max())
        dual = float((rho * np.abs(divergence(V, F, zn - z)) / M)[free].max())
        z = zn
        rounds = it + 1
        if tol > 0.0 and primal <= tol and dual <= tol:
            break
        if adapt_rho:
            if primal > 10.0 * dual:
                rho *= 2.0
            elif dual > 10.0 * primal:
                rho *= 0.5
    return u, y, z, (rounds, primal, dual, rho)



def face_gradient_vjp(V, F, u, W):
    """d(sum_f <W_f, (G u)_f>)/dV [n][3] for per-vertex u [n] and per-face vectors W [m][3] held
    fixed. Per face, G u = N x E / |N|^2 with N = (p1 - p0) x (p2 - p0) and E = sum_c u_c e_c (e_c
    the edge opposite corner c), so <W, G u> = N . (E x W) / |N|^2; differentiated through E
    (linear in the positions) and through N (both in the numerator and in |N|^2)."""
    V, F, u, W = _f64(V), _i32(F), _f64(u), _f64(W)
    P = V[F]
    uf = u[F]
    e = np.stack([P[:, 2] - P[:, 1], P[:, 0] - P[:, 2], P[:, 1] - P[:, 0]], axis=1)
    E = np.einsum("fc,fcd->fd", uf, e)
    a, b = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]
    N = np.cross(a, b)
    nn = np.sum(N * N, axis=1)
    g = np.zeros((F.shape[0], 3, 3))
    # through E: N . (dE x W) = dE . (W x N), dE = sum_c (u_{c+1} - u_{c+2}) dp_c
    wxn = np.cross(W, N) / nn[:, None]
    for c in range(3):
        g[:, c] += (uf[:, (c + 1) % 3] - uf[:, (c + 2) % 3])[:, None] * wxn
    # through N: d(N . X / |N|^2) = v . dN with v = X / |N|^2 - 2 (N . X) N / |N|^4, X = E x W;
    # v . dN = da . (b x v) + db . (v x a)
    X = np.cross(E, W)
    sval = np.sum(N * X, axis=1) / nn
    v = X / nn[:, None] - 2.0 * (sval / nn)[:, None] * N
    ga, gb = np.cross(b, v), np.cross(v, a)
    g[:, 1] += ga
    g[:, 2] += gb
    g[:, 0] -= ga + gb
    out = np.zeros_like(V)
    np.add.at(out, F.ravel(), g.reshape(-1, 3))
    return out


def rgd_round(V, F, sources, y, z, rho, beta, beta_k, tol=1e-14):
    """One round T(y, z) of the geodesic ADMM (its listing, fixed rho): u = rgd_u_step(y, z),
    g = G u, z_new = P(y / rho + g), y_new = y + rho (beta_k g + (1 - beta_k) z - z_new).
    Returns (y_new, z_new, u)."""
    y, z = _f64(y), _f64(z)
    u = rgd_u_step(V, F, sources, y, z, rho, beta, tol=tol)
    g = face_gradient(V, F, u)
    a = y / rho + g
    zn = a / np.maximum(np.linalg.norm(a, axis=1), 1.0)[:, None]
    yn = y + rho * (beta_k * g + (1.0 - beta_k) * z - zn)
    return yn, zn, u


def rgd_round_vjp(V, F, sources, y, z, rho, beta, beta_k, wy, wz, tol=1e-14):
    """Vector-Jacobian product of one round (rgd_round) for cotangents wy, wz [m][3] of y_new and
    z_new, by the chain rule through its three steps:
      y_new: y gets wy, g gets rho beta_k wy, z gets rho (1 - beta_k) wy, z_new gets -rho wy;
      z_new = P(a), a = y / rho + g: abar = dP(a)^T (wz - rho wy), with dP = I inside the unit ball
        (|a| <= 1) and (I - ahat ahat^T) / |a| outside; y gets abar / rho, g gets abar;
      g = G u: u gets G^T gbar, V gets the derivative of <gbar, G u> at fixed u;
      u = rgd_u_step(y, z): rgd_u_step_vjp.
    Returns (gV [n][3], gy [m][3], gz [m][3])."""
    V, F, y, z, wy, wz = _f64(V), _i32(F), _f64(y), _f64(z), _f64(wy), _f64(wz)
    u = rgd_u_step(V, F, sources, y, z, rho, beta, tol=tol)
    grads, _ = hat_gradients(V, F)
    g = np.einsum("fcd,fc->fd", grads, u[F])
    a = y / rho + g
    na = np.linalg.norm(a, axis=1)
    zb = wz - rho * wy
    ah = a / na[:, None]
    outside = na > 1.0
    abar = np.where(outside[:, None], (zb - np.sum(ah * zb, axis=1)[:, None] * ah) / na[:, None], zb)
    gy = wy + abar / rho
    gz = rho * (1.0 - beta_k) * wy
    gbar = rho * beta_k * wy + abar
    gu = np.zeros(V.shape[0])
    np.add.at(gu, F.ravel(), np.einsum("fcd,fd->fc", grads, gbar).ravel())
    gV = face_gradient_vjp(V, F, u, gbar)
    gVu, gyu, gzu = rgd_u_step_vjp(V, F, sources, y, z, rho, beta, gu, tol=tol)
    return gV + gVu, gy + gyu, gz + gzu


def rgd_admm_vjp(V, F, sources, y, z, rho, beta, beta_k, gu, tol=1e-14):
    """dl/dV for l(u*) with u* = rgd_u_step(y*, z*) at a fixed point (y*, z*) = T(y*, z*) of the
    ADMM round (the fixed-point implicit layer of the framework section on implicit
    differentiation, applied to the geodesics application): with (gV0, gy0, gz0) the u-step's VJP
    of gu, solve w = (gy0, gz0) + J^T w (J = dT/d(y, z)), then dl/dV = gV0 + (dT/dV)^T w. J^T is
    formed column by column from rgd_round_vjp and the system is solved densely, so this is for
    small meshes. Returns (gV [n][3], w_y [m][3], w_z [m][3])."""
    V, F, y, z = _f64(V), _i32(F), _f64(y), _f64(z)
    m = F.shape[0]
    gV0, gy0, gz0 = rgd_u_step_vjp(V, F, sources, y, z, rho, beta, gu, tol=tol)
    JT = np.zeros((6 * m, 6 * m))
    for j in range(6 * m):
        e = np.zeros(6 * m)
        e[j] = 1.0
        _, cy, cz = rgd_round_vjp(V, F, sources, y, z, rho, beta, beta_k, e[:3 * m].reshape(m, 3),
                                  e[3 * m:].reshape(m, 3), tol=tol)
        JT[:, j] = np.concatenate([cy.ravel(), cz.ravel()])
    w = np.linalg.solve(np.eye(6 * m) - JT, np.concatenate([gy0.ravel(), gz0.ravel()]))
    wy, wz = w[:3 * m].reshape(m, 3), w[3 * m:].reshape(m, 3)
    gVw, _, _ = rgd_round_vjp(V, F, sources, y, z, rho, beta, beta_k, wy, wz, tol=tol)
    return gV0 + gVw, wy, wz

def num_threads():
    return 1
