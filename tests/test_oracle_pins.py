"""Pins of the FP64 CPU oracle to facts fixed by geometry and linear algebra (no GPU).

Each test checks the oracle against something other than itself: closed-form values
(tests/golden/), a different formula for the same object (the P1 finite-element stiffness
matrix, Heron's area), invariants (symmetry, zero row sums, linear precision, rigid-motion
invariance of the gradient, a scaling identity), a library routine (numpy's dense solve) and
brute force (central finite differences of the whole forward pass).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2602_12105_gb300 import meshgen as mg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = np.array([float(v) for v in vals])
    return out


def _dense(rowptr, col, val, n):
    D = np.zeros((n, n))
    for i in range(n):
        for e in range(rowptr[i], rowptr[i + 1]):
            D[i, col[e]] += val[e]
    return D


def _fem_stiffness(V, F):
    """P1 finite-element stiffness K_ab = sum_f area_f grad(phi_a) . grad(phi_b), with
    grad(phi_a) = n x (p_{a+2} - p_{a+1}) / (2 area) on each face (hat functions)."""
    n = V.shape[0]
    K = np.zeros((n, n))
    for f in F:
        P = V[f]
        x = np.cross(P[1] - P[0], P[2] - P[0])
        s = np.linalg.norm(x)
        nrm = x / s
        grads = [np.cross(nrm, P[(a + 2) % 3] - P[(a + 1) % 3]) / s for a in range(3)]
        for a in range(3):
            for b in range(3):
                K[f[a], f[b]] += 0.5 * s * grads[a] @ grads[b]
    return K


def _heron_area(V, F):
    tot = 0.0
    for f in F:
        a = np.linalg.norm(V[f[1]] - V[f[0]])
        b = np.linalg.norm(V[f[2]] - V[f[1]])
        c = np.linalg.norm(V[f[0]] - V[f[2]])
        s = 0.5 * (a + b + c)
        tot += math.sqrt(max(s * (s - a) * (s - b) * (s - c), 0.0))
    return tot


# ----------------------------------------------------------------------------- closed forms
def test_right_triangle_golden():
    g = _read_golden("right_triangle.txt")
    V = g["positions"].reshape(3, 3)
    F = g["faces"].reshape(1, 3).astype(np.int32)
    cot, area = oracle.face_geometry(V, F)
    np.testing.assert_allclose(cot[0], g["cot"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(area, g["area"], rtol=1e-15)
    np.testing.assert_allclose(oracle.mass(V, F), g["mass"], rtol=1e-15)
    rowptr, col, Lval = oracle.laplacian(V, F)
    np.testing.assert_allclose(_dense(rowptr, col, Lval, 3), g["L"].reshape(3, 3), atol=1e-15)


def test_regular_tetrahedron_golden():
    g = _read_golden("regular_tetrahedron.txt")
    V, F = mg.regular_tetrahedron(float(g["edge"][0]))
    cot, area = oracle.face_geometry(V, F)
    np.testing.assert_allclose(cot, g["cot"][0], rtol=1e-14)
    np.testing.assert_allclose(area, g["area"][0], rtol=1e-14)
    np.testing.assert_allclose(oracle.mass(V, F), g["mass"][0], rtol=1e-14)
    rowptr, col, Lval = oracle.laplacian(V, F)
    D = _dense(rowptr, col, Lval, 4)
    off = D[~np.eye(4, dtype=bool)]
    np.testing.assert_allclose(off, g["L_offdiag"][0], rtol=1e-14)
    np.testing.assert_allclose(np.diag(D), g["L_diag"][0], rtol=1e-14)


def test_flat_grid_is_five_point_stencil():
    """On a flat regular grid the cotangents are exactly 1 (45 degrees) and 0 (90 degrees):
    interior rows are the 5-point stencil (4 on the diagonal, -1 on axis neighbours, exactly 0
    on the split diagonal) and interior masses are h^2."""
    nx = ny = 9
    h = 0.125
    V, F = mg.grid_mesh(nx, ny, h)
    rowptr, col, Lval = oracle.laplacian(V, F)
    M = oracle.mass(V, F)
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            v = j * nx + i
            cols = col[rowptr[v]:rowptr[v + 1]]
            vals = Lval[rowptr[v]:rowptr[v + 1]]
            expect = {v: 4.0, v - 1: -1.0, v + 1: -1.0, v - nx: -1.0, v + nx: -1.0,
                      v - nx - 1: 0.0, v + nx + 1: 0.0}
            assert sorted(cols.tolist()) == sorted(expect.keys())
            for c, x in zip(cols, vals):
                assert x == expect[int(c)], (v, c, x)
            assert abs(M[v] - h * h) <= 1e-15 * h * h


# ----------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("level", [1, 3])
def test_closed_mesh_symmetry_and_row_sums(level):
    rng = np.random.default_rng(7)
    V = mg.radial_perturb(mg.icosphere(level)[0], 0.05, rng)
    F = mg.icosphere(level)[1]
    n = V.shape[0]
    rowptr, col, Lval = oracle.laplacian(V, F)
    D = _dense(rowptr, col, Lval, n)
    assert np.array_equal(D, D.T), "L must be exactly symmetric"
    scale = np.abs(Lval).max()
    assert np.abs(D.sum(axis=1)).max() <= 1e-13 * scale
    # adjoint dot-product test <Ax, y> = <x, Ay> through the oracle's own SpMV
    x, y = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    lhs = np.sum(oracle.spmv(rowptr, col, Lval, x) * y)
    rhs = np.sum(x * oracle.spmv(rowptr, col, Lval, y))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_planar_linear_precision():
    """On a planar patch, L annihilates linear functions at interior vertices."""
    rng = np.random.default_rng(3)
    V, F, interior = mg.jittered_planar_grid(14, 11, 0.1, 0.3, rng)
    rowptr, col, Lval = oracle.laplacian(V, F)
    for trial in range(3):
        a, b, c = rng.standard_normal(3)
        f = a * V[:, 0] + b * V[:, 1] + c
        Lf = oracle.spmv(rowptr, col, Lval, f[:, None])[:, 0]
        scale = np.abs(Lval).max() * np.abs(f).max()
        assert np.abs(Lf[interior]).max() <= 1e-13 * scale
        assert np.abs(Lf[~interior]).max() > 1e-6 * scale  # boundary rows are not zero


@pytest.mark.parametrize("which", ["ico2", "grid"])
def test_laplacian_equals_fem_stiffness(which):
    """The cotangent Laplacian equals the P1 finite-element stiffness matrix."""
    rng = np.random.default_rng(11)
    if which == "ico2":
        Vc, F = mg.icosphere(2)
        V = mg.radial_perturb(Vc, 0.1, rng)
    else:
        V, F, _ = mg.jittered_planar_grid(7, 6, 0.2, 0.3, rng)
        V[:, 2] = 0.3 * rng.standard_normal(V.shape[0])
    n = V.shape[0]
    rowptr, col, Lval = oracle.laplacian(V, F)
    K = _fem_stiffness(V, F)
    D = _dense(rowptr, col, Lval, n)
    assert np.abs(D - K).max() <= 1e-13 * np.abs(K).max()


def test_total_mass_converges_to_sphere_area():
    """Sum of M is the polyhedral area (Heron) and rises monotonically toward 4 pi."""
    prev, errs = 0.0, []
    for level in range(0, 9):
        V, F = mg.icosphere(level)
        tot = oracle.mass(V, F).sum()
        if level <= 4:
            assert abs(tot - _heron_area(V, F)) <= 1e-12 * tot
        assert prev < tot < 4 * math.pi
        errs.append(4 * math.pi - tot)
        prev = tot
    ratios = [errs[i] / errs[i + 1] for i in range(3, len(errs) - 1)]
    assert all(3.5 < r < 4.5 for r in ratios), ratios  # second-order convergence
    assert errs[-1] / (4 * math.pi) < 1e-4


# ----------------------------------------------------------------------------- solvers
def test_dense_cholesky_and_pcg_match_numpy():
    p = mg.config_ico3(seed=0)
    rowptr, col, Aval, Lval, M = oracle.operator(p.V, p.F, p.t)
    R = M[:, None] * p.B
    X_chol = oracle.dense_cholesky_solve(rowptr, col, Aval, R)
    X_np = np.linalg.solve(_dense(rowptr, col, Aval, p.n), R)
    assert np.linalg.norm(X_chol - X_np) <= 1e-12 * np.linalg.norm(X_np)
    X_pcg, iters, rel, st = oracle.pcg_solve(rowptr, col, Aval, R, tol=1e-14)
    assert st == oracle.OK and (rel <= 1e-13).all()
    assert np.linalg.norm(X_pcg - X_np) <= 1e-12 * np.linalg.norm(X_np)
    # residual recomputed independently with a dense product
    res = R - _dense(rowptr, col, Aval, p.n) @ X_pcg
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(R, axis=0)).max() <= 1e-13


def test_pcg_reports_not_converged():
    p = mg.config_ico3(seed=0)
    rowptr, col, Aval, Lval, M = oracle.operator(p.V, p.F, p.t)
    X, iters, rel, st = oracle.pcg_solve(rowptr, col, Aval, M[:, None] * p.B, tol=1e-14, max_iter=2)
    assert st == oracle.ERR_NOT_CONVERGED and (iters == 2).all() and (rel > 1e-14).all()


# ----------------------------------------------------------------------------- gradient
def _loss(V, F, B, t, T, b_is_V):
    r = oracle.forward_adjoint(V, F, B, t, T, b_is_V, method="dense")
    return r["loss"]


@pytest.mark.parametrize("b_is_V", [True, False])
def test_gradient_matches_central_differences(b_is_V):
    rng = np.random.default_rng(5)
    Vc, F = mg.icosphere(1)
    V = mg.radial_perturb(Vc, 0.05, rng)
    t = 3e-2
    B = V if b_is_V else rng.uniform(-1, 1, size=V.shape)
    T = Vc if b_is_V else rng.uniform(-1, 1, size=V.shape)
    r = oracle.forward_adjoint(V, F, B, t, T, b_is_V, method="dense")
    g = r["gV"]
    h = 1e-6
    idx = rng.choice(V.size, size=8, replace=False)
    for flat in idx:
        i, d = divmod(int(flat), 3)
        Vp, Vm = V.copy(), V.copy()
        Vp[i, d] += h
        Vm[i, d] -= h
        fd = (_loss(Vp, F, Vp if b_is_V else B, t, T, b_is_V) - _loss(Vm, F, Vm if b_is_V else B, t, T, b_is_V)) / (2 * h)
        assert abs(fd - g[i, d]) <= 1e-6 * np.abs(g).max() + 1e-9, (i, d, fd, g[i, d])
    # d loss / d t
    fd_t = (_loss(V, F, B, t + h * t, T, b_is_V) - _loss(V, F, B, t - h * t, T, b_is_V)) / (2 * h * t)
    assert abs(fd_t - r["gt"]) <= 1e-6 * abs(r["gt"]) + 1e-9
    if not b_is_V:
        for flat in idx[:4]:
            i, c = divmod(int(flat), 3)
            Bp, Bm = B.copy(), B.copy()
            Bp[i, c] += h
            Bm[i, c] -= h
            fd = (_loss(V, F, Bp, t, T, False) - _loss(V, F, Bm, t, T, False)) / (2 * h)
            assert abs(fd - r["gB"][i, c]) <= 1e-6 * np.abs(r["gB"]).max() + 1e-9


def test_gradient_rigid_invariance_and_scaling_identity():
    """With B independent of V the loss is invariant to rigid motions of V, so
    sum_i gV_i = 0 and sum_i V_i x gV_i = 0; and since L is scale invariant while M scales with
    the square of the size, sum_i V_i . gV_i = 2 <Lambda, M (B - U)>."""
    rng = np.random.default_rng(9)
    Vc, F = mg.icosphere(3)
    V = mg.radial_perturb(Vc, 0.05, rng) + np.array([0.3, -0.2, 0.1])
    B = rng.uniform(-1, 1, size=V.shape)
    T = rng.uniform(-1, 1, size=V.shape)
    r = oracle.forward_adjoint(V, F, B, 2e-3, T, False)
    g = r["gV"]
    scale = np.abs(g).max() * V.shape[0]
    assert np.abs(g.sum(axis=0)).max() <= 1e-12 * scale
    assert np.abs(np.cross(V, g).sum(axis=0)).max() <= 1e-12 * scale * np.abs(V).max()
    lhs = float(np.sum(V * g))
    rhs = 2.0 * float(np.sum(r["Lam"] * (r["M"][:, None] * (B - r["U"]))))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + abs(rhs))


# ----------------------------------------------------------------------------- M-norm objective
def test_mass_vjp_area_scaling_and_central_differences():
    """d(sum_i M_i w_i)/dV: with w = 1 the sum is the surface area, a homogeneous function of
    degree 2 in V, so sum_i V_i . gV_i = 2 * area (Euler), and the gradient of a rigidly moved
    mesh rotates with it; for general w it matches central differences of oracle.mass."""
    rng = np.random.default_rng(21)
    Vc, F = mg.icosphere(2)
    V = mg.radial_perturb(Vc, 0.05, rng)
    g1 = oracle.mass_vjp(V, F, np.ones(V.shape[0]))
    area = float(oracle.mass(V, F).sum())
    assert abs(float(np.sum(V * g1)) - 2.0 * area) <= 1e-12 * area
    assert np.abs(g1.sum(axis=0)).max() <= 1e-12 * np.abs(g1).max() * V.shape[0]
    w = rng.random(V.shape[0])
    g = oracle.mass_vjp(V, F, w)
    h = 1e-6
    for flat in rng.choice(V.size, 12, replace=False):
        i, c = divmod(int(flat), 3)
        Vp, Vm = V.copy(), V.copy()
        Vp[i, c] += h
        Vm[i, c] -= h
        fd = (oracle.mass(Vp, F) @ w - oracle.mass(Vm, F) @ w) / (2 * h)
        assert abs(fd - g[i, c]) <= 1e-7 * np.abs(g).max()


def test_mnorm_objective_gradient_matches_central_differences():
    """The inverse-fairing objective 1/2 ||T - g(V)||_M^2 (§7.1, B = V): its adjoint gradient
    plus the mass term against central differences of the whole forward computation."""
    rng = np.random.default_rng(22)
    Vc, F = mg.icosphere(2)
    V = mg.radial_perturb(Vc, 0.03, rng)
    T = Vc.copy()
    t = 5e-3
    r = oracle.mnorm_objective(V, F, T, t)
    g = r["gV"]
    h = 1e-6
    for flat in rng.choice(V.size, 10, replace=False):
        i, c = divmod(int(flat), 3)
        Vp, Vm = V.copy(), V.copy()
        Vp[i, c] += h
        Vm[i, c] -= h
        fd = (oracle.mnorm_objective(Vp, F, T, t)["loss"] - oracle.mnorm_objective(Vm, F, T, t)["loss"]) / (2 * h)
        assert abs(fd - g[i, c]) <= 1e-6 * np.abs(g).max() + 1e-12


def test_fairing_step_is_a_descent_step():
    """The Sobolev step -eta (M + tL)^-1 g is a descent direction (the operator is SPD), so a
    small step lowers the objective, and the step equals V - eta A^-1 g."""
    rng = np.random.default_rng(23)
    Vc, F = mg.icosphere(2)
    T = mg.radial_perturb(Vc, 0.03, rng)
    V = T.copy()
    t = 1e-2
    r = oracle.mnorm_objective(V, F, T, t)
    A = np.zeros((V.shape[0], V.shape[0]))
    for i in range(V.shape[0]):
        A[i, r["col"][r["rowptr"][i]:r["rowptr"][i + 1]]] = r["Aval"][r["rowptr"][i]:r["rowptr"][i + 1]]
    gs = np.linalg.solve(A, r["gV"])
    assert float(np.sum(r["gV"] * gs)) > 0.0
    eta = 1e-2 / np.abs(gs).max()
    V1, loss0 = oracle.fairing_step(V, F, T, t, eta)
    assert abs(loss0 - r["loss"]) <= 1e-15 * max(1.0, r["loss"])
    assert np.abs(V1 - (V - eta * gs)).max() <= 1e-12 * np.abs(V).max()
    assert oracle.mnorm_objective(V1, F, T, t)["loss"] < loss0


# ----------------------------------------------------------------------------- errors
def test_validation_errors():
    V, F = mg.octahedron()
    assert oracle.validate(F, 6) == oracle.OK
    bad = F.copy(); bad[0, 0] = 6
    assert oracle.validate(bad, 6) == oracle.ERR_INDEX
    bad = F.copy(); bad[0, 1] = bad[0, 0]
    assert oracle.validate(bad, 6) == oracle.ERR_DEGENERATE
    assert oracle.validate(F, 7) == oracle.ERR_ARG  # vertex 6 unused
    Vd = V.copy(); Vd[2] = Vd[0]  # collapse a face
    with pytest.raises(oracle.OracleError):
        oracle.face_geometry(Vd, F)
