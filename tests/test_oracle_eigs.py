"""Pins of the oracle's shift-invert subspace iteration (Eq. eigiter, §5), the forward half of the
eigenvector row: each step solves (M + tL) Y = M U with the smoothing operator and M-orthonormalizes
Y (Q, with a canonical sign per column). What fixes its results independently of the oracle:

- dense generalized eigendecomposition of the pencil (L, M) (scipy.linalg.eigh) on small meshes;
- the constant vector is an exact eigenvector with eigenvalue 0 (L has zero row sums);
- U^T M U = I, and a converged U is a fixed point of the step;
- the canonical sign rule on hand-made columns."""
import numpy as np
import pytest

import oracle

sl = pytest.importorskip("scipy.linalg")


def _flat_grid(nx, ny):
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(nx, ny, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.0
    return V, p.F


def _dense(rowptr, col, val, n):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, col[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
    return D


def test_canonical_sign_rule():
    U = np.array([[0.5, 0.2], [-1.0, 0.3], [1.0, -0.3]])
    S = oracle.canonical_sign(U)
    # column 0: the first entry of largest magnitude is -1 (row 1): flipped
    assert np.array_equal(S[:, 0], [-0.5, 1.0, -1.0])
    # column 1: the largest magnitude 0.3 is reached first at row 1 (+0.3): kept
    assert np.array_equal(S[:, 1], U[:, 1])


@pytest.mark.parametrize("nx,ny", [(13, 9), (15, 7), (10, 7)])
def test_subspace_iteration_matches_dense_pencil(nx, ny):
    """Aspect ratios away from 1 keep the four lowest eigenvalues apart, so the subspace
    iteration converges to the individual eigenvectors; they must equal the dense generalized
    eigenvectors of (L, M) with the same canonical signs."""
    V, F = _flat_grid(nx, ny)
    n = V.shape[0]
    rowptr, col, _, Lval, M = oracle.operator(V, F, 1.0)
    w, X = sl.eigh(_dense(rowptr, col, Lval, n), np.diag(M))
    U0 = np.random.default_rng(1).uniform(-1, 1, (n, 4))
    U, lam = oracle.subspace_iteration(V, F, 1.0, U0, 200)
    assert np.abs(lam - w[:4]).max() <= 1e-10 * max(1.0, w[3])
    assert np.abs(U - oracle.canonical_sign(X[:, :4])).max() <= 1e-8


def test_constant_mode_orthonormality_and_fixed_point():
    from paper_2602_12105_gb300 import meshgen as mg
    V, F = mg.icosphere(2)
    V = V * (1.0 + 0.02 * np.random.default_rng(3).standard_normal((V.shape[0], 1)))
    n = V.shape[0]
    _, _, _, _, M = oracle.operator(V, F, 0.5)
    U0 = np.random.default_rng(4).uniform(-1, 1, (n, 3))
    U, lam = oracle.subspace_iteration(V, F, 0.5, U0, 60)
    # the constant vector, M-normalized, with a positive sign; eigenvalue 0
    assert np.abs(U[:, 0] - 1.0 / np.sqrt(M.sum())).max() <= 1e-10
    assert abs(lam[0]) <= 1e-10
    assert np.abs(U.T @ (M[:, None] * U) - np.eye(3)).max() <= 1e-12
    # a converged U is (to rounding) a fixed point of the step
    U2, _ = oracle.subspace_iteration(V, F, 0.5, U, 1)
    assert np.abs(U2[:, 0] - U[:, 0]).max() <= 1e-12


def _bumpy_grid():
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(10, 7, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.05 * np.random.default_rng(5).standard_normal(V.shape[0])
    return V, p.F


def test_eigs_vjp_matches_central_differences():
    """d(sum c * U*)/dV through the converged eigenvectors, against central differences of
    fully converged subspace iterations (step 1e-6) at sampled coordinates."""
    V, F = _bumpy_grid()
    n, k = V.shape[0], 3
    U0 = np.random.default_rng(1).uniform(-1, 1, (n, k))
    c = np.random.default_rng(2).standard_normal((n, k))

    def converged(Vx):
        return oracle.subspace_iteration(Vx, F, 1.0, U0, 150)[0]

    U = converged(V)
    g = oracle.eigs_vjp(V, F, 1.0, U, c, 150)
    eps = 1e-6
    for i, d in [(0, 2), (13, 0), (25, 2), (40, 1), (66, 2), (69, 0)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[i, d] += eps
        Vm[i, d] -= eps
        fd = (np.sum(c * converged(Vp)) - np.sum(c * converged(Vm))) / (2 * eps)
        assert abs(fd - g[i, d]) <= 1e-6 * max(1.0, abs(fd)), (i, d, fd, g[i, d])


def test_eigs_vjp_does_not_depend_on_the_shift():
    """The converged eigenvectors do not depend on t, so neither may their gradient, although
    every step of the adjoint uses the shifted operator."""
    V, F = _bumpy_grid()
    n, k = V.shape[0], 3
    U = oracle.subspace_iteration(V, F, 1.0, np.random.default_rng(1).uniform(-1, 1, (n, k)), 150)[0]
    c = np.random.default_rng(3).standard_normal((n, k))
    g1 = oracle.eigs_vjp(V, F, 1.0, U, c, 150)
    g2 = oracle.eigs_vjp(V, F, 0.3, U, c, 400)
    assert np.abs(g1 - g2).max() <= 1e-9 * np.abs(g1).max()
