"""Pins of the oracle's u-step of the ADMM scheme for regularized geodesic distances (formulation
eq. edelstein): b = m - D y + rho D z, then L u = b / (beta + rho) with u = 0 on the sources. What
fixes it independently of the oracle:

- the hat-function gradients reproduce linear functions exactly (the tangential part of a);
- D G equals the cotangent Laplacian of the C oracle (the P1 stiffness matrix), entry by entry;
- the u-step equals a sparse direct solve of the reduced system (scipy), and is 0 on the sources."""
import numpy as np
import pytest

import oracle

sp = pytest.importorskip("scipy.sparse")
spl = pytest.importorskip("scipy.sparse.linalg")


def _mesh(seed=0):
    from paper_2602_12105_gb300 import meshgen as mg
    V, F = mg.icosphere(2)
    return mg.radial_perturb(V, 0.05, np.random.default_rng(seed)), F


def test_hat_gradients_reproduce_linear_functions():
    V, F = _mesh()
    a = np.array([0.3, -1.2, 0.7])
    g = oracle.face_gradient(V, F, V @ a)
    P = V[F]
    N = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nh = N / np.linalg.norm(N, axis=1)[:, None]
    assert np.abs(g - (a[None, :] - (nh @ a)[:, None] * nh)).max() <= 1e-13


def test_divergence_of_gradient_is_the_cotangent_laplacian():
    V, F = _mesh(1)
    n = V.shape[0]
    rowptr, col, Lval = oracle.laplacian(V, F)
    L = np.zeros((n, n))
    for i in range(n):
        L[i, col[rowptr[i]:rowptr[i + 1]]] = Lval[rowptr[i]:rowptr[i + 1]]
    DG = np.stack([oracle.divergence(V, F, oracle.face_gradient(V, F, e)) for e in np.eye(n)], axis=1)
    assert np.abs(DG - L).max() <= 1e-13 * np.abs(L).max()


def test_u_step_is_the_reduced_sparse_solve():
    V, F = _mesh(2)
    n, m = V.shape[0], F.shape[0]
    rng = np.random.default_rng(3)
    y, z = rng.standard_normal((m, 3)), rng.standard_normal((m, 3))
    src = [0, 7, 40]
    rho, beta = 2.0, 0.5
    u = oracle.rgd_u_step(V, F, src, y, z, rho, beta)
    rowptr, col, Lval = oracle.laplacian(V, F)
    L = sp.csr_matrix((Lval, col, rowptr), shape=(n, n))
    b = (oracle.mass(V, F) - oracle.divergence(V, F, y) + rho * oracle.divergence(V, F, z)) / (beta + rho)
    free = np.setdiff1d(np.arange(n), src)
    ref = np.zeros(n)
    ref[free] = spl.spsolve(L[free][:, free].tocsc(), b[free])
    assert np.all(u[src] == 0.0)
    assert np.abs(u - ref).max() <= 1e-11 * np.abs(ref).max()
