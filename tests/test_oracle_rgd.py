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


def test_u_step_gradients_match_central_differences():
    """d(gu . u)/d(V, y, z) through the u-step against central differences (step 1e-6), and the
    positional gradient is translation invariant (sum over vertices is 0)."""
    from paper_2602_12105_gb300 import meshgen as mg
    V, F = mg.icosphere(1)
    V = mg.radial_perturb(V, 0.05, np.random.default_rng(0))
    n, m = V.shape[0], F.shape[0]
    rng = np.random.default_rng(1)
    y, z, gu = rng.standard_normal((m, 3)), rng.standard_normal((m, 3)), rng.standard_normal(n)
    src, rho, beta = [0, 5], 2.0, 0.5
    gV, gy, gz = oracle.rgd_u_step_vjp(V, F, src, y, z, rho, beta, gu)

    def loss(Vx, yx, zx):
        return float(gu @ oracle.rgd_u_step(Vx, F, src, yx, zx, rho, beta))

    eps = 1e-6
    for i, d in [(1, 0), (7, 2), (20, 1), (41, 2)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[i, d] += eps
        Vm[i, d] -= eps
        fd = (loss(Vp, y, z) - loss(Vm, y, z)) / (2 * eps)
        assert abs(fd - gV[i, d]) <= 1e-7 * max(1.0, abs(fd)), (i, d, fd, gV[i, d])
    for j, d in [(3, 1), (50, 0)]:
        for which, g in (("y", gy), ("z", gz)):
            p_, m_ = (y.copy(), y.copy()) if which == "y" else (z.copy(), z.copy())
            p_[j, d] += eps
            m_[j, d] -= eps
            fd = ((loss(V, p_, z) - loss(V, m_, z)) if which == "y" else (loss(V, y, p_) - loss(V, y, m_))) / (2 * eps)
            assert abs(fd - g[j, d]) <= 1e-7 * max(1.0, abs(fd)), (which, j, d, fd, g[j, d])
    assert np.abs(gV.sum(axis=0)).max() <= 1e-10 * np.abs(gV).max()


def test_admm_approaches_the_euclidean_distance_on_a_flat_square():
    """With beta = 0 the problem is the geodesic distance (max m^T u under |G u| <= 1, u = 0 at
    the source); on a flat convex square that is the Euclidean distance from the source corner.
    300 rounds on a 17 x 17 grid reach it within the discretisation error (2.4% of the largest
    distance here), satisfy the gradient bound to 0.2%, and stay 0 at the source."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(17, 17, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.0
    u, y, z, stats = oracle.rgd_admm(V, p.F, [0], rho=10.0, beta=0.0, beta_k=1.0, iters=300)
    d = np.linalg.norm(V - V[0], axis=1)
    assert u[0] == 0.0
    assert np.abs(u - d).max() <= 0.03 * d.max()
    assert np.linalg.norm(oracle.face_gradient(V, p.F, u), axis=1).max() <= 1.005
    assert stats[0] == 300 and stats[1] <= 5e-3


def test_admm_stops_on_its_residuals_with_rho_balancing():
    """With a tolerance the rounds stop as soon as both residuals meet it, and residual balancing
    changes rho only by factors of 2; the result still approaches the distance."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(17, 17, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.0
    u, y, z, (rounds, primal, dual, rho) = oracle.rgd_admm(V, p.F, [0], rho=1.0, beta=0.0, beta_k=1.0, iters=2000,
                                                          tol=1e-3, adapt_rho=True)
    assert rounds < 2000 and primal <= 1e-3 and dual <= 1e-3
    assert np.log2(rho) == round(np.log2(rho))
    d = np.linalg.norm(V - V[0], axis=1)
    assert np.abs(u - d).max() <= 0.04 * d.max()


def _bumpy_grid(nx, ny, seed=0, amp=0.05):
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(nx, ny, seed=seed, t=1.0)
    V = p.V.copy()
    V[:, 2] = amp * np.random.default_rng(seed + 7).standard_normal(p.n)
    return V, p.F


def test_round_vjp_matches_central_differences():
    """The VJP of one ADMM round against central differences of the round in y, z and V, at
    iterates where some faces are projected onto the unit ball and others are not."""
    V, F = _bumpy_grid(6, 5, seed=1)
    m = F.shape[0]
    rng = np.random.default_rng(3)
    rho, beta, bk = 1.7, 0.3, 1.4
    y = 1.5 * rng.standard_normal((m, 3))
    z = 0.4 * rng.standard_normal((m, 3))
    wy, wz = rng.standard_normal((m, 3)), rng.standard_normal((m, 3))
    yn, zn, u = oracle.rgd_round(V, F, [0, 7], y, z, rho, beta, bk)
    a = np.linalg.norm(y / rho + oracle.face_gradient(V, F, u), axis=1)
    assert (a > 1.0).sum() >= 5 and (a < 1.0).sum() >= 5
    gV, gy, gz = oracle.rgd_round_vjp(V, F, [0, 7], y, z, rho, beta, bk, wy, wz)

    def ell(V_, y_, z_):
        yn_, zn_, _ = oracle.rgd_round(V_, F, [0, 7], y_, z_, rho, beta, bk)
        return np.sum(wy * yn_) + np.sum(wz * zn_)

    eps = 1e-6
    for _ in range(2):
        dV, dy, dz = rng.standard_normal(V.shape), rng.standard_normal(y.shape), rng.standard_normal(z.shape)
        for want, fd in ((np.sum(gV * dV), ell(V + eps * dV, y, z) - ell(V - eps * dV, y, z)),
                         (np.sum(gy * dy), ell(V, y + eps * dy, z) - ell(V, y - eps * dy, z)),
                         (np.sum(gz * dz), ell(V, y, z + eps * dz) - ell(V, y, z - eps * dz))):
            assert abs(fd / (2 * eps) - want) <= 1e-6 * max(1.0, abs(want)), (fd / (2 * eps), want)


def test_face_gradient_vjp_matches_central_differences():
    V, F = _bumpy_grid(5, 4, seed=2)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(V.shape[0])
    W = rng.standard_normal((F.shape[0], 3))
    g = oracle.face_gradient_vjp(V, F, u, W)
    dV = rng.standard_normal(V.shape)
    eps = 1e-6
    fd = (np.sum(W * oracle.face_gradient(V + eps * dV, F, u)) - np.sum(W * oracle.face_gradient(V - eps * dV, F, u)))
    assert abs(fd / (2 * eps) - np.sum(g * dV)) <= 1e-7 * max(1.0, abs(np.sum(g * dV)))


def _converged(V, F, rho, beta, bk, y=None, z=None):
    u, y, z, st = oracle.rgd_admm(V, F, [0], rho, beta, bk, 20000, y=y, z=z, tol=1e-13)
    assert st[0] < 20000, st
    return u, y, z


def test_admm_vjp_matches_central_differences_of_the_converged_distance():
    """The fixed-point VJP of the ADMM against central differences of <c, u*(V)> with u* the
    distance the rounds converge to (tol 1e-13 on both residuals)."""
    V, F = _bumpy_grid(6, 5, seed=0)
    rho, beta, bk = 2.0, 0.5, 1.0
    u, y, z = _converged(V, F, rho, beta, bk)
    rng = np.random.default_rng(11)
    c = rng.standard_normal(V.shape[0])
    gV, wy, wz = oracle.rgd_admm_vjp(V, F, [0], y, z, rho, beta, bk, c)
    dV = rng.standard_normal(V.shape)
    dV[:, 2] *= 0.2
    eps = 1e-5
    up = _converged(V + eps * dV, F, rho, beta, bk, y, z)[0]
    um = _converged(V - eps * dV, F, rho, beta, bk, y, z)[0]
    fd = np.sum(c * (up - um)) / (2 * eps)
    want = np.sum(gV * dV)
    assert abs(fd - want) <= 1e-5 * max(1.0, abs(want)), (fd, want)
    # a planted mistake: the u-step's own gradient alone (no fixed-point solve) is far off
    gV0, _, _ = oracle.rgd_u_step_vjp(V, F, [0], y, z, rho, beta, c)
    assert abs(np.sum(gV0 * dV) - fd) > 1e-2 * abs(fd)


def test_admm_vjp_does_not_depend_on_rho_and_is_translation_invariant():
    """u* solves the regularized problem (formulation eq. edelstein), which has no rho: the
    fixed points reached with two penalties give the same u* and the same dl/dV. And u* does not
    change when the mesh is translated, so the rows of dl/dV sum to zero."""
    V, F = _bumpy_grid(5, 5, seed=4)
    beta, bk = 0.5, 1.0
    c = np.random.default_rng(2).standard_normal(V.shape[0])
    u1, y1, z1 = _converged(V, F, 2.0, beta, bk)
    u2, y2, z2 = _converged(V, F, 5.0, beta, bk)
    assert np.abs(u1 - u2).max() <= 1e-10
    g1 = oracle.rgd_admm_vjp(V, F, [0], y1, z1, 2.0, beta, bk, c)[0]
    g2 = oracle.rgd_admm_vjp(V, F, [0], y2, z2, 5.0, beta, bk, c)[0]
    assert np.abs(g1 - g2).max() <= 1e-8 * np.abs(g1).max()
    assert np.abs(g1.sum(axis=0)).max() <= 1e-10 * np.abs(g1).max()


def test_over_relaxation_changes_the_path_not_the_fixed_point():
    """The dual step's over-relaxation term rho ((beta_k - 1)(z_old - G u)) changes the path of the
    rounds but not their fixed points: at a fixed point z_new = z_old = z and y_new = y, so the dual
    step reads rho beta_k (G u - z) = 0, i.e. G u = z, and the z-step z = P(y / rho + G u); neither
    condition involves beta_k (beta_k != 0). The converged distance and the gradient through the
    fixed point must therefore agree at beta_k = 1 and 1.5, while the paths differ. A sign error in
    the term moves the fixed point (to z = beta_k G u / (2 - beta_k) with the sign of the
    (1 - beta_k) z_old part flipped), which this catches at beta_k = 1.5."""
    V, F = _bumpy_grid(5, 5, seed=6)
    rho, beta = 2.0, 0.5
    c = np.random.default_rng(9).standard_normal(V.shape[0])
    u1, y1, z1 = _converged(V, F, rho, beta, 1.0)
    u15, y15, z15 = _converged(V, F, rho, beta, 1.5)
    assert np.abs(u1 - u15).max() <= 1e-10 * np.abs(u1).max()
    assert np.abs(z1 - z15).max() <= 1e-9
    g1 = oracle.rgd_admm_vjp(V, F, [0], y1, z1, rho, beta, 1.0, c)[0]
    g15 = oracle.rgd_admm_vjp(V, F, [0], y15, z15, rho, beta, 1.5, c)[0]
    assert np.abs(g1 - g15).max() <= 1e-10 * np.abs(g1).max()
    # the paths differ: after the same few rounds from the same start the iterates are apart
    a = oracle.rgd_admm(V, F, [0], rho, beta, 1.0, 5)
    b = oracle.rgd_admm(V, F, [0], rho, beta, 1.5, 5)
    assert np.abs(a[1] - b[1]).max() > 1e-3
