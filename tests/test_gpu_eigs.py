"""Parity of the eigenvector iteration (ig_eigs: shift-invert subspace iteration of Eq. eigiter,
§5) with the oracle's, step for step from the same start basis: the GPU's U and eigenvalues
against the oracle's after the same number of steps (the two sides solve each step to 1e-13 and
exactly, so they agree to about 1e-12; the test allows 1e-9), on meshes of one, several and many
256-row tiles, converged and not; repeat calls give the same bits; bad arguments and dependent
start columns are reported."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12105_gb300 import api as _api
    return _api


def _t(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def _flat_grid(nx, ny):
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(nx, ny, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.0
    return V, p.F


def _sphere(level, seed):
    from paper_2602_12105_gb300 import meshgen as mg
    V, F = mg.icosphere(level)
    V = V * (1.0 + 0.02 * np.random.default_rng(seed).standard_normal((V.shape[0], 1)))
    return V, F


def _case(name):
    if name == "grid13x9":
        V, F = _flat_grid(13, 9)
        return V, F, 1.0, 4, 40
    if name == "ico3":
        V, F = _sphere(3, 5)
        return V, F, 0.05, 3, 25
    if name == "grid70x50":
        V, F = _flat_grid(70, 50)
        return V, F, 2.0, 4, 12
    raise KeyError(name)


@pytest.mark.parametrize("name", ["grid13x9", "ico3", "grid70x50"])
def test_eigs_matches_oracle_step_for_step(api, name):
    V, F, t, k, iters = _case(name)
    n = V.shape[0]
    U0 = np.random.default_rng(9).uniform(-1, 1, (n, k))
    Uo, lamo = oracle.subspace_iteration(V, F, t, U0, iters)
    mesh = api.Mesh(_t(F, torch.int32), n)
    mesh.assemble(_t(V), t)
    U, lam = mesh.eigs(_t(U0), iters, opts=api.make_opts(rel_tol=1e-13))
    Uh = U.cpu().numpy()
    assert np.abs(Uh - Uo).max() <= 1e-9, np.abs(Uh - Uo).max()
    assert np.abs(lam.numpy() - lamo).max() <= 1e-9 * max(1.0, float(np.abs(lamo).max()))
    # M-orthonormal columns
    M = mesh.mass().cpu().numpy()
    assert np.abs(Uh.T @ (M[:, None] * Uh) - np.eye(k)).max() <= 1e-12
    # the same bits on a second call
    U2, lam2 = mesh.eigs(_t(U0), iters, opts=api.make_opts(rel_tol=1e-13))
    assert torch.equal(U, U2) and torch.equal(lam, lam2)


def test_eigs_converges_to_the_dense_pencil(api):
    """After enough steps the result is the lowest eigenvectors of (L, M), the constant one first."""
    sl = pytest.importorskip("scipy.linalg")
    V, F = _flat_grid(15, 7)
    n = V.shape[0]
    rowptr, col, _, Lval, M = oracle.operator(V, F, 1.0)
    Ld = np.zeros((n, n))
    for i in range(n):
        Ld[i, col[rowptr[i]:rowptr[i + 1]]] = Lval[rowptr[i]:rowptr[i + 1]]
    w, X = sl.eigh(Ld, np.diag(M))
    mesh = api.Mesh(_t(F, torch.int32), n)
    mesh.assemble(_t(V), 1.0)
    U, lam = mesh.eigs(_t(np.random.default_rng(2).uniform(-1, 1, (n, 4))), 200,
                       opts=api.make_opts(rel_tol=1e-13))
    assert np.abs(lam.numpy() - w[:4]).max() <= 1e-9 * w[3]
    assert np.abs(U.cpu().numpy() - oracle.canonical_sign(X[:, :4])).max() <= 1e-7


def test_eigs_errors(api):
    from paper_2602_12105_gb300 import _native as N
    V, F = _flat_grid(13, 9)
    n = V.shape[0]
    mesh = api.Mesh(_t(F, torch.int32), n)
    with pytest.raises(N.IgError) as e:
        mesh.eigs(_t(np.ones((n, 2))), 3)
    assert e.value.status == N.IG_ERR_STATE
    mesh.assemble(_t(V), 1.0)
    with pytest.raises(N.IgError) as e:
        mesh.eigs(_t(np.ones((n, 5))), 3)
    assert e.value.status == N.IG_ERR_INVALID_ARG
    with pytest.raises(N.IgError) as e:
        mesh.eigs(_t(np.ones((n, 2))), 0)
    assert e.value.status == N.IG_ERR_INVALID_ARG
    # two equal start columns: the Gram matrix is singular
    U0 = np.random.default_rng(0).uniform(-1, 1, (n, 3))
    U0[:, 2] = U0[:, 1]
    with pytest.raises(N.IgError) as e:
        mesh.eigs(_t(U0), 2)
    assert e.value.status == N.IG_ERR_NONFINITE
    # the mesh still solves afterwards
    U, lam = mesh.eigs(_t(np.random.default_rng(1).uniform(-1, 1, (n, 2))), 5)
    assert np.isfinite(U.cpu().numpy()).all()


def _bumpy_grid(nx=10, ny=7, seed=5):
    V, F = _flat_grid(nx, ny)
    V[:, 2] = 0.05 * np.random.default_rng(seed).standard_normal(V.shape[0])
    return V, F


@pytest.mark.parametrize("nx,ny,k,t", [(10, 7, 3, 1.0), (63, 50, 4, 0.5)])
def test_eigs_vjp_matches_oracle(api, nx, ny, k, t):
    """dl/dV through the fixed point, with the same converged U and cotangent on both sides
    (3500 rows in the second case: 14 tiles, the oracle solving by PCG)."""
    V, F = _bumpy_grid(nx, ny)
    n = V.shape[0]
    U0 = np.random.default_rng(1).uniform(-1, 1, (n, k))
    iters = 150 if n < 1000 else 60
    U, _ = oracle.subspace_iteration(V, F, t, U0, iters)
    c = np.random.default_rng(2).standard_normal((n, k))
    ref = oracle.eigs_vjp(V, F, t, U, c, iters)
    mesh = api.Mesh(_t(F, torch.int32), n)
    mesh.assemble(_t(V), t)
    g = mesh.eigs_vjp(_t(V), _t(U), _t(c), iters, opts=api.make_opts(rel_tol=1e-13)).cpu().numpy()
    assert np.abs(g - ref).max() <= 1e-8 * np.abs(ref).max(), (np.abs(g - ref).max(), np.abs(ref).max())


def test_eigs_autograd_matches_central_differences(api):
    """Through the autograd wrapper: d(sum c * U)/dV against central differences of the
    converged GPU eigenvectors (step 1e-5: each solve stops at 1e-13, so smaller steps would
    see that rounding) at sampled coordinates."""
    V, F = _bumpy_grid()
    n, k = V.shape[0], 3
    U0 = _t(np.random.default_rng(1).uniform(-1, 1, (n, k)))
    c = _t(np.random.default_rng(2).standard_normal((n, k)))
    mesh = api.Mesh(_t(F, torch.int32), n)
    opts = api.make_opts(rel_tol=1e-13)
    Vt = _t(V).requires_grad_(True)
    U, lam = api.eigs(mesh, Vt, 1.0, U0, 150, opts=opts)
    (U * c).sum().backward()
    g = Vt.grad.cpu().numpy()
    eps = 1e-5
    for i, d in [(0, 2), (13, 0), (25, 2), (66, 2)]:
        vals = []
        for sgn in (1.0, -1.0):
            Vp = V.copy()
            Vp[i, d] += sgn * eps
            mesh.assemble(_t(Vp), 1.0)
            Up, _ = mesh.eigs(U0, 150, opts=opts)
            vals.append(float((Up * c).sum()))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - g[i, d]) <= 1e-6 * max(1.0, abs(fd)), (i, d, fd, g[i, d])
