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
