"""Edge cases of the path: the smallest mesh (one triangle), empty inputs, tile-boundary sizes
(rows a multiple of the tile size, and one more), right-hand sides with some zero columns, k = 1
and k = 4 batches, and a batch of one mesh — each against the oracle or the single-mesh result."""
import numpy as np
import pytest

import oracle
from gpu_util import rel2

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


def _oracle_solve(V, F, t, B):
    rowptr, col, A, L, M = oracle.operator(V, F, t)
    return oracle.dense_cholesky_solve(rowptr, col, A, M[:, None] * B)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_triangle(api, precision):
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.1]])
    F = np.array([[0, 1, 2]], dtype=np.int32)
    B = np.array([[1.0, -2.0, 0.5], [0.0, 1.0, 2.0], [-1.0, 0.3, 0.0]])
    mesh = api.Mesh(_t(F, torch.int32), 3)
    mesh.assemble(_t(V), 0.3, precision)
    U, info = mesh.solve(_t(B), opts=api.make_opts(rel_tol=1e-14), info=True)
    assert info["status"] == 0
    assert rel2(U.cpu().numpy(), _oracle_solve(V, F, 0.3, B)) <= 1e-12


def test_empty_inputs_are_rejected(api):
    from paper_2602_12105_gb300 import _native as N
    with pytest.raises((N.IgError, ValueError)):
        api.Mesh(torch.zeros((0, 3), dtype=torch.int32, device=DEV), 0)
    with pytest.raises((N.IgError, ValueError)):
        api.Mesh(torch.zeros((0, 3), dtype=torch.int32, device=DEV), 5)


@pytest.mark.parametrize("nx,ny", [(64, 16), (64, 17), (32, 33)])
def test_tile_boundary_sizes(api, nx, ny):
    """Small meshes get 256-row tiles: 1024 rows fill four tiles exactly; 1088 and 1056 rows end
    in a ragged fifth tile."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(nx, ny, seed=5, t=2e-3)
    mesh = api.Mesh(_t(p.F, torch.int32), p.n)
    mesh.assemble(_t(p.V), p.t)
    U = mesh.solve(_t(p.B), opts=api.make_opts(rel_tol=1e-14))
    assert rel2(U.cpu().numpy(), _oracle_solve(p.V, p.F, p.t, p.B)) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_some_zero_columns(api, precision):
    """Zero columns converge at once to zero; the other columns are unaffected."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(40, 30, seed=6, t=1e-3)
    B = p.B.copy()
    B[:, 1] = 0.0
    mesh = api.Mesh(_t(p.F, torch.int32), p.n)
    mesh.assemble(_t(p.V), p.t, precision)
    U, info = mesh.solve(_t(B), opts=api.make_opts(rel_tol=1e-13), info=True)
    assert info["status"] == 0
    Uh = U.cpu().numpy()
    assert float(np.abs(Uh[:, 1]).max()) == 0.0
    ref = _oracle_solve(p.V, p.F, p.t, B)
    assert rel2(Uh[:, [0, 2]], ref[:, [0, 2]]) <= 1e-10


@pytest.mark.parametrize("k", [1, 4])
def test_batch_column_counts_and_single_mesh_batch(api, k):
    from paper_2602_12105_gb300 import meshgen as mg
    rng = np.random.default_rng(7 + k)
    probs = [mg.config_grid(30, 20, seed=8, t=1e-3), mg.problem_icosphere(3, 0.02, 3e-3, rng)]
    meshes = [api.Mesh(_t(q.F, torch.int32), q.n) for q in probs]
    Bs = [_t(rng.uniform(-1, 1, (q.n, k))) for q in probs]
    opts = api.make_opts(rel_tol=1e-13)
    for sub in (meshes, meshes[:1]):
        batch = api.Batch(sub)
        batch.assemble([_t(q.V) for q in probs[:len(sub)]], [q.t for q in probs[:len(sub)]])
        Us = batch.solve(Bs[:len(sub)], opts=opts)
        for q, U, B in zip(probs, Us, Bs):
            ref = _oracle_solve(q.V, q.F, q.t, B.cpu().numpy())
            assert rel2(U.cpu().numpy(), ref) <= 1e-10
        batch.close()


@pytest.mark.parametrize("max_iter", [1, 2, 3, 7])
def test_iteration_cap_is_exact_on_a_multi_tile_mesh(api, max_iter):
    """A solve that cannot meet its tolerance stops after exactly max_iter iterations with
    NOT_CONVERGED: in the graph loop (two iterations per pass of its WHILE body, so an odd cap ends
    inside a pass, and the completing CTA decides from the counter and cap it read at entry) and
    in the host loop, with the same bits. The iterate is the oracle's Jacobi-PCG iterate after as
    many iterations (the same algorithm in FP64; only the order of the sums differs)."""
    from paper_2602_12105_gb300 import _native as N
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(160, 150, seed=5)  # 24,000 rows: many FP64 tiles, the multi-CTA loop
    B = np.random.default_rng(6).uniform(-1, 1, (p.n, 3))
    mesh = api.Mesh(_t(p.F, torch.int32), p.n)
    mesh.assemble(_t(p.V), p.t)
    out = {}
    for launch in ("graph", "host"):
        U, info = mesh.solve(_t(B), opts=api.make_opts(rel_tol=1e-300, max_iter=max_iter, launch=launch), info=True)
        assert info["status"] == N.IG_ERR_NOT_CONVERGED and info["iterations"] == max_iter, (launch, info)
        out[launch] = U.cpu().numpy()
    assert np.array_equal(out["graph"], out["host"])
    rowptr, col, A, L, M = oracle.operator(p.V, p.F, p.t)
    X, iters, _, st = oracle.pcg_solve(rowptr, col, A, M[:, None] * B, tol=1e-300, max_iter=max_iter)
    assert st == oracle.ERR_NOT_CONVERGED and list(iters) == [max_iter] * 3
    assert rel2(out["graph"], X) <= 1e-12
