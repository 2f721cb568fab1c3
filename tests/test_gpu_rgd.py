"""Parity of the regularized-geodesic ADMM u-step (ig_rgd_u_step) with the oracle's on the same
seeded inputs: perturbed icospheres and a bumpy grid of 14 tiles, several sources, random per-face
y and z. Both sides solve the source-constrained Laplacian, the GPU to 1e-13 and the oracle
directly (or by PCG to 1e-14 above 3000 vertices); with the reduced Laplacian's condition number
up to about 1e4 on these meshes the two agree to 1e-8 of max |u|. The sources stay exactly 0; the
mesh must be assembled again afterwards; bad arguments are reported."""
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


def _case(name):
    from paper_2602_12105_gb300 import meshgen as mg
    if name.startswith("ico"):
        V, F = mg.icosphere(int(name[3:]))
        return mg.radial_perturb(V, 0.05, np.random.default_rng(4)), F, [0, 7, 40]
    p = mg.config_grid(70, 50, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.05 * np.random.default_rng(5).standard_normal(V.shape[0])
    return V, p.F, [0, 1234, 3499]


@pytest.mark.parametrize("name", ["ico2", "ico3", "grid70x50"])
def test_u_step_matches_oracle(api, name):
    V, F, src = _case(name)
    n, m = V.shape[0], F.shape[0]
    rng = np.random.default_rng(6)
    y, z = rng.standard_normal((m, 3)), rng.standard_normal((m, 3))
    rho, beta = 2.0, 0.5
    ref = oracle.rgd_u_step(V, F, src, y, z, rho, beta)
    mesh = api.Mesh(_t(F, torch.int32), n)
    u, info = mesh.rgd_u_step(_t(V), src, _t(y), _t(z), rho, beta, opts=api.make_opts(rel_tol=1e-13), info=True)
    assert info["status"] == 0
    uh = u.cpu().numpy()
    assert np.all(uh[src] == 0.0)
    assert np.abs(uh - ref).max() <= 1e-8 * np.abs(ref).max(), (np.abs(uh - ref).max(), np.abs(ref).max())


def test_u_step_leaves_the_mesh_to_be_assembled(api):
    from paper_2602_12105_gb300 import _native as N
    V, F, src = _case("ico2")
    n, m = V.shape[0], F.shape[0]
    mesh = api.Mesh(_t(F, torch.int32), n)
    y = z = _t(np.zeros((m, 3)))
    mesh.rgd_u_step(_t(V), src, y, z, 1.0, 0.0)
    B = _t(np.random.default_rng(0).uniform(-1, 1, (n, 3)))
    with pytest.raises(N.IgError) as e:
        mesh.solve(B)
    assert e.value.status == N.IG_ERR_STATE
    # assembled again, the smoothing solve is the usual one
    mesh.assemble(_t(V), 1e-2)
    U = mesh.solve(B, opts=api.make_opts(rel_tol=1e-13)).cpu().numpy()
    rowptr, col, A, L, M = oracle.operator(V, F, 1e-2)
    ref = oracle.dense_cholesky_solve(rowptr, col, A, M[:, None] * B.cpu().numpy())
    assert np.abs(U - ref).max() <= 1e-10 * np.abs(ref).max()


def test_u_step_errors(api):
    from paper_2602_12105_gb300 import _native as N
    V, F, src = _case("ico2")
    n, m = V.shape[0], F.shape[0]
    mesh = api.Mesh(_t(F, torch.int32), n)
    y = z = _t(np.zeros((m, 3)))
    for bad_src, rho, beta in [([], 1.0, 0.0), ([n], 1.0, 0.0), ([-1], 1.0, 0.0), ([0], 0.0, 0.0),
                               ([0], -1.0, 1.0)]:
        with pytest.raises(N.IgError) as e:
            mesh.rgd_u_step(_t(V), bad_src, y, z, rho, beta)
        assert e.value.status == N.IG_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["ico2", "grid70x50"])
def test_u_step_gradients_match_oracle(api, name):
    V, F, src = _case(name)
    n, m = V.shape[0], F.shape[0]
    rng = np.random.default_rng(8)
    y, z, gu = rng.standard_normal((m, 3)), rng.standard_normal((m, 3)), rng.standard_normal(n)
    rho, beta = 2.0, 0.5
    rgV, rgy, rgz = oracle.rgd_u_step_vjp(V, F, src, y, z, rho, beta, gu)
    mesh = api.Mesh(_t(F, torch.int32), n)
    opts = api.make_opts(rel_tol=1e-13)
    u = mesh.rgd_u_step(_t(V), src, _t(y), _t(z), rho, beta, opts=opts)
    gV, gy, gz = mesh.rgd_u_step_vjp(_t(V), src, _t(y), _t(z), rho, beta, u, _t(gu), opts=opts)
    for got, ref in ((gV, rgV), (gy, rgy), (gz, rgz)):
        got = got.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (np.abs(got - ref).max(), np.abs(ref).max())


def test_u_step_autograd_matches_central_differences(api):
    """Through the autograd wrapper: d(gu . u)/dV and d/dy at sampled entries against central
    differences of GPU u-steps (step 1e-5; each solve stops at 1e-13)."""
    V, F, src = _case("ico2")
    n, m = V.shape[0], F.shape[0]
    rng = np.random.default_rng(9)
    y, z, gu = _t(rng.standard_normal((m, 3))), _t(rng.standard_normal((m, 3))), _t(rng.standard_normal(n))
    mesh = api.Mesh(_t(F, torch.int32), n)
    opts = api.make_opts(rel_tol=1e-13)
    Vt = _t(V).requires_grad_(True)
    yt = y.clone().requires_grad_(True)
    (api.rgd_u_step(mesh, Vt, yt, z, src, 2.0, 0.5, opts=opts) * gu).sum().backward()
    eps = 1e-5

    def loss(Vx, yx):
        return float((mesh.rgd_u_step(Vx, src, yx, z, 2.0, 0.5, opts=opts) * gu).sum())

    for i, d in [(1, 0), (9, 2), (77, 1)]:
        Vp, Vm = _t(V), _t(V)
        Vp[i, d] += eps
        Vm[i, d] -= eps
        fd = (loss(Vp, y) - loss(Vm, y)) / (2 * eps)
        assert abs(fd - float(Vt.grad[i, d])) <= 1e-6 * max(1.0, abs(fd)), (i, d, fd, float(Vt.grad[i, d]))
    for j, d in [(5, 1), (200, 2)]:
        yp, ym = y.clone(), y.clone()
        yp[j, d] += eps
        ym[j, d] -= eps
        fd = (loss(_t(V), yp) - loss(_t(V), ym)) / (2 * eps)
        assert abs(fd - float(yt.grad[j, d])) <= 1e-6 * max(1.0, abs(fd)), (j, d, fd, float(yt.grad[j, d]))


@pytest.mark.parametrize("name,iters", [("ico2", 30), ("grid70x50", 8)])
def test_admm_rounds_match_oracle(api, name, iters):
    """Rounds of the ADMM (u-step, projection z-step, over-relaxed dual step) from zero iterates,
    against the oracle's rounds: u, y and z within 1e-8 of their largest entries."""
    V, F, src = _case(name)
    n = V.shape[0]
    rho, beta, beta_k = 5.0, 0.1, 1.5
    ru, ry, rz, rst = oracle.rgd_admm(V, F, src, rho, beta, beta_k, iters)
    mesh = api.Mesh(_t(F, torch.int32), n)
    u, y, z, st = mesh.rgd_admm(_t(V), src, rho, beta, beta_k, iters, opts=api.make_opts(rel_tol=1e-13))
    for got, ref in ((u, ru), (y, ry), (z, rz)):
        got = got.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (np.abs(got - ref).max(), np.abs(ref).max())
    assert st["rounds"] == iters
    assert abs(st["primal"] - rst[1]) <= 1e-8 * max(1.0, rst[1])
    assert abs(st["dual"] - rst[2]) <= 1e-8 * max(1.0, rst[2])


def test_admm_stopping_and_rho_balancing_match_oracle(api):
    """With a tolerance and residual balancing, the GPU takes the same decisions as the oracle:
    the same number of rounds and the same final rho, and the same iterates."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(17, 17, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.0
    ru, ry, rz, rst = oracle.rgd_admm(V, p.F, [0], 1.0, 0.0, 1.0, 2000, tol=1e-3, adapt_rho=True)
    mesh = api.Mesh(_t(p.F, torch.int32), p.n)
    u, y, z, st = mesh.rgd_admm(_t(V), [0], 1.0, 0.0, 1.0, 2000, tol=1e-3, adapt_rho=True,
                                opts=api.make_opts(rel_tol=1e-13))
    assert st["rounds"] == rst[0] and st["rho"] == rst[3], (st, rst)
    assert st["primal"] <= 1e-3 and st["dual"] <= 1e-3
    assert np.abs(u.cpu().numpy() - ru).max() <= 1e-7 * np.abs(ru).max()


def test_admm_reports_unconverged_u_steps(api):
    """A u-step solve that stops at its iteration cap is reported (the worst status over the
    rounds: a warning and solve_status in Python, IG_ERR_NOT_CONVERGED from the C ABI), and the
    rounds still run and write their outputs."""
    from paper_2602_12105_gb300 import _native as N
    V, F, src = _case("grid70x50")
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    with pytest.warns(UserWarning, match="max_iter"):
        u, y, z, st = mesh.rgd_admm(_t(V), src, 5.0, 0.1, 1.0, 3, opts=api.make_opts(rel_tol=1e-13, max_iter=2))
    assert st["solve_status"] == N.IG_ERR_NOT_CONVERGED and st["rounds"] == 3
    assert bool(torch.isfinite(u).all())
    u, y, z, st = mesh.rgd_admm(_t(V), src, 5.0, 0.1, 1.0, 3, opts=api.make_opts(rel_tol=1e-10))
    assert st["solve_status"] == N.IG_OK


def test_admm_warm_start_skips_solves_near_the_fixed_point(api):
    """Started from converged iterates, every round after the first finds the previous u already
    within the solver tolerance and needs no solve; u stays the oracle's."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(17, 17, seed=0, t=1.0)
    V = p.V.copy()
    V[:, 2] = 0.0
    ru, ry, rz, rst = oracle.rgd_admm(V, p.F, [0], 1.0, 0.0, 1.0, 20000, tol=1e-12)
    mesh = api.Mesh(_t(p.F, torch.int32), p.n)
    u, y, z, st = mesh.rgd_admm(_t(V), [0], 1.0, 0.0, 1.0, 5, y=_t(ry), z=_t(rz), opts=api.make_opts(rel_tol=1e-8))
    assert st["warm_rounds_without_solve"] >= 3, st
    assert np.abs(u.cpu().numpy() - ru).max() <= 1e-7 * np.abs(ru).max()
