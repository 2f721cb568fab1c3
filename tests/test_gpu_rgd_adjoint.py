"""Parity of the fixed-point adjoint of the regularized-geodesic ADMM (ig_rgd_admm_vjp) with the
oracle's on the same seeded inputs. The oracle forms J^T of one round column by column and solves
(I - J^T) w = (gy0, gz0) densely; the GPU solves the same system by restarted GMRES (to 1e-12, with
each product through one constrained Laplacian solve to 1e-13). Both take the fixed point (y*, z*)
the oracle's rounds converged to. On larger meshes, where the dense solve is out of reach, the
gradient is checked against central differences of the GPU's own converged distance, and against
translation invariance."""
import warnings

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


def _bumpy_grid(nx, ny, seed=0, amp=0.05):
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_grid(nx, ny, seed=seed, t=1.0)
    V = p.V.copy()
    V[:, 2] = amp * np.random.default_rng(seed + 7).standard_normal(p.n)
    return V, p.F


@pytest.fixture(scope="module")
def small_case():
    V, F = _bumpy_grid(7, 6, seed=0)
    rho, beta, bk = 2.0, 0.5, 1.3
    u, y, z, st = oracle.rgd_admm(V, F, [0, 5], rho, beta, bk, 20000, tol=1e-13)
    assert st[0] < 20000
    c = np.random.default_rng(11).standard_normal(V.shape[0])
    gV, wy, wz = oracle.rgd_admm_vjp(V, F, [0, 5], y, z, rho, beta, bk, c)
    return dict(V=V, F=F, rho=rho, beta=beta, bk=bk, y=y, z=z, c=c, gV=gV, wy=wy, wz=wz)


@pytest.mark.parametrize("restart", [100, 20])
def test_admm_vjp_matches_oracle(api, small_case, restart):
    k = small_case
    V, F = k["V"], k["F"]
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    gV, info, w = mesh.rgd_admm_vjp(_t(V), [0, 5], _t(k["y"]), _t(k["z"]), k["rho"], k["beta"], k["bk"], _t(k["c"]),
                                    restart=restart, max_iter=2000, tol=1e-12, strict=True, return_w=True,
                                    opts=api.make_opts(rel_tol=1e-13))
    assert info["converged"] and info["rel_resid"] <= 1e-12
    gV = gV.cpu().numpy()
    scale = np.abs(k["gV"]).max()
    assert np.abs(gV - k["gV"]).max() <= 1e-8 * scale, (np.abs(gV - k["gV"]).max(), scale)
    w = w.cpu().numpy()
    for got, ref in ((w[0], k["wy"]), (w[1], k["wz"])):
        assert np.abs(got - ref).max() <= 1e-8 * max(np.abs(k["wy"]).max(), np.abs(k["wz"]).max())


def test_admm_vjp_reports_a_gmres_that_stops_early(api, small_case):
    k = small_case
    V, F = k["V"], k["F"]
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    args = (_t(V), [0, 5], _t(k["y"]), _t(k["z"]), k["rho"], k["beta"], k["bk"], _t(k["c"]))
    with pytest.warns(RuntimeWarning):
        gV, info = mesh.rgd_admm_vjp(*args, restart=3, max_iter=2, tol=1e-12)
    assert info["iterations"] == 2 and not info["converged"] and info["rel_resid"] > 1e-12
    assert torch.isfinite(gV).all()
    with pytest.raises(Exception):
        mesh.rgd_admm_vjp(*args, restart=3, max_iter=2, tol=1e-12, strict=True)
    with pytest.raises(Exception):
        mesh.rgd_admm_vjp(*args, restart=0)
    # gu = 0: the adjoint is 0 and GMRES stops at once
    gV, info = mesh.rgd_admm_vjp(*args[:7], torch.zeros(V.shape[0], dtype=torch.float64, device=DEV), strict=True)
    assert info["iterations"] == 0 and info["converged"]
    assert float(gV.abs().max()) == 0.0


def test_admm_gradient_matches_central_differences(api, small_case):
    """The autograd gradient of <c, u*(V)> through rgd_distance against central differences of the
    GPU's own converged distance (rounds warm-started from the fixed point, to 1e-13)."""
    k = small_case
    V, F = k["V"], k["F"]
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    opts = api.make_opts(rel_tol=1e-13)
    c = _t(k["c"])
    Vt = _t(V).requires_grad_(True)
    u = api.rgd_distance(mesh, Vt, [0, 5], k["rho"], k["beta"], k["bk"], max_rounds=20000, tol=1e-13,
                         gmres=dict(restart=50, max_iter=2000, tol=1e-12, strict=True), opts=opts)
    (g,) = torch.autograd.grad((c * u).sum(), Vt)
    g = g.detach().cpu().numpy()
    assert np.abs(g - k["gV"]).max() <= 1e-7 * np.abs(k["gV"]).max()
    dV = np.random.default_rng(2).standard_normal(V.shape)
    dV[:, 2] *= 0.2
    eps = 1e-5

    def dist(Vp):
        up, _, _, st = mesh.rgd_admm(_t(Vp), [0, 5], k["rho"], k["beta"], k["bk"], 20000, tol=1e-13,
                                     y=_t(k["y"]), z=_t(k["z"]), opts=opts)
        assert st["rounds"] < 20000
        return up

    fd = float((c * (dist(V + eps * dV) - dist(V - eps * dV))).sum()) / (2 * eps)
    want = float(np.sum(g * dV))
    assert abs(fd - want) <= 1e-5 * max(1.0, abs(want)), (fd, want)


def test_admm_vjp_solves_the_oracles_adjoint_system_on_a_larger_mesh(api):
    """A 40 x 40 bumpy grid (1600 vertices, 3042 faces: 18 chunks of the GMRES inner products and
    several tiles of every row and face kernel), at the iterates of 200 rounds (the adjoint system
    is defined at any (y, z)). The oracle checks the GPU's w in its own equations: one product of
    the oracle's round VJP gives the residual of (I - J^T) w = (gy0, gz0), which must match the
    residual GMRES reports (so its estimate is the true one), and the gradient
    gV0 + (dT/dV)^T w; the rows of dl/dV sum to zero (translation invariance)."""
    V, F = _bumpy_grid(40, 40, seed=3)
    m = F.shape[0]
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    opts = api.make_opts(rel_tol=1e-13)
    rho, beta, bk, src = 2.0, 0.5, 1.0, [0, 817]
    _, y, z, _ = mesh.rgd_admm(_t(V), src, rho, beta, bk, 200, opts=opts)
    c = np.random.default_rng(1).standard_normal(V.shape[0])
    # away from a fixed point the adjoint system converges slowly (GMRES(100) reaches about 6e-6 in
    # 1500 steps here): 600 steps, and the residual they reach is measured in the oracle's equations
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)
        gV, info, w = mesh.rgd_admm_vjp(_t(V), src, y, z, rho, beta, bk, _t(c), restart=100, max_iter=600,
                                        tol=1e-10, return_w=True, opts=opts)
    y, z, gV, w = (x.cpu().numpy() for x in (y, z, gV, w))
    gV0, gy0, gz0 = oracle.rgd_u_step_vjp(V, F, src, y, z, rho, beta, c)
    gVw, jy, jz = oracle.rgd_round_vjp(V, F, src, y, z, rho, beta, bk, w[0], w[1])
    rhs = np.concatenate([gy0.ravel(), gz0.ravel()])
    res = np.concatenate([(w[0] - jy).ravel(), (w[1] - jz).ravel()]) - rhs
    ref = gV0 + gVw
    assert np.abs(gV - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.abs(gV.sum(axis=0)).max() <= 1e-8 * np.abs(gV).max()
    assert np.linalg.norm(res) <= max(2.0 * info["rel_resid"], 1e-10) * np.linalg.norm(rhs), \
        (np.linalg.norm(res), np.linalg.norm(rhs), info)
    assert m == 3042 and info["rel_resid"] <= 1e-4, info
