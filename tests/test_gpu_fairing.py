"""The inverse-fairing loop of §7.1 on the device, against the oracle: the mass gradient
d(sum_i M_i w_i)/dV, the M-norm objective 1/2 ||T - g(V)||_M^2 through autograd (the smoothing
solve and the differentiable mass composed by torch), and whole Sobolev-preconditioned steps."""
import numpy as np
import pytest

import oracle
from gpu_util import case, rel2

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


@pytest.mark.parametrize("name", ["octa", "ico3", "grid61x53", "ico5"])
def test_mass_vjp_matches_oracle(api, name):
    V, F, t, B, T = case(name, seed=31)
    w = np.random.default_rng(32).random(V.shape[0])
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    g = mesh.mass_vjp(_t(V), _t(w)).cpu().numpy()
    ref = oracle.mass_vjp(V, F, w)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


def _sphere(level, seed, sigma=0.03):
    from paper_2602_12105_gb300 import meshgen as mg
    Vc, F = mg.icosphere(level)
    T = mg.radial_perturb(Vc, sigma, np.random.default_rng(seed))
    return T, F


@pytest.mark.parametrize("level,t", [(2, 5e-3), (4, 1e-3)])
def test_mnorm_objective_autograd_matches_oracle(api, level, t):
    """U = smooth(mesh, V, None, t); loss = 0.5 * sum_i M_i(V) |U_i - T_i|^2 through autograd."""
    T, F = _sphere(level, seed=33)
    V = T * 1.02
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    opts = api.make_opts(rel_tol=1e-14, max_iter=50000)
    Vd = _t(V).requires_grad_(True)
    U = api.smooth(mesh, Vd, None, t, opts=opts)
    M = api.mass(mesh, Vd)
    loss = 0.5 * (M[:, None] * (U - _t(T)) ** 2).sum()
    loss.backward()
    ref = oracle.mnorm_objective(V, F, T, t)
    assert abs(float(loss.detach()) - ref["loss"]) <= 1e-12 * ref["loss"]
    assert rel2(Vd.grad.cpu().numpy(), ref["gV"]) <= 1e-10


@pytest.mark.parametrize("name,level,t", [("sphere2", 2, 1e-2), ("sphere4", 4, 2e-3)])
def test_fairing_step_matches_oracle(api, name, level, t):
    T, F = _sphere(level, seed=34)
    V = T.copy()
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    opts = api.make_opts(rel_tol=1e-14, max_iter=50000)
    ref = oracle.mnorm_objective(V, F, T, t)
    eta = 0.05
    V1_ref, loss_ref = oracle.fairing_step(V, F, T, t, eta)
    fair = api.InverseFairing(mesh, _t(T), t, eta, opts=opts)
    Vd = _t(V)
    loss, infos = fair.step(Vd, info=True)
    assert [i["status"] for i in infos] == [0, 0, 0], infos
    assert abs(loss - loss_ref) <= 1e-12 * loss_ref
    step_gpu = Vd.cpu().numpy() - V
    step_ref = V1_ref - V
    assert rel2(step_gpu, step_ref) <= 1e-9, (rel2(step_gpu, step_ref), ref["loss"])


def test_fairing_loop_inflates_and_lowers_the_objective(api):
    """V starts at the targets (the paper's initialisation); smoothing shrinks the mesh, so the
    optimisation must inflate V for g(V) to come back to T: the objective falls step after step
    and the mean radius grows. Mixed precision follows the FP64 steps closely."""
    T, F = _sphere(4, seed=35, sigma=0.02)
    t = 2e-3
    mesh = api.Mesh(_t(F, torch.int32), T.shape[0])
    fair = api.InverseFairing(mesh, _t(T), t, eta=1.0)
    Vd = _t(T)
    losses = [fair.step(Vd) for _ in range(12)]
    assert all(b < a for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.1 * losses[0]
    r0 = np.linalg.norm(T, axis=1).mean()
    r1 = np.linalg.norm(Vd.cpu().numpy(), axis=1).mean()
    assert r1 > r0
    mesh2 = api.Mesh(_t(F, torch.int32), T.shape[0])
    fair32 = api.InverseFairing(mesh2, _t(T), t, eta=1.0, precision="mixed")
    V32 = _t(T)
    for _ in range(12):
        fair32.step(V32, want_loss=False)
    assert rel2(V32.cpu().numpy() - T, Vd.cpu().numpy() - T) <= 1e-7
