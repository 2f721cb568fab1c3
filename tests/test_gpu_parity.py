"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances (FP64 path): pattern bit-exact; A and M within 1e-12 of max|.|; U, Lambda-driven
gradients gV, gB and dl/dt within 1e-10 relative 2-norm when both sides solve to 1e-13 or
tighter. Sizes span several 256-row tiles with a ragged last tile.
"""
import numpy as np
import pytest

import oracle
from gpu_util import CASES, assert_close, case, rel2

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


def _oracle_solve(rowptr, col, Aval, R):
    n = rowptr.shape[0] - 1
    if n <= 3000:
        return oracle.dense_cholesky_solve(rowptr, col, Aval, R)
    X, iters, rel, st = oracle.pcg_solve(rowptr, col, Aval, R, tol=1e-14)
    return X


@pytest.mark.parametrize("name", CASES)
def test_pattern_and_operator(api, name):
    V, F, t, B, T = case(name)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t)
    mesh.check()
    rowptr, col = mesh.pattern()
    A, M = mesh.operator()
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    assert np.array_equal(rowptr.cpu().numpy().astype(np.int64), o_rowptr)
    assert np.array_equal(col.cpu().numpy(), o_col)
    A, M = A.cpu().numpy(), M.cpu().numpy()
    assert np.abs(A - o_A).max() <= 1e-12 * np.abs(o_A).max()
    assert np.abs(M - o_M).max() <= 1e-12 * np.abs(o_M).max()
    # L itself, from an assembly at t = 1: A(t=1) - M
    mesh.assemble(_t(V), 1.0)
    A1, M1 = mesh.operator()
    L = A1.cpu().numpy()
    L[o_col == np.repeat(np.arange(V.shape[0]), np.diff(o_rowptr))] -= M1.cpu().numpy()
    assert np.abs(L - o_L).max() <= 1e-12 * np.abs(o_L).max()


def _min_angle(V, F):
    P = V[F]
    ang = []
    for c in range(3):
        a, b = P[:, (c + 1) % 3] - P[:, c], P[:, (c + 2) % 3] - P[:, c]
        cosv = np.einsum("ij,ij->i", a, b) / np.linalg.norm(a, axis=1) / np.linalg.norm(b, axis=1)
        ang.append(np.arccos(np.clip(cosv, -1, 1)))
    return float(np.min(ang))


@pytest.mark.parametrize("name", CASES)
def test_forward_and_adjoint(api, name):
    """U within 1e-10; the gradient within max(1e-10, 1e-12 / theta_min): the derivative of a
    cotangent, d cot / d theta = -1 / sin^2 theta, amplifies rounding by about 1/theta on faces
    with a tiny angle theta, so two exact formulas of the same gradient agree only to that."""
    V, F, t, B, T = case(name)
    gtol = max(1e-10, 1e-12 / _min_angle(V, F))
    n = V.shape[0]
    mesh = api.Mesh(_t(F, torch.int32), n)
    mesh.assemble(_t(V), t)
    opts = api.make_opts(rel_tol=1e-13)
    U, info = mesh.solve(_t(B), opts=opts, info=True)
    assert info["status"] == 0, info
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    U_ref = _oracle_solve(o_rowptr, o_col, o_A, o_M[:, None] * B)
    assert_close(U.cpu().numpy(), U_ref, 1e-10, "U")
    # adjoint for l = 0.5 ||U - T||^2, both sides using their own U
    G = U - _t(T)
    gV, gB, gt, ainfo = mesh.adjoint(_t(V), _t(B), False, U, G, want_gB=True, want_gt=True, opts=opts, info=True)
    assert ainfo["status"] == 0, ainfo
    Lam_ref = _oracle_solve(o_rowptr, o_col, o_A, U_ref - T)
    gV_ref, gB_ref, gt_ref = oracle.vjp(V, F, t, U_ref, Lam_ref, B, False)
    assert_close(gV.cpu().numpy(), gV_ref, gtol, "gV")
    assert_close(gB.cpu().numpy(), gB_ref, 1e-10, "gB")
    assert abs(gt.item() - gt_ref) <= gtol * max(abs(gt_ref), 1e-300)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_column_counts(api, k):
    V, F, t, B, T = case("grid61x53", seed=3, k=k)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t)
    opts = api.make_opts(rel_tol=1e-13)
    U = mesh.solve(_t(B), opts=opts)
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    U_ref = _oracle_solve(o_rowptr, o_col, o_A, o_M[:, None] * B)
    assert_close(U.cpu().numpy(), U_ref, 1e-10, "U")
    gV, gB, gt = mesh.adjoint(_t(V), _t(B), False, U, U - _t(T), want_gB=True, want_gt=True, opts=opts)
    Lam_ref = _oracle_solve(o_rowptr, o_col, o_A, U_ref - T)
    gV_ref, gB_ref, gt_ref = oracle.vjp(V, F, t, U_ref, Lam_ref, B, False)
    assert_close(gV.cpu().numpy(), gV_ref, 1e-10, "gV")
    assert_close(gB.cpu().numpy(), gB_ref, 1e-10, "gB")


def test_b_is_V_autograd_matches_oracle(api):
    """The differentiable step on the noisy-icosphere workload (B = V, target the clean sphere)."""
    from paper_2602_12105_gb300 import meshgen as mg
    p = mg.config_ico3(seed=1)
    mesh = api.Mesh(_t(p.F, torch.int32), p.n)
    V = _t(p.V).requires_grad_(True)
    opts = api.make_opts(rel_tol=1e-13)
    U = api.smooth(mesh, V, None, p.t, opts=opts)
    loss = 0.5 * ((U - _t(p.T)) ** 2).sum()
    loss.backward()
    ref = oracle.forward_adjoint(p.V, p.F, p.B, p.t, p.T, True)
    assert_close(U.detach().cpu().numpy(), ref["U"], 1e-10, "U")
    assert_close(V.grad.cpu().numpy(), ref["gV"], 1e-10, "gV")
    assert abs(loss.item() - ref["loss"]) <= 1e-10 * ref["loss"]


def test_autograd_b_and_t(api):
    V, F, t, B, T = case("ico3", seed=4)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    Vt = _t(V).requires_grad_(True)
    Bt = _t(B).requires_grad_(True)
    tt = torch.tensor(t, dtype=torch.float64, device=DEV, requires_grad=True)
    U = api.smooth(mesh, Vt, Bt, tt, opts=api.make_opts(rel_tol=1e-13))
    (0.5 * ((U - _t(T)) ** 2).sum()).backward()
    ref = oracle.forward_adjoint(V, F, B, t, T, False)
    assert_close(Vt.grad.cpu().numpy(), ref["gV"], 1e-10, "gV")
    assert_close(Bt.grad.cpu().numpy(), ref["gB"], 1e-10, "gB")
    assert abs(tt.grad.item() - ref["gt"]) <= 1e-10 * abs(ref["gt"])


def test_gpu_central_differences(api):
    """Brute force on the GPU itself: central differences of the GPU loss against its gradient."""
    from paper_2602_12105_gb300 import meshgen as mg
    rng = np.random.default_rng(2)
    Vc, F = mg.icosphere(2)
    V = mg.radial_perturb(Vc, 0.05, rng)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    opts = api.make_opts(rel_tol=1e-14, max_iter=5000)

    def loss_of(Vn):
        U = mesh.assemble(_t(Vn), 2e-2).solve(_t(Vn), opts=opts)
        return 0.5 * float(((U - _t(Vc)) ** 2).sum())

    Vt = _t(V).requires_grad_(True)
    U = api.smooth(mesh, Vt, None, 2e-2, opts=opts)
    (0.5 * ((U - _t(Vc)) ** 2).sum()).backward()
    g = Vt.grad.cpu().numpy()
    h = 1e-6
    for flat in rng.choice(V.size, 8, replace=False):
        i, d = divmod(int(flat), 3)
        Vp, Vm = V.copy(), V.copy()
        Vp[i, d] += h
        Vm[i, d] -= h
        fd = (loss_of(Vp) - loss_of(Vm)) / (2 * h)
        assert abs(fd - g[i, d]) <= 1e-6 * np.abs(g).max() + 1e-9


def test_determinism_and_launch_modes(api):
    V, F, t, B, T = case("ico5", seed=5)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t)
    Bt = _t(B)
    U1 = mesh.solve(Bt, opts=api.make_opts(launch="graph"))
    U2 = mesh.solve(Bt, opts=api.make_opts(launch="graph"))
    U3 = mesh.solve(Bt, opts=api.make_opts(launch="host"))
    assert torch.equal(U1, U2)
    assert torch.equal(U1, U3)
    g1 = mesh.adjoint(_t(V), Bt, False, U1, U1 - _t(T), want_gt=True)
    g2 = mesh.adjoint(_t(V), Bt, False, U1, U1 - _t(T), want_gt=True)
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[2], g2[2])


def test_config_tolerance_residual_under_oracle_operator(api):
    """At the default tolerance (1e-10) the GPU solution's residual, measured with the ORACLE's
    operator, stays within rel_tol * (1 + 1e-3)."""
    V, F, t, B, T = case("ico5", seed=6)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t)
    U, info = mesh.solve(_t(B), info=True)
    assert info["status"] == 0
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    R = o_M[:, None] * B
    res = R - oracle.spmv(o_rowptr, o_col, o_A, U.cpu().numpy())
    rel = np.linalg.norm(res, axis=0) / np.linalg.norm(R, axis=0)
    assert rel.max() <= 1e-10 * (1 + 1e-3), rel
    assert max(info["true_rel_residual"]) <= 1e-10 * (1 + 1e-3)


# ------------------------------------------------------------------------------- edge cases
def test_error_statuses(api):
    from paper_2602_12105_gb300 import _native as N
    from paper_2602_12105_gb300 import meshgen as mg
    V, F = mg.octahedron()
    bad = F.copy(); bad[2, 1] = 6
    with pytest.raises(N.IgError) as e:
        api.Mesh(_t(bad, torch.int32), 6)
    assert e.value.status == N.IG_ERR_INDEX_OUT_OF_RANGE
    bad = F.copy(); bad[2, 1] = bad[2, 0]
    with pytest.raises(N.IgError) as e:
        api.Mesh(_t(bad, torch.int32), 6)
    assert e.value.status == N.IG_ERR_DEGENERATE_FACE
    with pytest.raises(N.IgError) as e:
        api.Mesh(_t(F, torch.int32), 7)
    assert e.value.status == N.IG_ERR_INVALID_ARG
    mesh = api.Mesh(_t(F, torch.int32), 6)
    with pytest.raises(N.IgError) as e:
        mesh.solve(_t(np.ones((6, 3))))
    assert e.value.status == N.IG_ERR_STATE
    # zero-area face
    Vd = V.copy(); Vd[4] = 0.5 * (Vd[0] + Vd[2])
    mesh.assemble(_t(Vd), 0.1)
    with pytest.raises(N.IgError) as e:
        mesh.check()
    assert e.value.status == N.IG_ERR_DEGENERATE_FACE
    # non-finite position
    Vn = V.copy(); Vn[1, 2] = np.nan
    mesh.assemble(_t(Vn), 0.1)
    with pytest.raises(N.IgError) as e:
        mesh.check()
    assert e.value.status == N.IG_ERR_NONFINITE
    # recovers after a good assembly
    mesh.assemble(_t(V), 0.1)
    mesh.check()
    # iteration cap
    Vc, Fi = mg.icosphere(3)
    mesh = api.Mesh(_t(Fi, torch.int32), Vc.shape[0])
    mesh.assemble(_t(Vc), 1e-2)
    U, info = mesh.solve(_t(np.random.default_rng(0).uniform(-1, 1, (Vc.shape[0], 3))),
                         opts=api.make_opts(max_iter=2), info=True)
    assert info["status"] == N.IG_ERR_NOT_CONVERGED and info["iterations"] == 2
    # zero right-hand side: exact zero solution, no iterations
    U, info = mesh.solve(_t(np.zeros((Vc.shape[0], 3))), info=True)
    assert info["status"] == 0 and info["iterations"] == 0 and float(U.abs().max()) == 0.0
    with pytest.raises(N.IgError) as e:
        mesh.solve(_t(np.zeros((Vc.shape[0], 5))))
    assert e.value.status == N.IG_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["tetra", "ico3", "planar_jitter", "sliver", "grid61x53"])
def test_small_mesh_cluster_loop_same_bits(api, name):
    """A single mesh of at most 16 FP64 tiles runs its whole iteration loop in one thread-block
    cluster (the graph launch mode; grid61x53 has 13 tiles); the host-launched mode runs the
    multi-CTA kernels. Same tile bodies, same partial sums in the same order: the same bits,
    forward and adjoint, and the same iteration counts."""
    V, F, t, B, T = case(name, seed=31)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t)
    res = {}
    for launch in ("graph", "host"):
        opts = api.make_opts(rel_tol=1e-12, launch=launch)
        U, fi = mesh.solve(_t(B), opts=opts, info=True)
        gV, gB, gt, ai = mesh.adjoint(_t(V), _t(B), False, U, U - _t(T), want_gt=True, opts=opts, info=True)
        res[launch] = (U, gV, gt, fi["iterations"], ai["iterations"])
    a, b = res["graph"], res["host"]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    assert a[3:] == b[3:]
