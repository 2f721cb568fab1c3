"""Mixed precision (FP32 inner Jacobi-PCG, FP64 residual refinement) against the FP64 oracle.

The refinement residual uses the FP64 operator, so the converged answer is the FP64 solution:
with both sides solved to 1e-13 the results match the oracle to 1e-10 like the FP64 path. At the
workload tolerance (1e-10) the residual under the oracle's operator stays within
1e-10 * (1 + 1e-3) and the solution differs from the FP64 GPU path by at most 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_close, case, rel2

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
    if rowptr.shape[0] - 1 <= 3000:
        return oracle.dense_cholesky_solve(rowptr, col, Aval, R)
    return oracle.pcg_solve(rowptr, col, Aval, R, tol=1e-14)[0]


@pytest.mark.parametrize("name", ["octa", "ico3", "grid61x53", "planar_jitter", "ico5"])
def test_mixed_forward_adjoint_match_oracle(api, name):
    V, F, t, B, T = case(name, seed=11)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t, precision="mixed")
    opts = api.make_opts(rel_tol=1e-13)
    U, info = mesh.solve(_t(B), opts=opts, info=True)
    assert info["status"] == 0, info
    assert info["refinements"] >= 2
    assert max(info["true_rel_residual"]) <= 1e-13 * (1 + 1e-3) * 10
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    U_ref = _oracle_solve(o_rowptr, o_col, o_A, o_M[:, None] * B)
    assert_close(U.cpu().numpy(), U_ref, 1e-10, "U")
    gV, gB, gt, ainfo = mesh.adjoint(_t(V), _t(B), False, U, U - _t(T), want_gB=True, want_gt=True, opts=opts,
                                     info=True)
    assert ainfo["status"] == 0, ainfo
    Lam_ref = _oracle_solve(o_rowptr, o_col, o_A, U_ref - T)
    gV_ref, gB_ref, gt_ref = oracle.vjp(V, F, t, U_ref, Lam_ref, B, False)
    assert_close(gV.cpu().numpy(), gV_ref, 1e-10, "gV")
    assert_close(gB.cpu().numpy(), gB_ref, 1e-10, "gB")
    assert abs(gt.item() - gt_ref) <= 1e-10 * abs(gt_ref)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_mixed_at_workload_tolerance(api, k):
    V, F, t, B, T = case("ico5", seed=12, k=k)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t, precision="mixed")
    Um, info = mesh.solve(_t(B), info=True)
    assert info["status"] == 0, info
    mesh.assemble(_t(V), t, precision="fp64")
    U64 = mesh.solve(_t(B))
    assert rel2(Um.cpu().numpy(), U64.cpu().numpy()) <= 1e-9
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    R = o_M[:, None] * B
    res = R - oracle.spmv(o_rowptr, o_col, o_A, Um.cpu().numpy())
    rel = np.linalg.norm(res, axis=0) / np.linalg.norm(R, axis=0)
    assert rel.max() <= 1e-10 * (1 + 1e-3), rel


def test_mixed_deterministic_and_launch_modes(api):
    V, F, t, B, T = case("grid61x53", seed=13)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t, precision="mixed")
    Bt = _t(B)
    U1 = mesh.solve(Bt, opts=api.make_opts(launch="graph"))
    U2 = mesh.solve(Bt, opts=api.make_opts(launch="graph"))
    U3 = mesh.solve(Bt, opts=api.make_opts(launch="host"))
    assert torch.equal(U1, U2) and torch.equal(U1, U3)


def test_mixed_refinement_cap(api):
    from paper_2602_12105_gb300 import _native as N
    V, F, t, B, T = case("ico5", seed=14)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t, precision="mixed")
    U, info = mesh.solve(_t(B), opts=api.make_opts(rel_tol=1e-13, max_refine=1), info=True)
    assert info["status"] == N.IG_ERR_NOT_CONVERGED and info["refinements"] == 1
    # the best iterate is still written and is a good approximation
    assert max(info["true_rel_residual"]) < 1e-3


@pytest.mark.parametrize("name,t_scale", [("ico5", 1.0), ("grid61x53", 1.0), ("planar_jitter", 1.0), ("sliver", 1.0),
                                          ("ico5", 1e-40), ("ico5", 1e41)])
def test_fp32_operator_is_the_fp64_operator_rounded_to_nearest(api, name, t_scale):
    """In mixed precision the FP32 copy of A is the FP64 operator rounded to nearest, ties to even,
    entry by entry: the assembly rounds with integer instructions, and numpy's float64 -> float32
    cast is that rounding. The scaled t puts off-diagonal entries below the float normal range
    (1e-40: float subnormals) and past the largest float (1e41: infinities)."""
    V, F, t, B, T = case(name, seed=21)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t * t_scale, precision="mixed")
    A64, _ = mesh.operator()
    a64 = A64.cpu().numpy()
    a32 = mesh.operator32().cpu().numpy()
    with np.errstate(over="ignore"):
        ref = a64.astype(np.float32)
    assert np.array_equal(a32.view(np.uint32), ref.view(np.uint32))


# ------------------------------------------------------------------------------- FP32 face geometry
# The mixed32 mode computes cotangents, areas and the per-face gradient in FP32 (FP64 for faces
# whose smallest corner has sin < 1e-2) and solves the FP32 operator A32 exactly (FP64 refinement).
# Its error against the FP64 oracle is that of the operator's FP32 rounding:
#   - each weight t cot / 2 and area / 3 is a few FP32 operations on edges that are exact to one
#     FP32 rounding (hi/lo split positions), so within about 4 u = 2.4e-7 of its value (u = 2^-24);
#     a row of A sums up to ~12 of them, so A and M are held to 1e-6 of max |A| and max |M|;
#   - U solves A32 U = M32 B, so its relative error is at most cond(A) times that of the operator;
#     with t small against the squared mesh spacing, cond(A) is a few, and U is held to 1e-6;
#   - dl/dV is a sum of per-face FP32 terms built from the same split data and U, Lambda, so it is
#     held to 2e-6 (relative to max |dl/dV|), and dl/dt to 1e-6.
# The translated meshes check that positions far from the origin keep that accuracy (the split
# takes differences of neighbouring vertices exactly; a plain FP32 copy of the positions would
# lose about |x| / |edge| ulps there).
R1_CASES = ["tetra", "octa", "ico3", "grid61x53", "planar_jitter", "ico5", "ico5_shifted", "grid61x53_shifted"]


@pytest.mark.parametrize("name", R1_CASES)
def test_fp32_geometry_matches_oracle(api, name):
    V, F, t, B, T = case(name.replace("_shifted", ""), seed=21)
    if name.endswith("_shifted"):
        V = V + np.array([1000.0, -2000.0, 500.0])
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t, precision="mixed32")
    A, M = mesh.operator()
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    assert_close(A.cpu().numpy(), o_A, 1e-6, "A32")
    assert_close(M.cpu().numpy(), o_M, 1e-6, "M")
    opts = api.make_opts(rel_tol=1e-13)
    U, info = mesh.solve(_t(B), opts=opts, info=True)
    assert info["status"] == 0, info
    # solved exactly for its own operator: the FP64 residual under A32 (as ig_operator returns it)
    R = M.cpu().numpy()[:, None] * B
    res = R - oracle.spmv(o_rowptr, o_col, A.cpu().numpy(), U.cpu().numpy())
    assert (np.linalg.norm(res, axis=0) / np.linalg.norm(R, axis=0)).max() <= 1e-13 * (1 + 1e-3)
    ref = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14)
    assert_close(U.cpu().numpy(), ref["U"], 1e-6, "U")
    gV, gB, gt, ainfo = mesh.adjoint(_t(V), _t(B), False, U, U - _t(T), want_gB=True, want_gt=True, opts=opts,
                                     info=True)
    assert ainfo["status"] == 0, ainfo
    assert_close(gV.cpu().numpy(), ref["gV"], 2e-6, "dl/dV")
    assert_close(gB.cpu().numpy(), ref["gB"], 1e-6, "dl/dB")
    assert abs(gt.item() - ref["gt"]) <= 1e-6 * abs(ref["gt"])


def test_fp32_geometry_symmetric_operator_and_batch_bits(api):
    """A32 is exactly symmetric (each edge's two weights are added in the same order by both of
    its rows), and a mesh gives the same bits alone and inside a batch in this mode too."""
    V, F, t, B, T = case("ico5", seed=22)
    n = V.shape[0]
    mesh = api.Mesh(_t(F, torch.int32), n)
    mesh.assemble(_t(V), t, precision="mixed32")
    A, M = mesh.operator()
    rowptr, col = mesh.pattern()
    rp, cl, a = rowptr.cpu().numpy(), col.cpu().numpy(), A.cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    vals = dict(zip(zip(rows.tolist(), cl.tolist()), a.tolist()))
    assert all(vals[(j, i)] == v for (i, j), v in vals.items())
    U1 = mesh.solve(_t(B))
    gV1, _, _ = mesh.adjoint(_t(V), _t(B), False, U1, U1 - _t(T))
    V2, F2, t2, B2, T2 = case("grid61x53", seed=23)
    other = api.Mesh(_t(F2, torch.int32), V2.shape[0])
    batch = api.Batch([other, mesh])
    batch.assemble([_t(V2), _t(V)], [t2, t], precision="mixed32")
    Us = batch.solve([_t(B2), _t(B)])
    gVs, _, _ = batch.adjoint([_t(V2), _t(V)], [_t(B2), _t(B)], False, Us, [Us[0] - _t(T2), Us[1] - _t(T)])
    assert torch.equal(Us[1], U1) and torch.equal(gVs[1], gV1)


def test_fp32_geometry_sliver_faces_take_the_fp64_path(api):
    """On the sliver mesh (a corner with sin = 2e-4, about 0.01 degrees) the weights of the sliver faces come
    from the FP64 path: the FP32 operator is within FP32 rounding (6e-8) of the FP64 one, where
    FP32 arithmetic on that face would lose a factor of about 1 / sin(theta) = 5e3 in accuracy."""
    V, F, t, B, T = case("sliver")
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t, precision="mixed32")
    A, M = mesh.operator()
    o_rowptr, o_col, o_A, o_L, o_M = oracle.operator(V, F, t)
    assert_close(A.cpu().numpy(), o_A, 2e-7, "A32 with slivers")
    assert_close(M.cpu().numpy(), o_M, 2e-7, "M with slivers")
