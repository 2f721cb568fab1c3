"""The cotangent clamp (ig_mesh_set_cot_clamp: every corner's cotangent enters L as
max(cot, clamp_min), the cotangent weights with a minimum of the paper's §4 ARAP listing, read per
corner) on the GPU against the oracle's clamped path (oracle.forward_adjoint(..., clamp_min)).

On a jittered grid with obtuse corners (some clamped): the operator within 1e-12, U and dl/dV
within 1e-10 with both sides solved to 1e-13 (FP64), dl/dt within 1e-10; the same in mixed
precision, and within the FP32-geometry tolerances (1e-6, 2e-6) with FP32 face geometry. Where no
corner is below the minimum the clamp changes no bit. Batches carry each mesh's own setting.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CMIN = 1e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_12105_gb300 import api as _api
    return _api


def _t(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def _obtuse_case(seed=12):
    from paper_2602_12105_gb300 import meshgen as mg
    rng = np.random.default_rng(seed)
    V, F, _ = mg.jittered_planar_grid(40, 31, 0.05, 0.45, rng)
    V[:, 2] = 0.01 * rng.standard_normal(V.shape[0])
    B = rng.uniform(-1, 1, (V.shape[0], 3))
    T = rng.uniform(-1, 1, (V.shape[0], 3))
    return V, F, 0.002, B, T


@pytest.mark.parametrize("precision,tol_a,tol_u,tol_g", [("fp64", 1e-12, 1e-10, 1e-10), ("mixed", 1e-12, 1e-10, 1e-10),
                                                          ("mixed32", 1e-6, 1e-6, 2e-6)])
def test_clamped_step_matches_oracle(api, precision, tol_a, tol_u, tol_g):
    V, F, t, B, T = _obtuse_case()
    P = V[F]
    cot = np.stack([np.einsum("ij,ij->i", P[:, (c + 1) % 3] - P[:, c], P[:, (c + 2) % 3] - P[:, c]) /
                    np.linalg.norm(np.cross(P[:, (c + 1) % 3] - P[:, c], P[:, (c + 2) % 3] - P[:, c]), axis=1)
                    for c in range(3)], axis=1)
    assert (cot < CMIN).sum() >= 20
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.set_cot_clamp(CMIN)
    mesh.assemble(_t(V), t, precision)
    ref = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14, clamp_min=CMIN)
    A, M = mesh.operator()
    assert_close(A.cpu().numpy(), ref["Aval"], tol_a, "A")
    opts = api.make_opts(rel_tol=1e-13)
    U, info = mesh.solve(_t(B), opts=opts, info=True)
    assert info["status"] == 0, info
    assert_close(U.cpu().numpy(), ref["U"], tol_u, "U")
    gV, gB, gt, ainfo = mesh.adjoint(_t(V), _t(B), False, U, U - _t(T), want_gB=True, want_gt=True, opts=opts,
                                     info=True)
    assert ainfo["status"] == 0, ainfo
    assert_close(gV.cpu().numpy(), ref["gV"], tol_g, "dl/dV")
    assert abs(gt.item() - ref["gt"]) <= tol_g * abs(ref["gt"])
    # the unclamped gradient differs there: the clamp is exercised
    plain = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14)
    assert np.abs(plain["gV"] - ref["gV"]).max() > 1e-3 * np.abs(ref["gV"]).max()


def test_clamp_off_and_inactive_change_no_bit(api):
    from paper_2602_12105_gb300 import meshgen as mg
    Vc, F = mg.icosphere(4)
    V = mg.radial_perturb(Vc, 0.01, np.random.default_rng(3))
    B = np.random.default_rng(4).uniform(-1, 1, V.shape)
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), 0.01)
    U0 = mesh.solve(_t(B))
    g0 = mesh.adjoint(_t(V), _t(B), False, U0, U0 - 1.0, want_gt=True)
    mesh.set_cot_clamp(CMIN)   # every corner of this sphere is acute: nothing is clamped
    mesh.assemble(_t(V), 0.01)
    U1 = mesh.solve(_t(B))
    g1 = mesh.adjoint(_t(V), _t(B), False, U1, U1 - 1.0, want_gt=True)
    assert torch.equal(U0, U1) and torch.equal(g0[0], g1[0]) and torch.equal(g0[2], g1[2])
    mesh.set_cot_clamp(None)
    mesh.assemble(_t(V), 0.01)
    assert torch.equal(mesh.solve(_t(B)), U0)


def test_clamp_needs_reassembly_and_geodesics_refuse_it(api):
    from paper_2602_12105_gb300 import _native as N
    V, F, t, B, T = _obtuse_case()
    mesh = api.Mesh(_t(F, torch.int32), V.shape[0])
    mesh.assemble(_t(V), t)
    mesh.set_cot_clamp(CMIN)
    with pytest.raises(N.IgError) as e:
        mesh.solve(_t(B))
    assert e.value.status == N.IG_ERR_STATE
    with pytest.raises(N.IgError) as e:
        mesh.rgd_u_step(_t(V), [0], torch.zeros((F.shape[0], 3), dtype=torch.float64, device=DEV),
                        torch.zeros((F.shape[0], 3), dtype=torch.float64, device=DEV), 1.0, 0.0)
    assert e.value.status == N.IG_ERR_STATE


def test_batch_carries_each_meshes_clamp(api):
    V, F, t, B, T = _obtuse_case()
    a = api.Mesh(_t(F, torch.int32), V.shape[0])
    b = api.Mesh(_t(F, torch.int32), V.shape[0])
    a.set_cot_clamp(CMIN)
    batch = api.Batch([a, b])
    batch.assemble([_t(V), _t(V)], [t, t])
    Us = batch.solve([_t(B), _t(B)], opts=api.make_opts(rel_tol=1e-13))
    ref_c = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14, clamp_min=CMIN)
    ref_p = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14)
    assert_close(Us[0].cpu().numpy(), ref_c["U"], 1e-10, "clamped mesh")
    assert_close(Us[1].cpu().numpy(), ref_p["U"], 1e-10, "plain mesh")
