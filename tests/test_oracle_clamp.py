"""Pins of the oracle's clamped cotangent weights (the cotangent weights with a minimum, clamp_min,
of the paper's §4 ARAP listing; read per corner: cot_c <- max(cot_c, clamp_min), with no derivative
through a clamped corner), checked against what the geometry fixes:

- a single obtuse triangle whose cotangents are known in closed form (5, 5 and -2.4);
- with clamping every off-diagonal entry of L is at most -clamp_min / 2 (an M-matrix), and L is
  still symmetric with zero row sums;
- where no corner is below the minimum, the clamped operator and gradient are the unclamped ones;
- the gradient of the clamped step matches central differences of the clamped loss on a mesh with
  clamped (obtuse) corners, in V and in t, while the unclamped gradient does not.
"""
import numpy as np

import oracle
from paper_2602_12105_gb300 import meshgen as mg

CMIN = 1e-5


def _dense(rowptr, col, val, n):
    D = np.zeros((n, n))
    for i in range(n):
        for e in range(rowptr[i], rowptr[i + 1]):
            D[i, col[e]] += val[e]
    return D


def _cots(V, F):
    P = V[F]
    out = np.empty((F.shape[0], 3))
    for c in range(3):
        ej, ek = P[:, (c + 1) % 3] - P[:, c], P[:, (c + 2) % 3] - P[:, c]
        out[:, c] = np.einsum("ij,ij->i", ej, ek) / np.linalg.norm(np.cross(ej, ek), axis=1)
    return out


def test_obtuse_triangle_closed_form():
    # (0,0), (2,0), (1,0.2): corners 0 and 1 have cot = 2 / 0.4 = 5, corner 2 has
    # cot = ((-1)(1) + (-0.2)(-0.2)) / 0.4 = -2.4; edge (0,1) is opposite corner 2
    V = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [1.0, 0.2, 0.0]])
    F = np.array([[0, 1, 2]], dtype=np.int32)
    L = _dense(*oracle.laplacian(V, F), 3)
    Lc = _dense(*oracle.laplacian(V, F, clamp_min=CMIN), 3)
    want = np.array([[1.3, 1.2, -2.5], [1.2, 1.3, -2.5], [-2.5, -2.5, 5.0]])
    want_c = np.array([[2.5 + CMIN / 2, -CMIN / 2, -2.5], [-CMIN / 2, 2.5 + CMIN / 2, -2.5], [-2.5, -2.5, 5.0]])
    assert np.abs(L - want).max() <= 1e-14
    assert np.abs(Lc - want_c).max() <= 1e-14


def _obtuse_mesh(seed=12):
    rng = np.random.default_rng(seed)
    V, F, _ = mg.jittered_planar_grid(12, 10, 0.1, 0.45, rng)
    V[:, 2] = 0.02 * rng.standard_normal(V.shape[0])
    return V, F


def test_clamped_laplacian_is_an_m_matrix():
    V, F = _obtuse_mesh()
    cot = _cots(V, F)
    assert (cot < CMIN).sum() >= 10  # there are obtuse corners to clamp
    n = V.shape[0]
    Lc = _dense(*oracle.laplacian(V, F, clamp_min=CMIN), n)
    L = _dense(*oracle.laplacian(V, F), n)
    off = ~np.eye(n, dtype=bool)
    pattern = (L != 0) & off
    assert (Lc[pattern] <= -CMIN / 2 * (1 - 1e-12)).all()
    assert (L[pattern] > 0).any()  # without the clamp some weights are positive
    assert np.abs(Lc - Lc.T).max() == 0.0
    assert np.abs(Lc.sum(axis=1)).max() <= 1e-13 * np.abs(Lc).max()


def test_clamp_below_every_cotangent_changes_nothing():
    Vc, F = mg.icosphere(3)
    V = mg.radial_perturb(Vc, 0.01, np.random.default_rng(4))
    assert _cots(V, F).min() > CMIN
    B = np.random.default_rng(5).uniform(-1, 1, (V.shape[0], 3))
    T = np.random.default_rng(6).uniform(-1, 1, (V.shape[0], 3))
    a = oracle.forward_adjoint(V, F, B, 0.01, T, False)
    b = oracle.forward_adjoint(V, F, B, 0.01, T, False, clamp_min=CMIN)
    for key in ("Aval", "U", "gV", "gB"):
        assert np.array_equal(a[key], b[key]), key
    assert a["gt"] == b["gt"]


def _loss(V, F, B, T, t, clamp_min):
    r = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14, clamp_min=clamp_min)
    return r["loss"]


def test_clamped_gradient_matches_central_differences():
    V, F = _obtuse_mesh()
    cot = _cots(V, F)
    # no corner within the finite-difference reach of the kink at CMIN
    assert np.abs(cot - CMIN).min() > 1e-3
    rng = np.random.default_rng(7)
    B = rng.uniform(-1, 1, (V.shape[0], 3))
    T = rng.uniform(-1, 1, (V.shape[0], 3))
    t = 0.02
    r = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14, clamp_min=CMIN)
    plain = oracle.forward_adjoint(V, F, B, t, T, False, tol=1e-14)
    h = 1e-6
    gmax = np.abs(r["gV"]).max()
    # vertices at clamped corners, where the clamp matters
    clamped_vertices = np.unique(F[cot < CMIN])
    worst_plain = 0.0
    for i in clamped_vertices[:6]:
        for d in range(2):
            Vp, Vm = V.copy(), V.copy()
            Vp[i, d] += h
            Vm[i, d] -= h
            fd = (_loss(Vp, F, B, T, t, CMIN) - _loss(Vm, F, B, T, t, CMIN)) / (2 * h)
            assert abs(fd - r["gV"][i, d]) <= 1e-6 * gmax + 1e-9, (i, d, fd, r["gV"][i, d])
            worst_plain = max(worst_plain, abs(fd - plain["gV"][i, d]))
    # a planted mistake: the unclamped gradient (derivative through the clamped corners) is off
    assert worst_plain > 1e-4 * gmax
    fd_t = (_loss(V, F, B, T, t + h, CMIN) - _loss(V, F, B, T, t - h, CMIN)) / (2 * h)
    assert abs(fd_t - r["gt"]) <= 1e-6 * abs(r["gt"]) + 1e-9
