"""Seeded synthetic inputs for the implicit-smoothing path (icospheres, height-field grids,
right-hand sides, targets, batches and request streams).

This module only builds input arrays. It holds none of the method's arithmetic (no
cotangents, masses, solves or gradients), so that the CPU oracle and the CUDA path can both
be fed from it without sharing any code of the method.

Shapes follow the paper's inverse mean-curvature-flow setting (§7.1): V is [n][3] float64
vertex positions, F is [m][3] int32 triangle indices ordered counter-clockwise (outward for
closed surfaces, +z for height fields).
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------- icospheres
def icosahedron():
    """The 12-vertex, 20-face regular icosahedron on the unit sphere, faces CCW outward."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array(
        [[-1, phi, 0], [1, phi, 0], [-1, -phi, 0], [1, -phi, 0],
         [0, -1, phi], [0, 1, phi], [0, -1, -phi], [0, 1, -phi],
         [phi, 0, -1], [phi, 0, 1], [-phi, 0, -1], [-phi, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return V, F


def _orient_outward(V, F):
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    F = F.copy()
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return F


def icosphere(level: int):
    """Unit icosphere by midpoint subdivision, re-projected to the sphere after every level.

    Level k has 10*4^k + 2 vertices and 20*4^k faces. Returns (V float64 [n][3],
    F int32 [m][3]) with faces CCW seen from outside (fresh copies; the construction is cached).
    """
    V, F = _icosphere_cached(level)
    return V.copy(), F.copy()


@functools.lru_cache(maxsize=16)
def _icosphere_cached(level: int):
    if level < 0:
        raise ValueError("level must be >= 0")
    V, F = icosahedron()
    F = _orient_outward(V, F)
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
        key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
        ukey, inv = np.unique(key, return_inverse=True)
        a, b = ukey // nv, ukey % nv
        mid = V[a] + V[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = F.shape[0]
        ab, bc, ca = (nv + inv[:m], nv + inv[m:2 * m], nv + inv[2 * m:])
        f0, f1, f2 = F[:, 0], F[:, 1], F[:, 2]
        F = np.concatenate([
            np.stack([f0, ab, ca], 1), np.stack([f1, bc, ab], 1),
            np.stack([f2, ca, bc], 1), np.stack([ab, bc, ca], 1)], axis=0)
        V = np.concatenate([V, mid], axis=0)
        V /= np.linalg.norm(V, axis=1, keepdims=True)
    return np.ascontiguousarray(V), np.ascontiguousarray(F.astype(np.int32))


def icosphere_vertex_count(level: int) -> int:
    return 10 * 4 ** level + 2


def radial_perturb(V, sigma: float, rng: np.random.Generator):
    """v <- v_hat * (1 + eps), eps ~ N(0, sigma) per vertex."""
    eps = rng.normal(0.0, sigma, size=V.shape[0])
    vhat = V / np.linalg.norm(V, axis=1, keepdims=True)
    return np.ascontiguousarray(vhat * (1.0 + eps)[:, None])


# ----------------------------------------------------------------------------- grids
def grid_faces(nx: int, ny: int):
    """Faces of a regular nx-by-ny vertex grid (vertex (i, j) has index j*nx + i).

    Each quad is split along its (i,j)-(i+1,j+1) diagonal into two triangles, CCW about +z.
    Faces are ordered quad by quad, row-major, two per quad.
    """
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    v00 = (j * nx + i).ravel()
    v10, v01, v11 = v00 + 1, v00 + nx, v00 + nx + 1
    F = np.empty((2 * v00.size, 3), dtype=np.int32)
    F[0::2] = np.stack([v00, v10, v11], 1)
    F[1::2] = np.stack([v00, v11, v01], 1)
    return F


def box_filter5(z):
    """5x5 mean filter with replicate padding."""
    zp = np.pad(z, 2, mode="edge")
    out = np.zeros_like(z)
    for dj in range(5):
        for di in range(5):
            out += zp[dj:dj + z.shape[0], di:di + z.shape[1]]
    return out / 25.0


def grid_mesh(nx: int, ny: int, h: float, heights=None):
    """Grid positions on [0,(nx-1)h] x [0,(ny-1)h]; heights is an (ny, nx) array or None."""
    x = np.arange(nx, dtype=np.float64) * h
    y = np.arange(ny, dtype=np.float64) * h
    X, Y = np.meshgrid(x, y, indexing="xy")
    Z = np.zeros_like(X) if heights is None else heights
    V = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    return np.ascontiguousarray(V), grid_faces(nx, ny)


def smoothed_heights(nx: int, ny: int, rng: np.random.Generator, amp: float = 0.05):
    """z = amp * N(0,1), then a 5x5 box filter (replicate padding)."""
    return box_filter5(amp * rng.standard_normal((ny, nx)))


# ----------------------------------------------------------------------------- problems
@dataclass
class Problem:
    """One smoothing problem: solve (M + tL) U = M B, loss 0.5*||U - T||^2."""
    name: str
    V: np.ndarray            # [n][3] float64
    F: np.ndarray            # [m][3] int32
    t: float
    B: np.ndarray            # [n][k] float64 (B is V itself when b_is_V)
    T: np.ndarray            # [n][k] float64 loss target
    b_is_V: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.V.shape[0]

    @property
    def m(self):
        return self.F.shape[0]


def problem_icosphere(level: int, sigma: float, t: float, rng: np.random.Generator, name=None):
    """Noisy icosphere smoothing: B = the noisy positions, target = the clean sphere."""
    Vc, F = icosphere(level)
    V = radial_perturb(Vc, sigma, rng)
    return Problem(name or f"ico{level}", V, F, t, V, Vc.copy(), b_is_V=True,
                   meta={"level": level, "sigma": sigma})


def problem_grid(nx: int, ny: int, h: float, t: float, seed: int, k: int = 3, name=None):
    """Height-field grid: B ~ U[-1,1]^{n x k} (seed), target T ~ U[-1,1] (seed + 1)."""
    rng = np.random.default_rng(seed)
    Z = smoothed_heights(nx, ny, rng)
    V, F = grid_mesh(nx, ny, h, Z)
    B = rng.uniform(-1.0, 1.0, size=(V.shape[0], k))
    T = np.random.default_rng(seed + 1).uniform(-1.0, 1.0, size=(V.shape[0], k))
    return Problem(name or f"grid{nx}x{ny}", V, F, t, B, T, b_is_V=False,
                   meta={"nx": nx, "ny": ny, "h": h})


def config_ico3(seed: int = 0):
    """Unit icosphere level 3 (642 vertices, 1280 faces), radial N(0, 0.01), t = 1e-3."""
    return problem_icosphere(3, 0.01, 1e-3, np.random.default_rng(seed), name="ico3")


def config_grid1024(seed: int = 0):
    """1024 x 1024 grid on [0,1]^2, t = h^2, 3 RHS of U[-1,1]."""
    h = 1.0 / 1023.0
    return problem_grid(1024, 1024, h, h * h, seed, name="grid1024")


def config_grid4096x2048(seed: int = 0):
    """4096 x 2048 grid with square cells h = 1/2047 on [0, 4095h] x [0, 1], t = h^2."""
    h = 1.0 / 2047.0
    return problem_grid(4096, 2048, h, h * h, seed, name="grid4096x2048")


def config_grid(side_x: int, side_y: int, seed: int = 0, t=None):
    """A smaller grid of the same family (unit height in y); t = h^2 unless given."""
    h = 1.0 / (side_y - 1)
    return problem_grid(side_x, side_y, h, h * h if t is None else t, seed,
                        name=f"grid{side_x}x{side_y}")


def config_batch(seed: int = 0, count: int = 256, levels=(2, 3, 4, 5, 6), sigma: float = 0.02):
    """Differentiation batch: icosphere levels uniform over `levels`, t log-uniform in
    [1e-4, 1e-2], radial perturbation N(0, sigma)."""
    rng = np.random.default_rng(seed)
    lv = rng.choice(np.asarray(levels), size=count)
    ts = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), size=count))
    base = {int(l): icosphere(int(l)) for l in np.unique(lv)}
    probs = []
    for b in range(count):
        Vc, F = base[int(lv[b])]
        V = radial_perturb(Vc, sigma, rng)
        probs.append(Problem(f"batch{b}_ico{int(lv[b])}", V, F, float(ts[b]), V, Vc.copy(),
                             b_is_V=True, meta={"level": int(lv[b]), "sigma": sigma}))
    return probs


@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str           # "ico" or "grid"
    size: int           # icosphere level or grid side
    t: float
    seed: int


def request_stream(count: int, rate_hz: float, seed: int = 0, n_min: float = 1e3, n_max: float = 2e6,
                   ico_levels=(4, 5, 6, 7, 8)):
    """Poisson arrivals; 50/50 icosphere or grid; vertex count log-uniform in [n_min, n_max]
    (an icosphere snaps to the nearest level in ico_levels, a grid is square with side
    round(sqrt(n))); t log-uniform in [1e-4, 1e-2]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    arr = np.cumsum(gaps) - gaps[0]
    kinds = rng.random(count) < 0.5
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=count))
    ts = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), size=count))
    lv = np.asarray(ico_levels)
    counts = np.array([icosphere_vertex_count(int(l)) for l in lv], dtype=np.float64)
    out = []
    for r in range(count):
        if kinds[r]:
            size = int(lv[np.argmin(np.abs(np.log(counts) - math.log(ns[r])))])
            kind = "ico"
        else:
            size = max(2, int(round(math.sqrt(ns[r]))))
            kind = "grid"
        out.append(Request(r, float(arr[r]), kind, size, float(ts[r]), seed * 1000003 + r))
    return out


def request_problem(req: Request, k: int = 3):
    """Materialise a request: icospheres get radial noise N(0, 0.01), B ~ U[-1,1]; grids as
    in the large-grid workload with h = 1/(side-1)."""
    if req.kind == "ico":
        rng = np.random.default_rng(req.seed)
        Vc, F = icosphere(req.size)
        V = radial_perturb(Vc, 0.01, rng)
        B = rng.uniform(-1.0, 1.0, size=(V.shape[0], k))
        T = np.random.default_rng(req.seed + 1).uniform(-1.0, 1.0, size=(V.shape[0], k))
        return Problem(f"req{req.rid}_ico{req.size}", V, F, req.t, B, T, False, {"level": req.size})
    side = req.size
    h = 1.0 / (side - 1)
    return problem_grid(side, side, h, req.t, req.seed, k=k, name=f"req{req.rid}_grid{side}")


# ----------------------------------------------------------------------------- tiny fixtures
def regular_tetrahedron(edge: float = 1.0):
    """Closed regular tetrahedron, faces CCW outward."""
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    V *= edge / (2.0 * math.sqrt(2.0))
    F = np.array([[0, 1, 2], [0, 2, 3], [0, 3, 1], [1, 3, 2]], dtype=np.int64)
    return V, _orient_outward(V, F).astype(np.int32)


def octahedron():
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float64)
    F = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int64)
    return V, _orient_outward(V, F).astype(np.int32)


def jittered_planar_grid(nx: int, ny: int, h: float, jitter: float, rng: np.random.Generator):
    """A planar (z = 0) grid whose interior vertices are moved in-plane by U[-jitter, jitter]*h."""
    V, F = grid_mesh(nx, ny, h)
    interior = np.zeros((ny, nx), dtype=bool)
    interior[1:-1, 1:-1] = True
    interior = interior.ravel()
    V[interior, :2] += rng.uniform(-jitter, jitter, size=(interior.sum(), 2)) * h
    return V, F, interior


def sliver_mesh():
    """Two triangles sharing an edge, one of them a near-degenerate sliver."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0.5, 1e-4, 0], [0.5, -1.0, 0.1]], dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 3, 1]], dtype=np.int32)
    return V, F
