"""Shared helpers of the GPU tests: seeded cases and comparisons against the CPU oracle.

The inputs come only from the seeded generators (paper_2602_12105_gb300.meshgen); every expected
value comes from the oracle run on those inputs.
"""
import numpy as np

from paper_2602_12105_gb300 import meshgen as mg


def rel2(a, b):
    """Relative 2-norm error of a against b."""
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - b) / (nb if nb > 0 else 1.0))


def relmax(a, b):
    """Largest elementwise error of a against b, relative to max |b|."""
    a, b = np.asarray(a), np.asarray(b)
    mb = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / (mb if mb > 0 else 1.0)) if b.size else 0.0


def assert_close(a, b, tol, what=""):
    """Both the relative 2-norm error and the largest elementwise error (relative to max |b|)
    within tol: the norm alone could hide a few wrong entries of a large array."""
    e2, em = rel2(a, b), relmax(a, b)
    assert e2 <= tol and em <= tol, f"{what}: rel 2-norm {e2:.3e}, max elementwise {em:.3e}, tol {tol:.1e}"


def case(name, seed=0, k=3):
    """Small cases that the oracle solves in seconds. Several span more than one 256-row tile
    with a ragged last tile (grid61x53: 3233 rows; ico5: 10242 rows)."""
    rng = np.random.default_rng(seed)
    if name == "tetra":
        V, F = mg.regular_tetrahedron(1.0)
        t = 0.1
    elif name == "octa":
        V, F = mg.octahedron()
        V = V * (1.0 + 0.1 * rng.standard_normal((V.shape[0], 1)))
        t = 0.05
    elif name == "ico3":
        p = mg.config_ico3(seed)
        return p.V, p.F, p.t, rng.uniform(-1, 1, (p.n, k)), rng.uniform(-1, 1, (p.n, k))
    elif name == "ico5":
        Vc, F = mg.icosphere(5)
        V = mg.radial_perturb(Vc, 0.02, rng)
        t = 1e-3
    elif name == "grid61x53":
        p = mg.config_grid(61, 53, seed=seed)
        V, F, t = p.V, p.F, p.t
    elif name == "sliver":
        V, F = mg.sliver_mesh()
        t = 0.3
    elif name == "planar_jitter":
        V, F, _ = mg.jittered_planar_grid(40, 31, 0.05, 0.3, rng)
        t = 0.0025
    else:
        raise KeyError(name)
    n = V.shape[0]
    return V, F, t, rng.uniform(-1, 1, (n, k)), rng.uniform(-1, 1, (n, k))


CASES = ["tetra", "octa", "sliver", "ico3", "grid61x53", "planar_jitter", "ico5"]
