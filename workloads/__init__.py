"""Seeded synthetic inputs shared by the tests, the oracle checks and ``bench.py``.

This module holds no arithmetic of the finite-element method: it only produces
macro meshes (vertex coordinates and tetrahedra), seeded random vectors in a
caller-given length, the parameters of the random Fourier field used for the
coefficient-inversion workload, and closed-form input functions (the
manufactured solution, the coefficient functions) evaluated at points the
caller supplies.

Macro meshes follow the paper's setting (Section 2): an unstructured coarse
mesh of macro-tetrahedra, each later refined uniformly.  The cube meshes use
the Kuhn (Freudenthal) split of a cube into 6 tetrahedra around its main
diagonal, which is conforming when the same split is used in every sub-cube.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "reference_tet", "kuhn_box", "cube6", "cube48", "cuboid36",
    "uniform", "uniform_keyed", "fourier_field_params", "fourier_field", "sin3_coeff",
    "manufactured_u", "manufactured_f", "viscosity_mu",
]


def reference_tet():
    """The reference macro-tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1)."""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    t = np.array([[0, 1, 2, 3]], dtype=np.int32)
    return v, t


def kuhn_box(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0, lz: float = 1.0):
    """Box [0,lx]x[0,ly]x[0,lz] split into nx*ny*nz sub-cubes of 6 Kuhn tetrahedra each.

    Every sub-cube is split along its (0,0,0)-(1,1,1) diagonal: for each
    permutation s of the axes the tetrahedron walks 0 -> e_s0 -> e_s0+e_s1 ->
    (1,1,1).  Vertices are numbered lexicographically (x fastest).
    """
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    verts = np.array([[x, y, z] for z in zs for y in ys for x in xs], dtype=np.float64)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for perm in itertools.permutations(range(3)):
                    p = [0, 0, 0]
                    path = [vid(i, j, k)]
                    for ax in perm:
                        p[ax] += 1
                        path.append(vid(i + p[0], j + p[1], k + p[2]))
                    tets.append(path)
    return verts, np.array(tets, dtype=np.int32)


def cube6():
    """Unit cube as 6 Kuhn macro-tetrahedra around the diagonal (0,0,0)-(1,1,1)."""
    return kuhn_box(1, 1, 1)


def cube48():
    """Unit cube as 2x2x2 sub-cubes of 6 Kuhn macro-tetrahedra (48 macros)."""
    return kuhn_box(2, 2, 2)


def cuboid36():
    """A 3x2x1 box of 36 Kuhn macro-tetrahedra (the paper's 36-macro cuboid, Section 7.1)."""
    return kuhn_box(3, 2, 1, 3.0, 2.0, 1.0)


def uniform(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """n values uniform on [-1, 1] from numpy's default_rng(seed)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n).astype(dtype)


_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """The splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014) on uint64 arrays."""
    z = (z + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
    return z ^ (z >> np.uint64(31))


def uniform_keyed(keys: np.ndarray, ncols: int, seed: int) -> np.ndarray:
    """Values uniform on [-1, 1) that depend only on a point's integer key, the column and the seed.

    keys: (P, K) integers identifying each point (the caller passes an exact global key, so every
    stored copy of a point shared by several macros receives the same values).  Returns (P, ncols):
    column c of point p is splitmix64 chained over (seed, key words, c), its top 53 bits scaled to
    [0, 1), then mapped to [-1, 1).  Counter-based, so any subset of points can be regenerated alone.
    """
    keys = np.asarray(keys, dtype=np.int64)
    with np.errstate(over="ignore"):
        h = np.full(len(keys), np.uint64(seed) ^ np.uint64(0x5851F42D4C957F2D), dtype=np.uint64)
        for c in range(keys.shape[1]):
            h = _splitmix64(h ^ keys[:, c].astype(np.uint64))
        out = np.empty((len(keys), ncols))
        for c in range(ncols):
            z = _splitmix64(h ^ np.uint64(c + 1))
            out[:, c] = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * out - 1.0


def fourier_field_params(seed: int = 0, modes: int = 8):
    """Wave vectors in {-2..2}^3 without 0 and phases in [0, 2 pi), seeded."""
    rng = np.random.default_rng(seed)
    kappas = []
    while len(kappas) < modes:
        kv = rng.integers(-2, 3, size=3)
        if np.any(kv != 0):
            kappas.append(kv)
    phases = rng.uniform(0.0, 2.0 * np.pi, modes)
    return np.array(kappas, dtype=np.float64), phases


def fourier_field(points: np.ndarray, seed: int = 0, amplitude: float = 0.5, modes: int = 8) -> np.ndarray:
    """g(x) = (amplitude/modes) * sum_m cos(2 pi kappa_m . x + phi_m); so |g| <= amplitude."""
    kappas, phases = fourier_field_params(seed, modes)
    arg = 2.0 * np.pi * (points @ kappas.T) + phases[None, :]
    return (amplitude / modes) * np.cos(arg).sum(axis=1)


def sin3_coeff(points: np.ndarray) -> np.ndarray:
    """k(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z) at the given points."""
    s = np.sin(2.0 * np.pi * points)
    return 1.0 + 0.5 * s[:, 0] * s[:, 1] * s[:, 2]


def manufactured_u(points: np.ndarray) -> np.ndarray:
    """u = sin(pi x) sin(pi y) sin(pi z) (zero on the unit cube's boundary)."""
    s = np.sin(np.pi * points)
    return s[:, 0] * s[:, 1] * s[:, 2]


def manufactured_f(points: np.ndarray) -> np.ndarray:
    """f = -Laplace(u) = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)."""
    return 3.0 * np.pi ** 2 * manufactured_u(points)


def viscosity_mu(points: np.ndarray) -> np.ndarray:
    """mu = 10^(3 (z - 0.5)), three orders of magnitude over the unit cube."""
    return 10.0 ** (3.0 * (points[:, 2] - 0.5))
