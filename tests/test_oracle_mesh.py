"""Pins of the oracle's refinement lattice and micro-tet enumeration (Section 2, Section 5.1)."""
import numpy as np
import pytest

import workloads as W
from oracle import mesh as M


@pytest.mark.parametrize("N", range(0, 9))
def test_lattice_count_and_order(N):
    pts = M.lattice_points(N)
    assert len(pts) == (N + 1) * (N + 2) * (N + 3) // 6 == M.lattice_size(N)
    assert np.all(pts.sum(axis=1) <= N) and pts.min() >= 0
    assert len({tuple(p) for p in pts}) == len(pts)
    # the packed position of the enumeration is 0..V-1
    assert np.array_equal(M.packed_position(pts, N), np.arange(len(pts)))


def test_level4_p1_count():
    # 969 P1 DoFs on one macro at level 4 (n = 16); 455 of them interior
    pts = M.lattice_points(16)
    assert len(pts) == 969
    interior = (pts.min(axis=1) > 0) & (pts.sum(axis=1) < 16)
    assert interior.sum() == 455


def _tetra(m):
    return m * (m + 1) * (m + 2) // 6 if m > 0 else 0


@pytest.mark.parametrize("level", range(0, 5))
def test_micro_tet_counts(level):
    """8^level micro-tets; per class the count the loop bounds B(o, n) of Section 5.1 give."""
    n = 2 ** level
    cls, tv = M.micro_tets(n)
    assert len(cls) == 8 ** level
    # sum_{z < B(n)} sum_{y < B(n-z)} B(n-z-y): white up n(n+1)(n+2)/6, blue/green (n-1)n(n+1)/6, white down (n-2)(n-1)n/6
    expect = [_tetra(n), _tetra(n - 1), _tetra(n - 1), _tetra(n - 1), _tetra(n - 1), _tetra(n - 2)]
    assert [int((cls == o).sum()) for o in range(6)] == expect
    # all vertices inside the macro
    assert tv.min() >= 0 and tv.sum(axis=2).max() <= n


def test_class_shapes_are_translates():
    """Within a class every micro-tet is a translate of the same index-space tetrahedron."""
    cls, tv = M.micro_tets(8)
    for o in range(6):
        rel = tv[cls == o] - tv[cls == o][:, :1, :]
        assert np.all(rel == rel[0])


@pytest.mark.parametrize("level", [1, 2, 3])
def test_volume_and_conformity(level):
    rng = np.random.default_rng(3)
    macro = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) + 0.2 * rng.standard_normal((4, 3))
    n = 2 ** level
    cls, tv = M.micro_tets(n)
    X = M.physical(macro, tv, n)
    vols = np.abs(np.linalg.det(np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1)))) / 6
    vmacro = abs(np.linalg.det((macro[1:] - macro[0]).T)) / 6
    assert np.all(vols > 0)
    assert np.isclose(vols.sum(), vmacro, rtol=1e-13)
    assert np.allclose(vols, vmacro / 8 ** level, rtol=1e-12)
    # every face shared by two micro-tets, or by one when it lies on a macro face
    faces = {}
    for t in tv:
        for a in range(4):
            f = tuple(sorted(tuple(p) for idx, p in enumerate(t) if idx != a))
            faces[f] = faces.get(f, 0) + 1
    for f, c in faces.items():
        f = np.array(f)
        on_macro_face = any(np.all(f[:, d] == 0) for d in range(3)) or np.all(f.sum(axis=1) == n)
        assert c == (1 if on_macro_face else 2)


def test_keys_identify_shared_points():
    v, t = W.cube6()
    for level in (1, 2, 3):
        N = 2 ** level
        pts = M.lattice_points(N)
        keys = np.concatenate([M.point_keys(t[m], pts, N) for m in range(len(t))])
        xyz = np.concatenate([M.physical(v[t[m]], pts, N) for m in range(len(t))])
        uniq, inv = np.unique(keys, axis=0, return_inverse=True)
        # (N+1)^3 distinct points on the unit cube lattice
        assert len(uniq) == (N + 1) ** 3
        # equal keys <=> equal physical position
        rep = np.zeros((len(uniq), 3))
        rep[inv] = xyz
        assert np.allclose(rep[inv], xyz, atol=1e-14)
        q = np.round(xyz * N).astype(np.int64)
        assert len(np.unique(q, axis=0)) == len(uniq)


def test_macro_mesh_validation():
    v, t = W.reference_tet()
    with pytest.raises(ValueError):
        M.MacroMesh(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 0, 1.0]]), t)
    with pytest.raises(ValueError):
        M.MacroMesh(np.vstack([v, [[0.3, 0.3, -1.0], [0.3, 0.3, -2.0]]]), np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]]))
    mm = M.MacroMesh(*W.cube6())
    assert mm.boundary_face.sum() == 12           # 6 cube faces x 2 triangles
    assert np.isclose(mm.volume(), 1.0)
    mm = M.MacroMesh(*W.cube48())
    assert mm.boundary_face.sum() == 6 * 4 * 2
