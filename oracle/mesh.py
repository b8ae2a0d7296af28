"""Hybrid tetrahedral grid: macro mesh, uniform refinement and the six micro-tet classes.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 2 and Fig. 3: every macro-tetrahedron with vertices P0..P3 is refined
uniformly ``level`` times; with n = 2^level the refined grid's vertices are
the index-space lattice points (i, j, k), i, j, k >= 0, i + j + k <= n, at
physical position P0 + (i/n)(P1-P0) + (j/n)(P2-P0) + (k/n)(P3-P0).  The
micro-tetrahedra fall into six classes, each a translate of one reference
tetrahedron in index space.  Section 5.1 gives the loop bounds of each class:
B(white up, m) = m, B(blue/green, m) = m - 1, B(white down, m) = m - 2.

Reading of the paper (its Fig. 3 is an image): the cube with origin c in index
space holds one white-up tet {000,100,010,001}, one white-down tet
{110,101,011,111} and the octahedron between them, which is split into four
tets around its (0,1,0)-(1,0,1) diagonal.  The four octahedron tets are the
blue/green up/down classes (their names are labels only).
Pinned by: micro-tet count 8^level, per-class counts from the loop bounds,
volume sum equal to the macro volume, face conformity (tests/test_oracle_mesh.py).
"""
from __future__ import annotations

import numpy as np

# Index-space vertex offsets of the six classes inside the cube at origin c.
CLASS_OFFSETS = np.array([
    [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]],   # white up
    [[0, 1, 0], [1, 0, 1], [1, 0, 0], [1, 1, 0]],   # octahedron tet ("blue up")
    [[0, 1, 0], [1, 0, 1], [1, 1, 0], [0, 1, 1]],   # octahedron tet ("blue down")
    [[0, 1, 0], [1, 0, 1], [0, 1, 1], [0, 0, 1]],   # octahedron tet ("green up")
    [[0, 1, 0], [1, 0, 1], [0, 0, 1], [1, 0, 0]],   # octahedron tet ("green down")
    [[1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]],   # white down
], dtype=np.int64)
CLASS_NAMES = ["white_up", "blue_up", "blue_down", "green_up", "green_down", "white_down"]
# B(o, m) = m - CLASS_SHRINK[o]  (Section 5.1)
CLASS_SHRINK = np.array([0, 1, 1, 1, 1, 2], dtype=np.int64)

# P2 local node order: the 4 vertices, then the edges in this order.
P2_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def lattice_size(N: int) -> int:
    """Number of lattice points with i + j + k <= N."""
    return (N + 1) * (N + 2) * (N + 3) // 6


def lattice_points(N: int) -> np.ndarray:
    """All lattice points (i, j, k), i+j+k <= N, with k slowest, then j, i fastest."""
    out = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            m = N - k - j
            row = np.empty((m + 1, 3), dtype=np.int64)
            row[:, 0] = np.arange(m + 1)
            row[:, 1] = j
            row[:, 2] = k
            out.append(row)
    return np.concatenate(out, axis=0)


def packed_position(pts: np.ndarray, N: int) -> np.ndarray:
    """Position of lattice points in the k-slowest / j / i-fastest enumeration.

    Written as the counts it is made of: all points of the planes below k,
    then all points of the rows below j inside plane k, then i.
    """
    pts = np.asarray(pts, dtype=np.int64)
    i, j, k = pts[..., 0], pts[..., 1], pts[..., 2]
    # points in planes k' < k: sum over k' of (m+1)(m+2)/2 with m = N - k'
    plane_sizes = np.array([(N - kk + 1) * (N - kk + 2) // 2 for kk in range(N + 1)], dtype=np.int64)
    plane_start = np.concatenate([[0], np.cumsum(plane_sizes)])
    m = N - k
    # rows j' < j in the plane: sum over j' of (m - j' + 1)
    row_start = j * (m + 1) - (j * (j - 1)) // 2
    return plane_start[k] + row_start + i


def micro_tets(n: int):
    """Micro-tets of one macro refined to n = 2^level intervals per edge.

    Returns (cls, verts): cls[e] in 0..5 and verts[e] the 4 index-space
    vertices, enumerated as in Algorithm 2 (sawtooth): class by class, and in
    each class z outermost, then y, x innermost, with exclusive upper bounds
    z < B(o, n), y < B(o, n - z), x < B(o, n - z - y).
    """
    cls_list, vert_list = [], []
    for o in range(6):
        s = int(CLASS_SHRINK[o])
        origins = []
        for z in range(max(n - s, 0)):
            for y in range(max(n - z - s, 0)):
                cnt = n - z - y - s
                if cnt <= 0:
                    continue
                row = np.empty((cnt, 3), dtype=np.int64)
                row[:, 0] = np.arange(cnt)
                row[:, 1] = y
                row[:, 2] = z
                origins.append(row)
        if not origins:
            continue
        origins = np.concatenate(origins, axis=0)
        cls_list.append(np.full(len(origins), o, dtype=np.int64))
        vert_list.append(origins[:, None, :] + CLASS_OFFSETS[o][None, :, :])
    return np.concatenate(cls_list), np.concatenate(vert_list, axis=0)


def physical(macro_xyz: np.ndarray, pts: np.ndarray, N: int) -> np.ndarray:
    """Physical position of lattice points (resolution N) of one macro with vertices macro_xyz (4,3)."""
    p0 = macro_xyz[0]
    e = macro_xyz[1:] - p0[None, :]
    pts = np.asarray(pts, dtype=np.float64)
    return p0 + (pts[..., 0:1] * e[0] + pts[..., 1:2] * e[1] + pts[..., 2:3] * e[2]) / N


def point_keys(macro_vids: np.ndarray, pts: np.ndarray, N: int) -> np.ndarray:
    """Exact global key of lattice points of one macro.

    A point's barycentric integer weights on the macro vertices are
    (N-i-j-k, i, j, k).  The key lists the (vertex id, weight) pairs with a
    nonzero weight, sorted by vertex id, padded with (-1, 0).  Two macros give
    the same key for a point exactly when the point is geometrically shared.
    """
    pts = np.asarray(pts, dtype=np.int64)
    w = np.stack([N - pts[:, 0] - pts[:, 1] - pts[:, 2], pts[:, 0], pts[:, 1], pts[:, 2]], axis=1)
    vid = np.broadcast_to(np.asarray(macro_vids, dtype=np.int64)[None, :], w.shape).copy()
    big = np.iinfo(np.int64).max
    vid_s = np.where(w > 0, vid, big)
    order = np.argsort(vid_s, axis=1, kind="stable")
    vid_sorted = np.take_along_axis(vid_s, order, axis=1)
    w_sorted = np.take_along_axis(w, order, axis=1)
    vid_sorted = np.where(vid_sorted == big, -1, vid_sorted)
    key = np.empty((len(pts), 8), dtype=np.int64)
    key[:, 0::2] = vid_sorted
    key[:, 1::2] = w_sorted
    return key


class MacroMesh:
    """Macro mesh with face classification (interior faces are shared by two macros).

    Raises ValueError for a degenerate macro (zero volume) or a face shared by
    more than two macros.
    """

    def __init__(self, vertices, tets):
        self.vertices = np.asarray(vertices, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        if self.tets.ndim != 2 or self.tets.shape[1] != 4:
            raise ValueError("tets must be (nt, 4)")
        if self.tets.min() < 0 or self.tets.max() >= len(self.vertices):
            raise ValueError("vertex index out of range")
        for t in self.tets:
            x = self.vertices[t]
            vol = abs(np.linalg.det((x[1:] - x[0]).T)) / 6.0
            scale = np.max(np.linalg.norm(x[1:] - x[0], axis=1)) ** 3
            if not vol > 1e-12 * scale:
                raise ValueError("degenerate macro-tetrahedron")
        faces = {}
        for m, t in enumerate(self.tets):
            for a in range(4):
                f = tuple(sorted(int(v) for idx, v in enumerate(t) if idx != a))
                faces.setdefault(f, []).append((m, a))
        for f, owners in faces.items():
            if len(owners) > 2:
                raise ValueError("non-manifold macro mesh (face shared by more than two macros)")
        self.faces = faces
        # boundary_face[m, a]: face of macro m opposite its local vertex a is on the domain boundary
        self.boundary_face = np.zeros((len(self.tets), 4), dtype=bool)
        for f, owners in faces.items():
            if len(owners) == 1:
                m, a = owners[0]
                self.boundary_face[m, a] = True

    @property
    def nmacro(self) -> int:
        return len(self.tets)

    def volume(self) -> float:
        x = self.vertices[self.tets]
        return float(np.abs(np.linalg.det(np.transpose(x[:, 1:] - x[:, :1], (0, 2, 1)))).sum() / 6.0)
