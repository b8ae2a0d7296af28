"""Global FE spaces and sparse operators of the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. 4.1: A = sum_T P_T A_T R_T.  The oracle forms A explicitly: each local
matrix (oracle.fe) is scattered into a global sparse matrix indexed by exact
DoF keys (oracle.mesh.point_keys), then y = A x is a sparse product.

Boundary conditions (the paper is silent; reading): DIRICHLET means
A_D = [[A_II, 0], [0, I]] -- rows of interior DoFs use interior columns only,
boundary rows return x; NEUMANN is the full A.  Boundary DoFs are those on
macro faces that belong to exactly one macro.

P2 DoFs are the lattice points of the doubled lattice (resolution 2n): a
micro-tet with index-space vertices p_a has its vertex DoFs at 2 p_a and its
edge DoFs at p_a + p_b.
Pinned by: symmetry, A.1 = 0 (Neumann), energy identities against exact
integrals, SPD Dirichlet matrix, cotangent formula at level 1, rigid-body
modes of the epsilon operator, linearity and finite differences of the
coefficient adjoint (tests/test_oracle_operator.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fe, quadrature
from .mesh import (MacroMesh, P2_EDGES, lattice_points, micro_tets, packed_position, physical, point_keys,
                   CLASS_OFFSETS, CLASS_SHRINK)


def local_nodes(tv: np.ndarray, degree: int) -> np.ndarray:
    """Lattice points (resolution degree*n) of the local nodes of micro-tets with vertices tv (E,4,3)."""
    if degree == 1:
        return tv
    edges = [tv[:, a] + tv[:, b] for a, b in P2_EDGES]
    return np.concatenate([2 * tv, np.stack(edges, axis=1)], axis=1)


class Space:
    """Continuous P1 or P2 Lagrange space on a macro mesh refined to ``level``."""

    def __init__(self, mesh: MacroMesh, level: int, degree: int):
        self.mesh, self.level, self.degree = mesh, level, degree
        self.n = 2 ** level
        self.N = self.n * degree
        self.pts = lattice_points(self.N)
        P = len(self.pts)
        keys = np.concatenate([point_keys(mesh.tets[m], self.pts, self.N) for m in range(mesh.nmacro)], axis=0)
        _, first, inv = np.unique(keys, axis=0, return_index=True, return_inverse=True)
        self.gid = inv.reshape(mesh.nmacro, P)
        self.ndof = int(inv.max()) + 1
        # coordinates of each DoF from its first occurrence
        owner_macro, owner_pos = np.divmod(first, P)
        self.coords = np.empty((self.ndof, 3))
        for m in range(mesh.nmacro):
            sel = owner_macro == m
            self.coords[sel] = physical(mesh.vertices[mesh.tets[m]], self.pts[owner_pos[sel]], self.N)
        # Dirichlet boundary: points on a boundary face (zero weight of the opposite vertex)
        w = np.stack([self.N - self.pts.sum(axis=1), self.pts[:, 0], self.pts[:, 1], self.pts[:, 2]], axis=1)
        self.boundary = np.zeros(self.ndof, dtype=bool)
        for m in range(mesh.nmacro):
            for a in range(4):
                if mesh.boundary_face[m, a]:
                    self.boundary[self.gid[m, w[:, a] == 0]] = True
        # micro-tets of every macro in sawtooth order, macro by macro
        cls, tv = micro_tets(self.n)
        nodes = local_nodes(tv, degree)
        pos = packed_position(nodes.reshape(-1, 3), self.N).reshape(nodes.shape[:2])
        self.elem_cls = np.tile(cls, mesh.nmacro)
        self.elem_macro = np.repeat(np.arange(mesh.nmacro), len(cls))
        self.elem_dofs = np.concatenate([self.gid[m][pos] for m in range(mesh.nmacro)], axis=0)
        self.elem_X = np.concatenate([physical(mesh.vertices[mesh.tets[m]], tv, self.n)
                                      for m in range(mesh.nmacro)], axis=0)

    @property
    def nloc(self) -> int:
        return 4 if self.degree == 1 else 10

    @property
    def interior(self) -> np.ndarray:
        return ~self.boundary

    def interpolate(self, f) -> np.ndarray:
        """Nodal interpolant of a function of points (ndof,3) -> (ndof,)."""
        return np.asarray(f(self.coords), dtype=np.float64)


def _scatter(space_rows, dofs_r, dofs_c, loc, nr, nc):
    E, a, b = loc.shape
    rows = np.repeat(dofs_r, b, axis=1).reshape(E, a, b)
    cols = np.repeat(dofs_c[:, None, :], a, axis=1)
    return sp.coo_matrix((loc.ravel(), (rows.ravel(), cols.ravel())), shape=(nr, nc)).tocsr()


def coefficient_at_quadrature(space: Space, coeff, quad_degree: int):
    """k at the mapped quadrature points of every element, (E, nq), or None for k = 1.

    coeff: ("const", value) | ("sin3",) | ("field", kspace, kvalues) | ("func", callable)
    """
    from workloads import sin3_coeff
    kind = coeff[0]
    if kind == "const":
        xi, w = quadrature.rule(quad_degree)
        return np.full((len(space.elem_X), len(w)), float(coeff[1]))
    if kind == "sin3":
        return sin3_coeff
    if kind == "func":
        return coeff[1]
    if kind == "field":
        kspace, kvals = coeff[1], np.asarray(coeff[2], dtype=np.float64)
        xi, _ = quadrature.rule(quad_degree)
        return fe.field_at_points(kspace.degree, xi, kvals[kspace.elem_dofs])
    raise ValueError(kind)


def diffusion_matrix(space: Space, coeff=("const", 1.0), quad_degree: int = 2, bc: str = "dirichlet"):
    """Global diffusion matrix (Eq. P1 / Eq. P2V) with the given coefficient and boundary mode."""
    kq = coefficient_at_quadrature(space, coeff, quad_degree)
    loc = fe.diffusion_local(space.elem_X, space.degree, quad_degree, kq)
    A = _scatter(None, space.elem_dofs, space.elem_dofs, loc, space.ndof, space.ndof)
    return apply_bc(A, space.boundary, bc)


def apply_bc(A, boundary, bc: str):
    if bc == "neumann":
        return A
    inner = sp.diags((~boundary).astype(np.float64))
    return (inner @ A @ inner + sp.diags(boundary.astype(np.float64))).tocsr()


def vector_boundary(space: Space) -> np.ndarray:
    return np.repeat(space.boundary, 3)


def epsilon_matrix(space: Space, mu, quad_degree: int = 4, bc: str = "dirichlet"):
    """Global P2-vector epsilon matrix, DoF index 3*gid + component; mu as in coefficient_at_quadrature."""
    assert space.degree == 2
    mq = coefficient_at_quadrature(space, mu, quad_degree)
    loc = fe.epsilon_local(space.elem_X, quad_degree, mq)
    vd = (3 * space.elem_dofs[:, :, None] + np.arange(3)[None, None, :]).reshape(len(space.elem_dofs), 30)
    A = _scatter(None, vd, vd, loc, 3 * space.ndof, 3 * space.ndof)
    return apply_bc(A, vector_boundary(space), bc)


def diffusion_coeff_adjoint(space: Space, kspace: Space, u, g, quad_degree: int = 2, bc: str = "dirichlet"):
    """dk_m = g^T (dA/dk_m) u for a P1/P2 coefficient field (linear in k).

    With DIRICHLET the derivative of A_D only touches interior rows and
    columns, so u and g enter with their boundary entries set to zero.
    """
    u = np.asarray(u, dtype=np.float64).copy()
    g = np.asarray(g, dtype=np.float64).copy()
    if bc == "dirichlet":
        u[space.boundary] = 0.0
        g[space.boundary] = 0.0
    K = fe.diffusion_coeff_derivative(space.elem_X, space.degree, kspace.degree, quad_degree)
    ue = u[space.elem_dofs]
    ge = g[space.elem_dofs]
    contrib = np.einsum("ei,emij,ej->em", ge, K, ue)
    dk = np.zeros(kspace.ndof)
    np.add.at(dk, kspace.elem_dofs, contrib)
    return dk


def epsilon_coeff_adjoint(space: Space, u, g, quad_degree: int = 4, bc: str = "dirichlet"):
    """dmu_m = g^T (dA/dmu_m) u for a P2 viscosity field; u, g of length 3*ndof."""
    u = np.asarray(u, dtype=np.float64).copy()
    g = np.asarray(g, dtype=np.float64).copy()
    if bc == "dirichlet":
        vb = vector_boundary(space)
        u[vb] = 0.0
        g[vb] = 0.0
    K = fe.epsilon_coeff_derivative(space.elem_X, quad_degree)
    vd = (3 * space.elem_dofs[:, :, None] + np.arange(3)[None, None, :]).reshape(len(space.elem_dofs), 30)
    contrib = np.einsum("ei,emij,ej->em", g[vd], K, u[vd])
    dk = np.zeros(space.ndof)
    np.add.at(dk, space.elem_dofs, contrib)
    return dk


# ---------------------------------------------------------------------------
# Sampled rows for a single macro (sizes too large to assemble)
# ---------------------------------------------------------------------------

def sampled_diffusion_rows(macro_xyz, level: int, degree: int, coeff, quad_degree: int, bc: str,
                           x_packed: np.ndarray, sample_pts: np.ndarray) -> np.ndarray:
    """(A x) at the given lattice points of ONE macro whose faces are all domain boundary.

    Computes, point by point, the sum over the micro-tets that contain the
    point of row(point) of A_T times the local x, with the same element
    matrices as the assembled operator.  coeff: ("const", v) | ("sin3",) |
    ("field", degree_k, k_packed) with k on the same single macro.
    """
    n = 2 ** level
    N = degree * n
    macro_xyz = np.asarray(macro_xyz, dtype=np.float64)
    x_packed = np.asarray(x_packed, dtype=np.float64)

    def on_boundary(p):
        return (p[..., 0] == 0) | (p[..., 1] == 0) | (p[..., 2] == 0) | (p.sum(axis=-1) == N)

    out = np.empty(len(sample_pts))
    for s, p in enumerate(np.asarray(sample_pts, dtype=np.int64)):
        if bc == "dirichlet" and on_boundary(p):
            out[s] = x_packed[packed_position(p[None], N)[0]]
            continue
        tets, rows = [], []
        lo = (p + degree - 1) // degree - 1
        hi = p // degree
        for cz in range(max(lo[2], 0), hi[2] + 1):
            for cy in range(max(lo[1], 0), hi[1] + 1):
                for cx in range(max(lo[0], 0), hi[0] + 1):
                    c = np.array([cx, cy, cz])
                    for o in range(6):
                        if c.sum() > n - 1 - CLASS_SHRINK[o]:
                            continue
                        tv = c[None, :] + CLASS_OFFSETS[o]
                        nodes = local_nodes(tv[None], degree)[0]
                        hit = np.nonzero(np.all(nodes == p[None, :], axis=1))[0]
                        if len(hit):
                            tets.append(tv)
                            rows.append(hit[0])
        tv = np.array(tets)
        X = physical(macro_xyz, tv, n)
        nodes = local_nodes(tv, degree)
        pos = packed_position(nodes.reshape(-1, 3), N).reshape(nodes.shape[:2])
        if coeff[0] == "const":
            kq = np.full((len(tv), len(quadrature.rule(quad_degree)[1])), float(coeff[1]))
        elif coeff[0] == "sin3":
            from workloads import sin3_coeff
            kq = sin3_coeff
        elif coeff[0] == "field":
            dk, kp = coeff[1], np.asarray(coeff[2], dtype=np.float64)
            kpos = packed_position(local_nodes(tv, dk).reshape(-1, 3), dk * n).reshape(len(tv), -1)
            xi, _ = quadrature.rule(quad_degree)
            kq = fe.field_at_points(dk, xi, kp[kpos])
        else:
            raise ValueError(coeff[0])
        loc = fe.diffusion_local(X, degree, quad_degree, kq)
        xl = x_packed[pos]
        if bc == "dirichlet":
            xl = np.where(on_boundary(nodes), 0.0, xl)
        out[s] = sum(loc[e, rows[e], :] @ xl[e] for e in range(len(tv)))
    return out
