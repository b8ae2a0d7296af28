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
    """dmu_m = g^T (dA/dmu_m) u for a P2 viscosity field; u, g of length 3*ndof, or (3*ndof, nrhs)
    for a batch, in which case the result is summed over the right-hand sides."""
    u = np.asarray(u, dtype=np.float64).copy()
    g = np.asarray(g, dtype=np.float64).copy()
    if u.ndim == 1:
        u, g = u[:, None], g[:, None]
    if bc == "dirichlet":
        vb = vector_boundary(space)
        u[vb] = 0.0
        g[vb] = 0.0
    K = fe.epsilon_coeff_derivative(space.elem_X, quad_degree)
    vd = (3 * space.elem_dofs[:, :, None] + np.arange(3)[None, None, :]).reshape(len(space.elem_dofs), 30)
    contrib = np.einsum("eir,emij,ejr->em", g[vd], K, u[vd], optimize=True)
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


def point_copies(mesh: MacroMesh, m: int, p, N: int):
    """Every (macro, local lattice point) that stores the point p (resolution N) of macro m.

    Exact: the point's global key (nonzero barycentric weights on global vertex ids) is matched
    against each macro's vertex list; a macro holds the point when it has all the key's vertices.
    """
    key = point_keys(mesh.tets[m], np.asarray(p, dtype=np.int64)[None], N)[0]
    vids, wts = key[0::2], key[1::2]
    out = []
    for m2 in range(mesh.nmacro):
        t2 = [int(v) for v in mesh.tets[m2]]
        if not all(int(v) in t2 for v, w in zip(vids, wts) if w > 0):
            continue
        w4 = np.zeros(4, dtype=np.int64)
        for v, w in zip(vids, wts):
            if w > 0:
                w4[t2.index(int(v))] = w
        out.append((m2, w4[1:].copy()))
    return out


def _on_dirichlet(mesh: MacroMesh, m: int, pts, N: int):
    """Lattice points (k, 3) or one point (3,) of macro m that lie on the domain boundary.

    A point lies in the relative interior of the face spanned by the macro vertices with a
    nonzero barycentric weight (its support); it is on a boundary face F exactly when its support
    is a subset of F's three vertices.  This also catches points on a macro edge or vertex that
    touches the boundary while none of that macro's own faces is boundary.
    """
    pts = np.asarray(pts, dtype=np.int64)
    one = pts.ndim == 1
    pts = pts.reshape(-1, 3)
    w = np.stack([N - pts.sum(axis=-1), pts[:, 0], pts[:, 1], pts[:, 2]], axis=-1)
    tet = [int(v) for v in mesh.tets[m]]
    hit = np.zeros(len(pts), dtype=bool)
    for face, owners in mesh.faces.items():
        if len(owners) != 1:
            continue
        outside = np.array([v not in face for v in tet])
        hit |= ~np.any((w > 0) & outside[None, :], axis=1)
    return bool(hit[0]) if one else hit


def incident_tets(q, n: int, degree: int):
    """Micro-tets of one macro (n intervals per edge) that have the lattice point q (resolution
    degree*n) as a local node: their index-space vertices (E, 4, 3) and q's local node number."""
    q = np.asarray(q, dtype=np.int64)
    lo = (q + degree - 1) // degree - 1
    hi = q // degree
    tets, rows = [], []
    for cz in range(max(lo[2], 0), hi[2] + 1):
        for cy in range(max(lo[1], 0), hi[1] + 1):
            for cx in range(max(lo[0], 0), hi[0] + 1):
                c = np.array([cx, cy, cz])
                for o in range(6):
                    if c.sum() > n - 1 - CLASS_SHRINK[o]:
                        continue
                    tv = c[None, :] + CLASS_OFFSETS[o]
                    hit = np.nonzero(np.all(local_nodes(tv[None], degree)[0] == q[None, :], axis=1))[0]
                    if len(hit):
                        tets.append(tv)
                        rows.append(int(hit[0]))
    return np.array(tets), np.array(rows)


def _epsilon_rows_of_copy(mesh, m, q, level, mu_packed, quad_degree):
    """Micro-tets of macro m around its local P2 point q: local nodes, packed positions of the
    nodes, q's row number and the local epsilon matrices with mu interpolated from mu_packed."""
    n, N = 2 ** level, 2 ** (level + 1)
    P = (N + 1) * (N + 2) * (N + 3) // 6
    tv, rows = incident_tets(q, n, 2)
    X = physical(mesh.vertices[mesh.tets[m]], tv, n)
    nodes = local_nodes(tv, 2)
    pos = packed_position(nodes.reshape(-1, 3), N).reshape(nodes.shape[:2])
    xi, _ = quadrature.rule(quad_degree)
    muq = fe.field_at_points(2, xi, np.asarray(mu_packed)[m * P + pos])
    return X, nodes, rows, muq


def sampled_epsilon_rows(mesh: MacroMesh, level: int, mu_packed: np.ndarray, x_at, samples, quad_degree: int = 4,
                         bc: str = "dirichlet") -> np.ndarray:
    """(A x) of the P2 vector epsilon operator at sampled points of a multi-macro mesh.

    Point by point: the sum, over every macro that stores the point and every micro-tet of that
    macro around it, of the point's three rows of the local matrix (fe.epsilon_local, mu
    interpolated from that macro's copy of the P2 field mu_packed) times the local x.  Points on
    the Dirichlet boundary return x; with DIRICHLET, boundary nodes enter with x = 0.
    x_at(m, pts) gives x at lattice points (k, 3) of macro m as (k, 3, nrhs); samples is a list
    of (macro, lattice point).  Returns (len(samples), 3, nrhs).
    """
    N = 2 ** (level + 1)
    out = []
    for m, p in samples:
        copies = point_copies(mesh, m, p, N)
        if bc == "dirichlet" and any(_on_dirichlet(mesh, m2, q, N) for m2, q in copies):
            out.append(np.asarray(x_at(m, np.asarray(p)[None]))[0])
            continue
        acc = 0.0
        for m2, q in copies:
            X, nodes, rows, muq = _epsilon_rows_of_copy(mesh, m2, q, level, mu_packed, quad_degree)
            loc = fe.epsilon_local(X, quad_degree, muq)                       # (E, 30, 30)
            xl = np.asarray(x_at(m2, nodes.reshape(-1, 3)), dtype=np.float64)  # (E*10, 3, nrhs)
            nrhs = xl.shape[-1]
            if bc == "dirichlet":
                xl = np.where(_on_dirichlet(mesh, m2, nodes.reshape(-1, 3), N)[:, None, None], 0.0, xl)
            xl = xl.reshape(len(X), 30, nrhs)
            for e in range(len(X)):
                acc = acc + loc[e, 3 * rows[e]:3 * rows[e] + 3, :] @ xl[e]
        out.append(acc)
    return np.array(out)


def sampled_epsilon_adjoint(mesh: MacroMesh, level: int, u_at, g_at, samples, quad_degree: int = 4,
                            bc: str = "dirichlet") -> np.ndarray:
    """dmu_m = sum_r g_r^T (dA/dmu_m) u_r at sampled P2 points m of a multi-macro mesh.

    The same sum over macros and micro-tets as sampled_epsilon_rows, with the derivative of the
    local matrix in the nodal value of mu at the point (fe.epsilon_coeff_derivative); with
    DIRICHLET, u and g enter with their boundary entries set to zero.  Returns (len(samples),).
    """
    N = 2 ** (level + 1)
    n = 2 ** level
    out = []
    for m, p in samples:
        acc = 0.0
        for m2, q in point_copies(mesh, m, p, N):
            tv, rows = incident_tets(q, n, 2)
            X = physical(mesh.vertices[mesh.tets[m2]], tv, n)
            nodes = local_nodes(tv, 2).reshape(-1, 3)
            K = fe.epsilon_coeff_derivative(X, quad_degree)                   # (E, 10, 30, 30)
            ul = np.asarray(u_at(m2, nodes), dtype=np.float64)
            gl = np.asarray(g_at(m2, nodes), dtype=np.float64)
            if bc == "dirichlet":
                zb = _on_dirichlet(mesh, m2, nodes, N)[:, None, None]
                ul = np.where(zb, 0.0, ul)
                gl = np.where(zb, 0.0, gl)
            nrhs = ul.shape[-1]
            ul = ul.reshape(len(X), 30, nrhs)
            gl = gl.reshape(len(X), 30, nrhs)
            for e in range(len(X)):
                acc += float(np.einsum("ir,ij,jr->", gl[e], K[e, rows[e]], ul[e]))
        out.append(acc)
    return np.array(out)


# ---------------------------------------------------------------------------
# Nedelec edge space (Eq. N1)
# ---------------------------------------------------------------------------

# Canonical index-space direction of the edge whose doubled-lattice midpoint has this parity.
EDGE_DIRS = {(1, 0, 0): (1, 0, 0), (0, 1, 0): (0, 1, 0), (0, 0, 1): (0, 0, 1), (1, 1, 0): (1, -1, 0),
             (1, 0, 1): (1, 0, -1), (0, 1, 1): (0, 1, -1), (1, 1, 1): (1, -1, 1)}


class EdgeSpace:
    """One DoF per micro-edge: the tangential integral of u along the edge.

    Global orientation: from the endpoint with the smaller global vertex number to the larger.
    The library's packed layout uses the doubled lattice of each macro (the P2 layout); an edge's
    entry is its tangential integral along the macro's canonical index direction of that edge
    (EDGE_DIRS), i.e. local_sign times the global value; vertex entries are zero.
    """

    def __init__(self, mesh: MacroMesh, level: int):
        self.mesh, self.level = mesh, level
        self.n = n = 2 ** level
        self.V1 = Space(mesh, level, 1)                                # vertices (global numbering)
        pts2 = lattice_points(2 * n)
        par = pts2 % 2
        self.edge_pos = np.nonzero(par.any(axis=1))[0]                 # packed positions of edge points
        ep = pts2[self.edge_pos]
        d = np.array([EDGE_DIRS[tuple(q)] for q in par[self.edge_pos]])
        tail, head = (ep - d) // 2, (ep + d) // 2
        vpos_t = packed_position(tail, n)
        vpos_h = packed_position(head, n)
        keys = np.concatenate([point_keys(mesh.tets[m], ep, 2 * n) for m in range(mesh.nmacro)], axis=0)
        _, inv = np.unique(keys, axis=0, return_inverse=True)
        E = len(ep)
        self.gid = inv.reshape(mesh.nmacro, E)
        self.ndof = int(inv.max()) + 1
        vt = np.stack([self.V1.gid[m][vpos_t] for m in range(mesh.nmacro)])
        vh = np.stack([self.V1.gid[m][vpos_h] for m in range(mesh.nmacro)])
        self.local_sign = np.where(vt < vh, 1.0, -1.0)                 # macro-local vs global orientation
        # global endpoints (tail -> head in global orientation)
        self.g_tail = np.empty(self.ndof, dtype=np.int64)
        self.g_head = np.empty(self.ndof, dtype=np.int64)
        self.g_tail[self.gid.reshape(-1)] = np.minimum(vt, vh).reshape(-1)
        self.g_head[self.gid.reshape(-1)] = np.maximum(vt, vh).reshape(-1)
        # Dirichlet (tangential trace): edges whose midpoint lies on a boundary face
        w = np.stack([2 * n - ep.sum(axis=1), ep[:, 0], ep[:, 1], ep[:, 2]], axis=1)
        self.boundary = np.zeros(self.ndof, dtype=bool)
        for m in range(mesh.nmacro):
            for a in range(4):
                if mesh.boundary_face[m, a]:
                    self.boundary[self.gid[m, w[:, a] == 0]] = True
        # elements: the micro-tets of the P1 space, their 6 edges and orientation signs
        Vg = self.V1.elem_dofs                                          # (nel, 4) global vertex ids
        cls, tv = micro_tets(n)
        mids = np.stack([tv[:, a] + tv[:, b] for a, b in P2_EDGES], axis=1)   # doubled midpoints
        edge_index = -np.ones(len(pts2), dtype=np.int64)
        edge_index[self.edge_pos] = np.arange(E)
        loc = edge_index[packed_position(mids.reshape(-1, 3), 2 * n)].reshape(len(tv), 6)
        self.elem_dofs = np.concatenate([self.gid[m][loc] for m in range(mesh.nmacro)], axis=0)
        a_idx = np.array([a for a, b in P2_EDGES])
        b_idx = np.array([b for a, b in P2_EDGES])
        self.elem_sign = np.where(Vg[:, a_idx] < Vg[:, b_idx], 1.0, -1.0)
        self.elem_X = self.V1.elem_X

    def interpolate_field(self, u) -> np.ndarray:
        """Tangential integrals (global orientation) of a vector field u(points) -> (npts, 3),
        by the 3-point Gauss rule on each edge (exact for fields of degree <= 5 along the edge)."""
        xt = self.V1.coords[self.g_tail]
        xh = self.V1.coords[self.g_head]
        g = np.array([0.5 - np.sqrt(15) / 10, 0.5, 0.5 + np.sqrt(15) / 10])
        gw = np.array([5.0, 8.0, 5.0]) / 18.0
        out = np.zeros(self.ndof)
        for t, wt in zip(g, gw):
            out += wt * np.einsum("ed,ed->e", u(xt + t * (xh - xt)), xh - xt)
        return out


def n1_matrix(space: EdgeSpace, alpha, beta, quad_degree: int = 4, bc: str = "dirichlet"):
    """Global curl-curl + mass matrix (Eq. N1); alpha / beta as in coefficient_at_quadrature
    (("const", v), ("func", f) or ("field", p1space, values))."""
    P1 = space.V1
    aq = coefficient_at_quadrature(P1, alpha, quad_degree)
    bq = coefficient_at_quadrature(P1, beta, quad_degree)
    loc = fe.n1_local(space.elem_X, quad_degree, aq, bq)
    s = space.elem_sign
    loc = loc * s[:, :, None] * s[:, None, :]
    A = _scatter(None, space.elem_dofs, space.elem_dofs, loc, space.ndof, space.ndof)
    return apply_bc(A, space.boundary, bc)


def n1_gradient(space: EdgeSpace) -> sp.csr_matrix:
    """Discrete gradient: (G p)_e = p(head) - p(tail) in the global orientation."""
    E = space.ndof
    rows = np.concatenate([np.arange(E), np.arange(E)])
    cols = np.concatenate([space.g_head, space.g_tail])
    vals = np.concatenate([np.ones(E), -np.ones(E)])
    return sp.coo_matrix((vals, (rows, cols)), shape=(E, space.V1.ndof)).tocsr()
