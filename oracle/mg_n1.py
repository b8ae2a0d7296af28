"""Multigrid for the Nedelec curl-curl + mass operator (Eq. N1): transfers, hybrid smoother, FMG.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 8 solves the N1 problem by full multigrid whose smoother is Hiptmair's hybrid smoother: a
smoothing step on the edge operator followed by one in the space of discrete gradients of P1
functions, on which the curl-curl part vanishes and plain edge smoothers do not reduce the error.
Readings where the paper is silent:
  * prolongation: the tangential integrals of the coarse Whitney field along the fine edges (the
    spaces are nested because refinement is uniform); restriction is its transpose;
  * edge smoother: the Chebyshev step of ``oracle.mg`` on D^{-1} A; nodal smoother: the same on
    A_p = G^T A G over the interior vertices (G the discrete gradient);
  * one hybrid step: edge Chebyshev, then r_p = G^T (b - A x), p = Chebyshev(A_p, r_p, 0),
    x <- x + G p; the V-cycle, FMG and stopping rule are those of ``oracle.mg``.
Pinned by: P reproduces the fine interpolant of the fields the coarse space holds exactly
(constants and rotations), P G_c = G_f P_1 (coarse gradients stay gradients), the V-cycle
contraction stays below a bound as the level grows, and FMG reaches the O(h) discretisation error
(tests/test_oracle_mg_n1.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp

from . import fe
from .assemble import EDGE_DIRS, EdgeSpace, n1_gradient, n1_matrix
from .mesh import CLASS_OFFSETS, P2_EDGES, lattice_points, packed_position
from .mg import _locate, chebyshev, power_iteration


def edge_prolongation(coarse: EdgeSpace, fine: EdgeSpace) -> sp.csr_matrix:
    """P: coarse edge DoFs -> the fine edge DoFs of the same Whitney field (fine.ndof x coarse.ndof).

    A fine edge lies in one coarse micro-tet (or on faces shared by several, where the tangential
    trace agrees); Whitney fields are linear there, so the integral along the edge is the value at
    its midpoint times the edge vector.  Everything is computed in the macro's index space, where
    line integrals of the affine-mapped basis are the same as in physical space.
    """
    assert fine.level == coarse.level + 1
    n_c = coarse.n
    pts_f = lattice_points(2 * fine.n)
    E = len(fine.edge_pos)
    _, first = np.unique(fine.gid.reshape(-1), return_index=True)
    m_of, k_of = np.divmod(first, E)
    cpos_to_edge = -np.ones(len(lattice_points(2 * n_c)), dtype=np.int64)
    cpos_to_edge[coarse.edge_pos] = np.arange(len(coarse.edge_pos))
    rows, cols, vals = [], [], []
    for m in range(fine.mesh.nmacro):
        sel = np.nonzero(m_of == m)[0]                                # fine global edges owned here
        if len(sel) == 0:
            continue
        k = k_of[sel]
        ep = pts_f[fine.edge_pos[k]]                                  # doubled fine lattice coordinates
        d = np.array([EDGE_DIRS[tuple(p)] for p in ep % 2], dtype=np.float64)
        q = ep / 4.0                                                  # midpoint in coarse index space
        t = d / 2.0                                                   # edge vector (canonical direction)
        cls, org, xi = _locate(q, n_c)
        V = org[:, None, :] + CLASS_OFFSETS[cls]                      # coarse micro-tet vertices (F,4,3)
        J = np.transpose(V[:, 1:, :] - V[:, :1, :], (0, 2, 1)).astype(np.float64)
        G = np.einsum("fji,aj->fai", np.linalg.inv(J), fe.GRAD_BARY)  # index-space grad lambda_a
        lam = fe.bary(xi)                                             # (F,4)
        vgid = coarse.V1.gid[m][packed_position(V.reshape(-1, 3), n_c)].reshape(len(sel), 4)
        sign_f = fine.local_sign[m, k]
        for a, b in P2_EDGES:
            phi = lam[:, a, None] * G[:, b, :] - lam[:, b, None] * G[:, a, :]
            val = np.einsum("fd,fd->f", phi, t) * sign_f * np.where(vgid[:, a] < vgid[:, b], 1.0, -1.0)
            mid = V[:, a, :] + V[:, b, :]                             # doubled coarse coordinates
            ce = coarse.gid[m][cpos_to_edge[packed_position(mid, 2 * n_c)]]
            rows.append(sel)
            cols.append(ce)
            vals.append(val)
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    keep = np.abs(vals) > 1e-14
    M = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(fine.ndof, coarse.ndof)).tocsr()
    M.sum_duplicates()
    return M


class N1Hierarchy:
    """Edge spaces, Dirichlet operators, gradient spaces and transfers on levels 0..L."""

    def __init__(self, mesh, L: int, alpha=("const", 1.0), beta=("const", 1.0), cheb_order: int = 2,
                 power_iters: int = 15, seed: int = 0):
        self.L = L
        self.spaces = [EdgeSpace(mesh, l) for l in range(L + 1)]
        self.A = [n1_matrix(s, alpha, beta, 4, "dirichlet") for s in self.spaces]
        self.dinv = [1.0 / A.diagonal() for A in self.A]
        self.P = [None] + [edge_prolongation(self.spaces[l - 1], self.spaces[l]) for l in range(1, L + 1)]
        self.order = cheb_order
        self.G, self.Ap, self.dinv_p, self.lam, self.lam_p = [], [], [], [], []
        for l, s in enumerate(self.spaces):
            Gi = n1_gradient(s)[:, np.nonzero(s.V1.interior)[0]].tocsr()   # gradients of interior hats
            Ap = (Gi.T @ self.A[l] @ Gi).tocsr()
            self.G.append(Gi)
            self.Ap.append(Ap)
            self.dinv_p.append(1.0 / Ap.diagonal() if Ap.shape[0] else np.zeros(0))
            rng = np.random.default_rng(seed)
            v0 = rng.uniform(-1.0, 1.0, s.ndof)
            v0[s.boundary] = 0.0
            self.lam.append(power_iteration(self.A[l], self.dinv[l], v0, power_iters)
                            if (~s.boundary).any() else 1.0)
            self.lam_p.append(power_iteration(Ap, self.dinv_p[-1], rng.uniform(-1.0, 1.0, Ap.shape[0]), power_iters)
                              if Ap.shape[0] else 1.0)
        self.coarse_lu = scipy.linalg.lu_factor(self.A[0].toarray())

    def smooth(self, l: int, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        """One hybrid step: Chebyshev on the edges, then on the gradients of the interior vertices."""
        A = self.A[l]
        x = chebyshev(A, self.dinv[l], b, x, self.lam[l], self.order)
        if self.Ap[l].shape[0]:
            rp = self.G[l].T @ (b - A @ x)
            p = chebyshev(self.Ap[l], self.dinv_p[l], rp, np.zeros_like(rp), self.lam_p[l], self.order)
            x = x + self.G[l] @ p
        return x

    def vcycle(self, l: int, b: np.ndarray, x: np.ndarray, nu1: int = 2, nu2: int = 2) -> np.ndarray:
        if l == 0:
            return scipy.linalg.lu_solve(self.coarse_lu, b)
        s = self.spaces[l]
        for _ in range(nu1):
            x = self.smooth(l, b, x)
        r = b - self.A[l] @ x
        r[s.boundary] = 0.0
        rc = self.P[l].T @ r
        rc[self.spaces[l - 1].boundary] = 0.0
        ec = self.vcycle(l - 1, rc, np.zeros_like(rc), nu1, nu2)
        ec[self.spaces[l - 1].boundary] = 0.0
        x = x + self.P[l] @ ec
        for _ in range(nu2):
            x = self.smooth(l, b, x)
        return x

    def fmg(self, b, nu1: int = 2, nu2: int = 2, tol: float = 1e-10, max_cycles: int = 50):
        """FMG then V-cycles on the finest level for the fine right-hand side b (coarse right-hand
        sides by restriction, boundary rows zero); returns (x, V-cycles after FMG, residual history)."""
        bs = [None] * (self.L + 1)
        bs[self.L] = np.asarray(b, dtype=np.float64).copy()
        bs[self.L][self.spaces[self.L].boundary] = 0.0
        for l in range(self.L, 0, -1):
            bs[l - 1] = self.P[l].T @ bs[l]
            bs[l - 1][self.spaces[l - 1].boundary] = 0.0
        x = scipy.linalg.lu_solve(self.coarse_lu, bs[0])
        for l in range(1, self.L + 1):
            x = self.P[l] @ x
            x = self.vcycle(l, bs[l], x, nu1, nu2)
        A, b = self.A[self.L], bs[self.L]
        nb = np.linalg.norm(b)
        hist = [np.linalg.norm(b - A @ x) / nb]
        cycles = 0
        while hist[-1] > tol and cycles < max_cycles:
            x = self.vcycle(self.L, b, x, nu1, nu2)
            cycles += 1
            hist.append(np.linalg.norm(b - A @ x) / nb)
        return x, cycles, hist


def load_vector(S: EdgeSpace, f, quad_degree: int = 5) -> np.ndarray:
    """b_e = integral of f . phi_e over the domain for a vector field f of points (n, 3) -> (n, 3),
    by element quadrature with the Whitney functions phi_e (global orientation); boundary entries
    (tangential trace) zero."""
    from . import quadrature
    from .mesh import P2_EDGES as EDGES
    xi, w = quadrature.rule(quad_degree)
    lam = fe.bary(xi)
    J, adet, Jinv = fe.jacobians(S.elem_X)
    G = np.einsum("eji,aj->eai", Jinv, fe.GRAD_BARY)
    pts = fe.map_points(S.elem_X, J, xi)
    fq = f(pts.reshape(-1, 3)).reshape(len(S.elem_X), len(w), 3)
    b = np.zeros(S.ndof)
    for e, (a, c) in enumerate(EDGES):
        phi = lam[None, :, a, None] * G[:, None, c, :] - lam[None, :, c, None] * G[:, None, a, :]
        np.add.at(b, S.elem_dofs[:, e], np.einsum("k,q,kqd,kqd->k", adet, w, fq, phi) * S.elem_sign[:, e])
    b[S.boundary] = 0.0
    return b
