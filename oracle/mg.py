"""Geometric multigrid of the oracle: transfers, Chebyshev smoother, V-cycle, FMG.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 8: full multigrid with V-cycles per level, a Chebyshev smoother of
order 2 (Adams et al. 2003; Baker et al. 2011) and an exact coarse solve.
Readings where the paper is silent:
  * prolongation P evaluates the coarse FE function at the fine nodes (the
    spaces are nested because refinement is uniform); restriction is P^T;
    residuals are restricted with their boundary rows zero and the coarse
    correction keeps zero boundary values;
  * the smoother is the Chebyshev iteration on D^{-1} A over
    [lo * lam, hi * lam] with lo = 0.1, hi = 1.1 and lam from power
    iteration on D^{-1} A; one smoothing step = one Chebyshev polynomial of
    the given order (order applications of A);
  * FMG solves level 0 exactly, then per level prolongs the previous
    solution and runs one V(nu1, nu2); further V-cycles run until
    ||b - A x||_2 / ||b||_2 <= tol; the coarse levels' right-hand sides are
    restrictions of the fine one.
Pinned by: P reproduces the fine interpolant of coarse-exact polynomials,
R = P^T, the V-cycle contraction factor stays below a fixed bound as the level
grows, and the discretisation error falls at the textbook rate
(tests/test_oracle_mg.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.linalg

from . import fe, quadrature
from .assemble import Space, diffusion_matrix
from .mesh import CLASS_OFFSETS, CLASS_SHRINK


def _locate(q: np.ndarray, n_c: int):
    """For index-space points q (F,3) at the coarse level, a containing coarse micro-tet.

    Returns (class, origin (F,3), reference coordinates xi (F,3)).
    """
    F = len(q)
    found = np.zeros(F, dtype=bool)
    cls = np.zeros(F, dtype=np.int64)
    org = np.zeros((F, 3), dtype=np.int64)
    xi = np.zeros((F, 3))
    base = np.floor(q).astype(np.int64)
    for d in np.array([[a, b, c] for a in (0, -1) for b in (0, -1) for c in (0, -1)]):
        c0 = base + d[None, :]
        for o in range(6):
            valid = np.all(c0 >= 0, axis=1) & (c0.sum(axis=1) <= n_c - 1 - CLASS_SHRINK[o])
            V = c0[:, None, :] + CLASS_OFFSETS[o][None, :, :]           # (F,4,3)
            J = np.transpose(V[:, 1:, :] - V[:, :1, :], (0, 2, 1)).astype(np.float64)
            loc = np.linalg.solve(J, (q - V[:, 0, :])[:, :, None])[:, :, 0]
            lam = np.concatenate([1.0 - loc.sum(axis=1, keepdims=True), loc], axis=1)
            inside = valid & np.all(lam >= -1e-12, axis=1) & ~found
            cls[inside] = o
            org[inside] = c0[inside]
            xi[inside] = loc[inside]
            found |= inside
    assert found.all(), "point location failed"
    return cls, org, xi


def prolongation(coarse: Space, fine: Space) -> sp.csr_matrix:
    """P: coarse FE function -> its values at the fine nodes (fine.ndof x coarse.ndof)."""
    assert fine.level == coarse.level + 1 and fine.degree == coarse.degree
    deg, n_c = fine.degree, coarse.n
    from .assemble import local_nodes
    from .mesh import packed_position
    P = len(fine.pts)
    # one owner copy per fine DoF
    _, first = np.unique(fine.gid.reshape(-1), return_index=True)
    m_of, p_of = np.divmod(first, P)
    rows, cols, vals = [], [], []
    for m in range(fine.mesh.nmacro):
        sel = np.nonzero(m_of == m)[0]
        if len(sel) == 0:
            continue
        q = fine.pts[p_of[sel]].astype(np.float64) / (2.0 * deg)   # coarse index space
        cls, org, xi = _locate(q, n_c)
        tv = org[:, None, :] + CLASS_OFFSETS[cls]                    # (F,4,3)
        nodes = local_nodes(tv, deg)
        cpos = packed_position(nodes.reshape(-1, 3), coarse.N).reshape(nodes.shape[:2])
        cg = coarse.gid[m][cpos]                                     # (F, nloc)
        phi = np.stack([fe.basis(deg, xi[f:f + 1])[0] for f in range(len(sel))])
        rows.append(np.repeat(sel, phi.shape[1]))
        cols.append(cg.reshape(-1))
        vals.append(phi.reshape(-1))
    rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    keep = np.abs(vals) > 1e-14
    M = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(fine.ndof, coarse.ndof)).tocsr()
    M.sum_duplicates()
    return M


def load_vector(space: Space, f, quad_degree: int = 5) -> np.ndarray:
    """b_i = integral of f phi_i (per element, quadrature of the given degree), boundary rows zero."""
    xi, w = quadrature.rule(quad_degree)
    J, adet, _ = fe.jacobians(space.elem_X)
    pts = fe.map_points(space.elem_X, J, xi)
    fq = f(pts.reshape(-1, 3)).reshape(len(space.elem_X), len(w))
    phi = fe.basis(space.degree, xi)                                 # (nq, nloc)
    be = np.einsum("e,q,eq,qi->ei", adet, w, fq, phi)
    b = np.zeros(space.ndof)
    np.add.at(b, space.elem_dofs, be)
    b[space.boundary] = 0.0
    return b


def l2_error(space: Space, uh: np.ndarray, u, quad_degree: int = 5) -> float:
    """|| u_h - u ||_L2 by element quadrature."""
    xi, w = quadrature.rule(quad_degree)
    J, adet, _ = fe.jacobians(space.elem_X)
    pts = fe.map_points(space.elem_X, J, xi)
    uq = u(pts.reshape(-1, 3)).reshape(len(space.elem_X), len(w))
    uhq = uh[space.elem_dofs] @ fe.basis(space.degree, xi).T
    return float(np.sqrt(np.einsum("e,q,eq->", adet, w, (uhq - uq) ** 2)))


def power_iteration(A, dinv: np.ndarray, v0: np.ndarray, iters: int) -> float:
    """Estimate of the largest eigenvalue of D^{-1} A: iters steps of v <- D^{-1}A v / ||.||."""
    v = v0 / np.linalg.norm(v0)
    lam = 0.0
    for _ in range(iters):
        w = dinv * (A @ v)
        lam = np.linalg.norm(w)
        v = w / lam
    return float(lam)


def chebyshev(A, dinv: np.ndarray, b: np.ndarray, x: np.ndarray, lam: float, order: int = 2,
              lo: float = 0.1, hi: float = 1.1) -> np.ndarray:
    """One Chebyshev smoothing step of the given order on D^{-1} A over [lo lam, hi lam].

    theta, delta: centre and half-width of the interval; the three-term
    recurrence of Chebyshev polynomials gives the update directions.
    """
    a, bb = lo * lam, hi * lam
    theta, delta = 0.5 * (bb + a), 0.5 * (bb - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = x.copy()
    r = dinv * (b - A @ x)
    d = r / theta
    for k in range(order):
        x = x + d
        if k == order - 1:
            break
        r = dinv * (b - A @ x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x


class Hierarchy:
    """Spaces, Dirichlet operators and transfers on levels 0..L (one FE degree)."""

    def __init__(self, mesh, L: int, degree: int, coeff=("const", 1.0), quad_degree: int = 4, cheb_order: int = 2,
                 power_iters: int = 15, seed: int = 0):
        self.L = L
        self.spaces = [Space(mesh, l, degree) for l in range(L + 1)]
        self.A = [diffusion_matrix(s, coeff, quad_degree, "dirichlet") for s in self.spaces]
        self.dinv = [1.0 / A.diagonal() for A in self.A]
        self.P = [None] + [prolongation(self.spaces[l - 1], self.spaces[l]) for l in range(1, L + 1)]
        self.order = cheb_order
        self.lam = []
        for l, s in enumerate(self.spaces):
            rng = np.random.default_rng(seed)
            v0 = rng.uniform(-1.0, 1.0, s.ndof)
            v0[s.boundary] = 0.0
            if s.interior.sum() == 0:
                self.lam.append(1.0)
            else:
                self.lam.append(power_iteration(self.A[l], self.dinv[l], v0, power_iters))
        A0 = self.A[0].toarray()
        self.coarse_cho = scipy.linalg.cho_factor(A0)

    def vcycle(self, l: int, b: np.ndarray, x: np.ndarray, nu1: int = 2, nu2: int = 2) -> np.ndarray:
        if l == 0:
            return scipy.linalg.cho_solve(self.coarse_cho, b)
        A, dinv, s = self.A[l], self.dinv[l], self.spaces[l]
        for _ in range(nu1):
            x = chebyshev(A, dinv, b, x, self.lam[l], self.order)
        r = b - A @ x
        r[s.boundary] = 0.0
        rc = self.P[l].T @ r
        rc[self.spaces[l - 1].boundary] = 0.0
        ec = self.vcycle(l - 1, rc, np.zeros_like(rc), nu1, nu2)
        ec[self.spaces[l - 1].boundary] = 0.0
        x = x + self.P[l] @ ec
        for _ in range(nu2):
            x = chebyshev(A, dinv, b, x, self.lam[l], self.order)
        return x

    def fmg(self, b, nu1: int = 2, nu2: int = 2, tol: float = 1e-10, max_cycles: int = 50):
        """FMG then V-cycles on the finest level for the fine right-hand side b.

        The right-hand sides of the coarser levels are restrictions of b: b_{l-1} = P_l^T b_l with
        the boundary rows zero (the same transfer the V-cycle applies to residuals).
        Returns (x, number of V-cycles on the finest level after FMG, history of relative residuals).
        """
        bs = [None] * (self.L + 1)
        bs[self.L] = np.asarray(b, dtype=np.float64).copy()
        bs[self.L][self.spaces[self.L].boundary] = 0.0
        for l in range(self.L, 0, -1):
            bs[l - 1] = self.P[l].T @ bs[l]
            bs[l - 1][self.spaces[l - 1].boundary] = 0.0
        x = scipy.linalg.cho_solve(self.coarse_cho, bs[0])
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
