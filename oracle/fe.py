"""P1 / P2 Lagrange bases and local element matrices by quadrature.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 1 and Eq. 4.1: the local matrix of a micro-tet T is
    A_T[j, i] = sum_q |det J| w_q  G(x_q, phi_i, phi_j)
with x_q = X0 + J xi_q the mapped quadrature points and J the Jacobian of the
affine map from the reference tetrahedron (columns X1-X0, X2-X0, X3-X0).
Integrands (Section 7):
  diffusion   G = k(x) grad phi_i . grad phi_j                (Eq. P1, Eq. P2V)
  epsilon     G = 2 mu(x) eps(phi_i e_c) : eps(phi_j e_d),  eps(u) = (grad u + grad u^T)/2
Everything here is vectorised over a batch of elements only; the arithmetic
of each element is exactly the formula above.
Pinned by: P1 closed form |T| G G^T, symmetry, zero row sums, the P2
reference-element matrix from exact symbolic integration, rigid-body null
space of the epsilon matrix (tests/test_oracle_fe.py).
"""
from __future__ import annotations

import numpy as np

from .mesh import P2_EDGES
from . import quadrature


def bary(xi: np.ndarray) -> np.ndarray:
    """Barycentric coordinates (lambda0..lambda3) of reference points xi (...,3)."""
    xi = np.asarray(xi, dtype=np.float64)
    return np.concatenate([1.0 - xi.sum(axis=-1, keepdims=True), xi], axis=-1)


GRAD_BARY = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def basis(degree: int, xi: np.ndarray) -> np.ndarray:
    """Reference basis values (nq, nloc)."""
    lam = bary(xi)
    if degree == 1:
        return lam
    vals = [lam[:, a] * (2.0 * lam[:, a] - 1.0) for a in range(4)]
    vals += [4.0 * lam[:, a] * lam[:, b] for a, b in P2_EDGES]
    return np.stack(vals, axis=1)


def basis_grad(degree: int, xi: np.ndarray) -> np.ndarray:
    """Reference basis gradients (nq, nloc, 3)."""
    lam = bary(np.atleast_2d(xi))
    nq = lam.shape[0]
    if degree == 1:
        return np.broadcast_to(GRAD_BARY[None], (nq, 4, 3)).copy()
    g = np.empty((nq, 10, 3))
    for a in range(4):
        g[:, a, :] = (4.0 * lam[:, a])[:, None] * GRAD_BARY[a][None, :] - GRAD_BARY[a][None, :]
    for e, (a, b) in enumerate(P2_EDGES):
        g[:, 4 + e, :] = 4.0 * (lam[:, a][:, None] * GRAD_BARY[b][None, :] + lam[:, b][:, None] * GRAD_BARY[a][None, :])
    return g


def jacobians(X: np.ndarray):
    """J (E,3,3) with columns X1-X0, X2-X0, X3-X0, |det J| (E,), J^{-1} (E,3,3)."""
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    det = np.linalg.det(J)
    return J, np.abs(det), np.linalg.inv(J)


def map_points(X: np.ndarray, J: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Physical quadrature points x_q = X0 + J xi_q, shape (E, nq, 3)."""
    return X[:, None, 0, :] + np.einsum("eij,qj->eqi", J, xi)


def phys_grads(Jinv: np.ndarray, ref_grad: np.ndarray) -> np.ndarray:
    """grad phi = J^{-T} grad_ref phi; ref_grad (nq, nloc, 3) -> (E, nq, nloc, 3)."""
    return np.einsum("eji,qnj->eqni", Jinv, ref_grad)


def diffusion_local(X: np.ndarray, degree: int, quad_degree: int, kq=None) -> np.ndarray:
    """Local diffusion matrices (E, nloc, nloc).

    kq: None for k = 1, else an array (E, nq) of k at the mapped points, or a
    callable k(points (E*nq, 3)) -> (E*nq,).
    """
    xi, w = quadrature.rule(quad_degree)
    J, adet, Jinv = jacobians(X)
    G = phys_grads(Jinv, basis_grad(degree, xi))                  # (E, nq, n, 3)
    if kq is None:
        kv = np.ones((len(X), len(w)))
    elif callable(kq):
        pts = map_points(X, J, xi)
        kv = kq(pts.reshape(-1, 3)).reshape(len(X), len(w))
    else:
        kv = np.asarray(kq, dtype=np.float64)
    scale = adet[:, None] * w[None, :] * kv                       # (E, nq)
    return np.einsum("eq,eqia,eqja->eij", scale, G, G)


def field_at_points(degree_k: int, xi: np.ndarray, kloc: np.ndarray) -> np.ndarray:
    """Value of a P1/P2 coefficient field at reference points: kloc (E, nloc_k) -> (E, nq)."""
    return kloc @ basis(degree_k, xi).T


def diffusion_coeff_derivative(X: np.ndarray, degree: int, degree_k: int, quad_degree: int) -> np.ndarray:
    """d A_T / d k_m for a P1/P2 coefficient field k = sum_m k_m psi_m.

    K[e, m, i, j] = sum_q |det J| w_q psi_m(x_q) grad phi_i . grad phi_j.
    """
    xi, w = quadrature.rule(quad_degree)
    J, adet, Jinv = jacobians(X)
    G = phys_grads(Jinv, basis_grad(degree, xi))
    psi = basis(degree_k, xi)                                      # (nq, nk)
    scale = adet[:, None] * w[None, :]                             # (E, nq)
    return np.einsum("eq,qm,eqia,eqja->emij", scale, psi, G, G)


def epsilon_local(X: np.ndarray, quad_degree: int, muq) -> np.ndarray:
    """Local P2-vector epsilon matrices (E, 30, 30), local index 3*node + component.

    A[(a,c),(b,d)] = sum_q |det J| w_q 2 mu(x_q) eps(phi_a e_c) : eps(phi_b e_d), and
    eps(phi_a e_c) : eps(phi_b e_d) = (delta_cd grad phi_a . grad phi_b + d_d phi_a d_c phi_b) / 2.
    muq: (E, nq) values at the mapped points or a callable of points.
    """
    xi, w = quadrature.rule(quad_degree)
    J, adet, Jinv = jacobians(X)
    G = phys_grads(Jinv, basis_grad(2, xi))                        # (E, nq, 10, 3)
    if callable(muq):
        pts = map_points(X, J, xi)
        mv = muq(pts.reshape(-1, 3)).reshape(len(X), len(w))
    else:
        mv = np.asarray(muq, dtype=np.float64)
    scale = adet[:, None] * w[None, :] * mv                        # (E, nq)
    gg = np.einsum("eq,eqad,eqbd->eab", scale, G, G)               # sum_q s grad phi_a . grad phi_b
    cross = np.einsum("eq,eqad,eqbc->eabdc", scale, G, G)          # [e,a,b,d,c] = sum_q s d_d phi_a d_c phi_b
    E = len(X)
    A = np.zeros((E, 10, 3, 10, 3))
    eye = np.eye(3)
    # 2 mu * (1/2) (delta_cd gg + cross) = mu (delta_cd gg + cross)
    A += gg[:, :, None, :, None] * eye[None, None, :, None, :]
    A += np.transpose(cross, (0, 1, 4, 2, 3))                      # -> [e, a, c, b, d]
    return A.reshape(E, 30, 30)


def epsilon_coeff_derivative(X: np.ndarray, quad_degree: int) -> np.ndarray:
    """d A_T / d mu_m for a P2 viscosity field mu = sum_m mu_m psi_m: (E, 10, 30, 30)."""
    xi, w = quadrature.rule(quad_degree)
    psi = basis(2, xi)
    out = np.empty((len(X), 10, 30, 30))
    for m in range(10):
        out[:, m] = epsilon_local(X, quad_degree, np.broadcast_to(psi[None, :, m], (len(X), len(w))))
    return out


# ---------------------------------------------------------------------------
# Lowest-order Nedelec (first kind) edge elements, Eq. N1 (Section 7.3)
# ---------------------------------------------------------------------------

def n1_local(X: np.ndarray, quad_degree: int, alpha_q, beta_q) -> np.ndarray:
    """Local curl-curl + mass matrices (E, 6, 6) on the local edges (a, b) of P2_EDGES, oriented a -> b.

    Basis (Whitney): phi_e = lambda_a grad lambda_b - lambda_b grad lambda_a, curl phi_e =
    2 grad lambda_a x grad lambda_b;  A[e, f] = sum_q |det J| w_q (alpha(x_q) curl phi_e . curl phi_f
    + beta(x_q) phi_e . phi_f).  alpha_q / beta_q: (E, nq) values or callables of points.
    """
    xi, w = quadrature.rule(quad_degree)
    J, adet, Jinv = jacobians(X)
    G = np.einsum("eji,aj->eai", Jinv, GRAD_BARY)                  # grad lambda_a, (E, 4, 3)

    def values(c):
        if callable(c):
            return c(map_points(X, J, xi).reshape(-1, 3)).reshape(len(X), len(w))
        return np.asarray(c, dtype=np.float64)
    av, bv = values(alpha_q), values(beta_q)
    lam = bary(xi)                                                 # (nq, 4)
    curl = np.stack([2.0 * np.cross(G[:, a], G[:, b]) for a, b in P2_EDGES], axis=1)   # (E, 6, 3)
    phi = np.stack([lam[None, :, a, None] * G[:, None, b, :] - lam[None, :, b, None] * G[:, None, a, :]
                    for a, b in P2_EDGES], axis=2)                 # (E, nq, 6, 3)
    sa = adet[:, None] * w[None, :] * av
    sb = adet[:, None] * w[None, :] * bv
    A = np.einsum("eq,eia,eja->eij", sa, curl, curl)
    A += np.einsum("eq,eqia,eqja->eij", sb, phi, phi)
    return A
