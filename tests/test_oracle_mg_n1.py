"""Pins of the oracle's Nedelec multigrid (Section 8 with Hiptmair's hybrid smoother, Eq. N1)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import assemble as A, mesh as M, mg, mg_n1


def _mesh(name="cube6"):
    return M.MacroMesh(*getattr(W, name)())


@pytest.mark.parametrize("name,level_c", [("cube6", 0), ("cube6", 1), ("cube6", 2), ("reference_tet", 1)])
def test_edge_prolongation_reproduces_coarse_fields(name, level_c):
    """The lowest-order Nedelec space holds the fields a + b x x exactly, on every level: the
    prolonged coarse interpolant is the fine interpolant."""
    mm = _mesh(name)
    Sc, Sf = A.EdgeSpace(mm, level_c), A.EdgeSpace(mm, level_c + 1)
    P = mg_n1.edge_prolongation(Sc, Sf)
    for E in (lambda x: np.tile([0.3, -1.2, 0.7], (len(x), 1)),
              lambda x: np.cross(np.array([0.5, -0.2, 1.1])[None, :], x),
              lambda x: np.array([1.0, 2.0, -0.5])[None, :] + np.cross(np.array([-0.7, 0.4, 0.9])[None, :], x)):
        assert np.abs(P @ Sc.interpolate_field(E) - Sf.interpolate_field(E)).max() < 1e-13


@pytest.mark.parametrize("name,level_c", [("cube6", 1), ("reference_tet", 2)])
def test_edge_prolongation_commutes_with_gradient(name, level_c):
    """A coarse gradient prolongs to the gradient of the prolonged P1 function: P_E G_c = G_f P_1."""
    mm = _mesh(name)
    Sc, Sf = A.EdgeSpace(mm, level_c), A.EdgeSpace(mm, level_c + 1)
    P = mg_n1.edge_prolongation(Sc, Sf)
    Pv = mg.prolongation(Sc.V1, Sf.V1)
    D = P @ A.n1_gradient(Sc) - A.n1_gradient(Sf) @ Pv
    assert abs(D).max() < 1e-13


def _asymptotic_rate(H, L, cycles=10):
    S = H.spaces[L]
    x = np.random.default_rng(0).uniform(-1.0, 1.0, S.ndof)
    x[S.boundary] = 0.0
    b = np.zeros(S.ndof)
    r0 = np.linalg.norm(H.A[L] @ x)
    rate = 0.0
    for _ in range(cycles):
        x = H.vcycle(L, b, x)
        r = np.linalg.norm(H.A[L] @ x)
        rate, r0 = r / r0, r
    return rate


def test_hybrid_vcycle_contraction_is_level_independent():
    """With the gradient-space correction the V(2,2) contraction stays below a fixed bound as the
    level grows; with the edge smoother alone the gradient components are not reduced and the
    cycle stalls (the reason for the hybrid smoother)."""
    mm = _mesh("cube6")
    rates, stalled = [], []
    for L in (2, 3, 4):
        H = mg_n1.N1Hierarchy(mm, L)
        rates.append(_asymptotic_rate(H, L))
        for l in range(L + 1):
            H.Ap[l] = H.Ap[l][:0, :0]                  # drop the nodal part of the smoother
        stalled.append(_asymptotic_rate(H, L))
    assert max(rates) < 0.4 and rates[-1] - rates[-2] < 0.03, rates
    assert min(stalled) > 0.9, stalled


def test_n1_fmg_reaches_the_discretisation_error():
    """FMG + V(2,2) cycles with the hybrid smoother solve the manufactured curl-curl + mass problem
    (E = (sin pi y sin pi z, sin pi x sin pi z, sin pi x sin pi y), alpha = beta = 1) to a relative
    residual of 1e-10 and give the direct solver's L2 error."""
    def E(p):
        s = np.sin(np.pi * p)
        return np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], axis=1)

    mm = _mesh("cube6")
    L = 3
    H = mg_n1.N1Hierarchy(mm, L)

    def load(S):
        return mg_n1.load_vector(S, lambda p: (2 * np.pi ** 2 + 1) * E(p))

    bs = [load(S) for S in H.spaces]
    x, cycles, hist = H.fmg(bs[L], tol=1e-10)
    assert hist[-1] <= 1e-10 and cycles <= 30, (cycles, hist[-1])
    xd = spla.spsolve(H.A[L].tocsc(), bs[L])
    assert np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max()


def test_gradient_space_operator_is_p1_diffusion_with_beta():
    """G^T A G over the vertices is the P1 diffusion operator with coefficient beta: curl grad = 0
    leaves the beta-mass of the Whitney gradients, which are the gradients of the P1 hat functions.
    (So the nodal part of the hybrid smoother is a P1 variable-coefficient apply.)"""
    mm = _mesh("cube6")
    S = A.EdgeSpace(mm, 2)
    a = 1.0 + 0.5 * np.sin(3.0 * S.V1.coords[:, 0])
    b = np.exp(W.fourier_field(S.V1.coords, seed=3))
    K = A.n1_matrix(S, ("field", S.V1, a), ("field", S.V1, b), 4, "neumann")
    G = A.n1_gradient(S)
    D = A.diffusion_matrix(S.V1, ("field", S.V1, b), 2, "neumann")
    assert abs(G.T @ K @ G - D).max() <= 1e-13 * abs(D).max()
