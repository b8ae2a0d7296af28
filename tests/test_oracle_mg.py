"""Pins of the oracle's multigrid pieces (Section 8): transfers, Chebyshev, V-cycle, FMG."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import assemble as A, mesh as M, mg

RNG = np.random.default_rng(5)


def _mesh(name="cube6"):
    return M.MacroMesh(*getattr(W, name)())


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("name", ["cube6", "reference_tet"])
def test_prolongation_reproduces_polynomials(degree, name):
    mm = _mesh(name)
    Sc, Sf = A.Space(mm, 1, degree), A.Space(mm, 2, degree)
    P = mg.prolongation(Sc, Sf)
    # partition of unity, and exact reproduction of polynomials of the element degree
    assert np.allclose(P @ np.ones(Sc.ndof), 1.0, atol=1e-14)
    if degree == 1:
        f = lambda p: 0.3 + p[:, 0] - 2.0 * p[:, 1] + 0.5 * p[:, 2]
    else:
        f = lambda p: 0.3 + p[:, 0] * p[:, 1] - 2.0 * p[:, 1] ** 2 + 0.5 * p[:, 2] - p[:, 0] * p[:, 2]
    assert np.allclose(P @ Sc.interpolate(f), Sf.interpolate(f), atol=1e-13)
    # coarse nodes are fine nodes: those rows are unit rows
    Pd = P.toarray()
    assert np.isclose(Pd.max(), 1.0)
    if degree == 1:
        # P1: every fine node is a coarse node (weight 1) or a coarse edge midpoint (1/2, 1/2)
        for row in Pd:
            nz = np.sort(row[np.abs(row) > 1e-14])
            assert np.allclose(nz, [1.0]) or np.allclose(nz, [0.5, 0.5])


def test_chebyshev_order1_is_damped_jacobi_and_order2_polynomial():
    mm = _mesh("reference_tet")
    S = A.Space(mm, 2, 1)
    K = A.diffusion_matrix(S, ("const", 1.0), 2, "dirichlet")
    dinv = 1.0 / K.diagonal()
    b, x0 = RNG.standard_normal(S.ndof), RNG.standard_normal(S.ndof)
    lam = 1.9
    theta = 0.5 * (0.1 + 1.1) * lam
    x1 = mg.chebyshev(K, dinv, b, x0, lam, order=1)
    assert np.allclose(x1, x0 + dinv * (b - K @ x0) / theta, atol=1e-14)
    # order 2: error propagation e -> p(D^{-1}A) e with p(t) = T2((theta - t)/delta) / T2(theta/delta)
    Kd = K.toarray()
    xs = np.linalg.solve(Kd, b)
    x2 = mg.chebyshev(K, dinv, b, x0, lam, order=2)
    delta = 0.5 * (1.1 - 0.1) * lam
    T2 = lambda s: 2 * s * s - 1
    Dh = np.diag(np.sqrt(dinv))
    ev, V = np.linalg.eigh(Dh @ Kd @ Dh)
    pmat = Dh @ V @ np.diag(T2((theta - ev) / delta) / T2(theta / delta)) @ V.T @ np.linalg.inv(Dh)
    assert np.allclose(x2 - xs, pmat @ (x0 - xs), atol=1e-12)


def test_power_iteration_approaches_max_eigenvalue():
    mm = _mesh("cube6")
    S = A.Space(mm, 2, 1)
    K = A.diffusion_matrix(S, ("const", 1.0), 2, "dirichlet")
    dinv = 1.0 / K.diagonal()
    v0 = RNG.uniform(-1, 1, S.ndof)
    v0[S.boundary] = 0.0
    I = ~S.boundary
    Kd = K.toarray()[np.ix_(I, I)]
    lam_true = np.max(np.linalg.eigvals(np.diag(dinv[I]) @ Kd).real)
    lam = mg.power_iteration(K, dinv, v0, 400)
    assert abs(lam - lam_true) < 1e-3 * lam_true
    assert mg.power_iteration(K, dinv, v0, 15) <= lam_true * (1 + 1e-12)


@pytest.mark.parametrize("degree", [1, 2])
def test_vcycle_contraction_is_level_independent(degree):
    mm = _mesh("cube6")
    rates = []
    Lmax = 4 if degree == 1 else 3
    H = mg.Hierarchy(mm, Lmax, degree, quad_degree=2 if degree == 1 else 4)
    for l in range(2, Lmax + 1):
        S = H.spaces[l]
        b = np.zeros(S.ndof)
        x = RNG.uniform(-1, 1, S.ndof)
        x[S.boundary] = 0.0
        r0 = np.linalg.norm(H.A[l] @ x)
        for _ in range(3):
            x = H.vcycle(l, b, x)
        rates.append((np.linalg.norm(H.A[l] @ x) / r0) ** (1 / 3))
    assert max(rates) < 0.25, rates
    assert max(rates) - min(rates) < 0.1, rates


def test_fmg_converges_and_discretisation_order():
    mm = _mesh("cube6")
    errs = {}
    for degree, L in [(1, 4), (2, 3)]:
        H = mg.Hierarchy(mm, L, degree, quad_degree=2 if degree == 1 else 4)
        bs = [mg.load_vector(s, W.manufactured_f) for s in H.spaces]
        x, cycles, hist = H.fmg(bs[L], tol=1e-10)
        assert hist[-1] <= 1e-10 and cycles <= 15
        # error on each level of the hierarchy, solved directly
        e = []
        for l in range(1, L + 1):
            xl = sp.linalg.spsolve(H.A[l].tocsc(), bs[l])
            e.append(mg.l2_error(H.spaces[l], xl, W.manufactured_u))
        errs[degree] = e
        assert np.isclose(mg.l2_error(H.spaces[L], x, W.manufactured_u), e[-1], rtol=1e-6)
    r1 = errs[1][-1] / errs[1][-2]     # O(h^2): ratio near 1/4
    r2 = errs[2][-1] / errs[2][-2]     # O(h^3): ratio near 1/8
    assert 0.2 < r1 < 0.3, errs[1]
    assert 0.09 < r2 < 0.16, errs[2]
