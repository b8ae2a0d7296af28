"""Pins of the oracle's local element matrices (Algorithm 1, Eq. P1, Eq. P2V, epsilon form)."""
import itertools

import numpy as np
import pytest

from oracle import fe

RNG = np.random.default_rng(7)
REF = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)


def _random_tets(E):
    return REF[None] + 0.25 * RNG.standard_normal((E, 4, 3))


def _bary_grads(X):
    """grad lambda_i from inverting [[1, x_a]] (independent of the Jacobian route)."""
    out = []
    for x in X:
        M = np.hstack([np.ones((4, 1)), x])
        out.append(np.linalg.inv(M)[1:, :].T)   # row i: grad of lambda_i
    return np.array(out)


def test_p1_closed_form():
    X = _random_tets(20)
    A = fe.diffusion_local(X, 1, 2)
    G = _bary_grads(X)
    vol = np.abs(np.linalg.det(np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1)))) / 6
    assert np.allclose(A, vol[:, None, None] * np.einsum("eia,eja->eij", G, G), rtol=1e-12, atol=1e-14)


def test_p1_cotangent_formula():
    """Off-diagonal P1 stiffness = -(1/6) |e_kl| cot(theta_kl), e_kl the edge opposite to edge ij."""
    X = _random_tets(10)
    A = fe.diffusion_local(X, 1, 1)
    for e, x in enumerate(X):
        for i, j in itertools.combinations(range(4), 2):
            k, l = [v for v in range(4) if v not in (i, j)]
            # dihedral angle at edge kl between faces (k,l,i) and (k,l,j)
            ekl = x[l] - x[k]
            ni = np.cross(ekl, x[i] - x[k])
            nj = np.cross(ekl, x[j] - x[k])
            cos = np.dot(ni, nj) / (np.linalg.norm(ni) * np.linalg.norm(nj))
            sin = np.linalg.norm(np.cross(ni, nj)) / (np.linalg.norm(ni) * np.linalg.norm(nj))
            expect = -np.linalg.norm(ekl) * (cos / sin) / 6.0
            assert abs(A[e, i, j] - expect) < 1e-12 * max(1, abs(expect))


@pytest.mark.parametrize("degree,qd", [(1, 2), (2, 2), (2, 4)])
def test_symmetry_and_row_sums(degree, qd):
    X = _random_tets(15)
    kq = lambda p: 1.0 + 0.5 * np.sin(p[:, 0]) * np.cos(p[:, 1]) + p[:, 2] ** 2
    A = fe.diffusion_local(X, degree, qd, kq)
    assert np.allclose(A, np.transpose(A, (0, 2, 1)), atol=1e-14)
    assert np.abs(A.sum(axis=2)).max() < 1e-13


def test_p2_reference_matrix_exact():
    """P2 stiffness on the reference and on an affine tet from exact symbolic integration."""
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    lam = [1 - x - y - z, x, y, z]
    phis = [lam[a] * (2 * lam[a] - 1) for a in range(4)] + [4 * lam[a] * lam[b] for a, b in
                                                           [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]]
    grads = [[sympy.diff(p, v) for v in (x, y, z)] for p in phis]
    Xt = np.array([REF, _random_tets(1)[0]])
    A = fe.diffusion_local(Xt, 2, 2)     # degree-2 rule is exact for the degree-2 integrand
    for t, X in enumerate(Xt):
        J = (X[1:] - X[0]).T
        Jinv = np.linalg.inv(J)
        det = abs(np.linalg.det(J))
        K = np.zeros((10, 10))
        for i in range(10):
            for j in range(i, 10):
                gi = np.array(grads[i], dtype=object)
                gj = np.array(grads[j], dtype=object)
                # physical gradient = J^{-T} grad_ref
                pi = [sum(Jinv[b, a] * gi[b] for b in range(3)) for a in range(3)]
                pj = [sum(Jinv[b, a] * gj[b] for b in range(3)) for a in range(3)]
                integrand = sympy.expand(sum(pi[a] * pj[a] for a in range(3)))
                val = sympy.integrate(integrand, (z, 0, 1 - x - y), (y, 0, 1 - x), (x, 0, 1))
                K[i, j] = K[j, i] = float(val) * det
        assert np.allclose(A[t], K, atol=1e-13, rtol=1e-12)
        if t == 0:
            # textbook entry on the reference tet: the diagonal of the vertex-0 function is 3/10
            assert np.isclose(K[0, 0], 0.3)


def test_variable_coefficient_against_closed_form():
    """k linear: integral of k grad phi_i . grad phi_j = (G_i.G_j) |T| k(centroid) for P1."""
    X = _random_tets(8)
    c = np.array([0.3, -0.2, 0.5])
    kq = lambda p: 2.0 + p @ c
    A = fe.diffusion_local(X, 1, 2, kq)
    G = _bary_grads(X)
    vol = np.abs(np.linalg.det(np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1)))) / 6
    kc = 2.0 + X.mean(axis=1) @ c
    assert np.allclose(A, (vol * kc)[:, None, None] * np.einsum("eia,eja->eij", G, G), rtol=1e-12, atol=1e-14)


def test_field_coefficient_derivative_is_linear_part():
    X = _random_tets(6)
    for degree, dk, qd in [(1, 1, 2), (2, 2, 4), (2, 1, 4)]:
        K = fe.diffusion_coeff_derivative(X, degree, dk, qd)
        kl = RNG.uniform(0.5, 2.0, (len(X), 4 if dk == 1 else 10))
        xi, _ = __import__("oracle.quadrature", fromlist=["rule"]).rule(qd)
        A = fe.diffusion_local(X, degree, qd, fe.field_at_points(dk, xi, kl))
        assert np.allclose(np.einsum("em,emij->eij", kl, K), A, rtol=1e-12, atol=1e-14)


def test_epsilon_rigid_modes_and_energy():
    X = _random_tets(6)
    mu = lambda p: 1.0 + p[:, 0] ** 2
    A = fe.epsilon_local(X, 4, mu)
    assert np.allclose(A, np.transpose(A, (0, 2, 1)), atol=1e-13)
    xi, _ = __import__("oracle.quadrature", fromlist=["rule"]).rule(4)
    for e, x in enumerate(X):
        # nodal positions of the P2 element
        nodes = np.vstack([x, [(x[a] + x[b]) / 2 for a, b in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]]])
        modes = []
        for c in range(3):
            t = np.zeros((10, 3)); t[:, c] = 1.0
            modes.append(t.reshape(-1))
        for w in np.eye(3):
            modes.append(np.cross(w[None, :], nodes).reshape(-1))
        for r in modes:
            assert np.abs(A[e] @ r).max() < 1e-12 * np.abs(A[e]).max()
    # constant mu, linear u = B x: u^T A u = 2 mu |sym B|^2 |T|
    Ac = fe.epsilon_local(X, 2, lambda p: np.full(len(p), 1.7))
    B = RNG.standard_normal((3, 3))
    for e, x in enumerate(X):
        nodes = np.vstack([x, [(x[a] + x[b]) / 2 for a, b in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]]])
        u = (nodes @ B.T).reshape(-1)
        vol = abs(np.linalg.det((x[1:] - x[0]).T)) / 6
        S = 0.5 * (B + B.T)
        assert np.isclose(u @ Ac[e] @ u, 2 * 1.7 * np.sum(S * S) * vol, rtol=1e-12)
