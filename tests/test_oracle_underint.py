"""Under-integration of the P2 variable-coefficient operator keeps the L2 order (Section 7.1).

The kernels offer the P2 diffusion operator with k(x) evaluated by the
degree-2 (4-point) rule instead of the degree-4 (14-point) rule.  For that to
be a valid cheaper variant the discretisation error must still fall as h^3 in
L2.  Pinned here on the oracle with a manufactured solution on the unit cube:
u = sin(pi x) sin(pi y) sin(pi z), k = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z),
f = -div(k grad u) = 3 pi^2 k u - grad k . grad u, solved exactly (sparse LU)
on three levels with both rules.
"""
import numpy as np
import scipy.sparse.linalg as spla

import workloads as W
from oracle import assemble as A, mesh as M, mg


def _f(points):
    """-div(k grad u) for the u and k above, in closed form."""
    p = np.pi
    s1 = np.sin(p * points)
    c1 = np.cos(p * points)
    s2 = np.sin(2 * p * points)
    c2 = np.cos(2 * p * points)
    u = s1[:, 0] * s1[:, 1] * s1[:, 2]
    k = W.sin3_coeff(points)
    grad_u = p * np.stack([c1[:, 0] * s1[:, 1] * s1[:, 2],
                           s1[:, 0] * c1[:, 1] * s1[:, 2],
                           s1[:, 0] * s1[:, 1] * c1[:, 2]], axis=1)
    grad_k = p * np.stack([c2[:, 0] * s2[:, 1] * s2[:, 2],
                           s2[:, 0] * c2[:, 1] * s2[:, 2],
                           s2[:, 0] * s2[:, 1] * c2[:, 2]], axis=1)
    return 3.0 * p * p * k * u - (grad_k * grad_u).sum(axis=1)


def _errors(quad_degree, levels):
    mm = M.MacroMesh(*W.cube6())
    out = []
    for level in levels:
        S = A.Space(mm, level, 2)
        K = A.diffusion_matrix(S, ("sin3",), quad_degree=quad_degree)
        b = mg.load_vector(S, _f)
        uh = spla.spsolve(K.tocsc(), b)
        out.append(mg.l2_error(S, uh, W.manufactured_u))
    return np.array(out)


def test_closed_form_rhs_matches_finite_differences():
    # the closed-form f against a central-difference -div(k grad u) at random interior points
    rng = np.random.default_rng(3)
    pts = 0.1 + 0.8 * rng.random((20, 3))
    h = 1e-4

    def flux(p, d):
        e = np.zeros(3)
        e[d] = h / 2
        du = (W.manufactured_u(p + e) - W.manufactured_u(p - e)) / h
        return W.sin3_coeff(p) * du

    fd = np.zeros(len(pts))
    for d in range(3):
        e = np.zeros(3)
        e[d] = h / 2
        fd -= (flux(pts + e, d) - flux(pts - e, d)) / h
    assert np.allclose(_f(pts), fd, rtol=1e-5, atol=1e-5)


def test_p2_under_integrated_variable_coefficient_is_third_order():
    levels = [1, 2, 3]
    e4 = _errors(2, levels)      # 4-point rule (under-integrated)
    e14 = _errors(4, levels)     # 14-point rule
    r4 = e4[1:] / e4[:-1]
    r14 = e14[1:] / e14[:-1]
    # O(h^3): the error falls by about 8 per refinement with either rule
    assert 0.09 < r4[-1] < 0.16, e4
    assert 0.09 < r14[-1] < 0.16, e14
    # and the cheaper rule costs little accuracy on the finest level
    assert abs(e4[-1] - e14[-1]) < 0.25 * e14[-1], (e4, e14)
