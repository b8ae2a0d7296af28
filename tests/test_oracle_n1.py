"""Pins of the oracle's lowest-order Nedelec curl-curl + mass operator (Eq. N1, Section 7.3)."""
import numpy as np
import pytest

import workloads as W
from oracle import assemble as A, fe, mesh as M

RNG = np.random.default_rng(17)


def _space(name, level):
    return A.EdgeSpace(M.MacroMesh(*getattr(W, name)()), level)


def test_whitney_tangential_moments():
    """int over edge f of phi_e . t_f = delta_ef (t_f = X_b - X_a, local orientation a -> b)."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])[None] + 0.2 * RNG.standard_normal((3, 4, 3))
    edges = M.P2_EDGES
    for x in X:
        Jinv = np.linalg.inv((x[1:] - x[0]).T)
        G = (Jinv.T @ fe.GRAD_BARY.T).T                     # grad lambda_a, rows
        for e, (a, b) in enumerate(edges):
            for f, (c, d) in enumerate(edges):
                # lambda along edge f: linear from vertex c to d; integrate with Simpson (exact, degree 1)
                tot = 0.0
                for s, wgt in ((0.0, 1 / 6), (0.5, 4 / 6), (1.0, 1 / 6)):
                    lam = np.zeros(4)
                    lam[c], lam[d] = 1 - s, s
                    phi = lam[a] * G[b] - lam[b] * G[a]
                    tot += wgt * phi @ (x[d] - x[c])
                assert abs(tot - (1.0 if e == f else 0.0)) < 1e-12


@pytest.mark.parametrize("name,level", [("reference_tet", 2), ("cube6", 1), ("cube48", 0)])
def test_gradients_in_curl_kernel(name, level):
    S = _space(name, level)
    alpha = ("func", lambda p: 1.0 + p[:, 0] + 0.3 * p[:, 2])
    Ac = A.n1_matrix(S, alpha, ("const", 0.0), 4, "neumann")
    G = A.n1_gradient(S)
    p = RNG.standard_normal(S.V1.ndof)
    assert np.abs(Ac @ (G @ p)).max() < 1e-12 * abs(Ac).max() * np.abs(G @ p).max() * 10
    # and the full operator on gradients is the beta-mass part only
    beta = ("const", 2.5)
    Af = A.n1_matrix(S, alpha, beta, 4, "neumann")
    Am = A.n1_matrix(S, ("const", 0.0), beta, 4, "neumann")
    assert np.allclose(Af @ (G @ p), Am @ (G @ p), atol=1e-12)


def test_energy_of_constant_and_rotational_fields():
    S = _space("cube6", 2)
    u0 = np.array([0.3, -1.2, 0.7])
    c = S.interpolate_field(lambda x: np.broadcast_to(u0, x.shape))
    beta = ("func", lambda p: 1.0 + p[:, 0])
    Am = A.n1_matrix(S, ("const", 0.0), beta, 4, "neumann")
    assert np.isclose(c @ Am @ c, 1.5 * u0 @ u0, rtol=1e-12)          # int (1 + x) |u0|^2 over the unit cube
    w = np.array([0.4, 0.1, -0.8])
    r = S.interpolate_field(lambda x: np.cross(w[None, :], x))      # curl(w x x) = 2 w
    Ac = A.n1_matrix(S, ("const", 1.7), ("const", 0.0), 4, "neumann")
    assert np.isclose(r @ Ac @ r, 1.7 * 4 * w @ w, rtol=1e-12)


def test_symmetry_and_dirichlet_spd():
    S = _space("cube6", 1)
    K = A.n1_matrix(S, ("const", 1.0), ("const", 0.5), 4, "dirichlet").toarray()
    assert np.allclose(K, K.T, atol=1e-14)
    assert np.linalg.eigvalsh(K).min() > 0
    Kn = A.n1_matrix(S, ("const", 1.0), ("const", 0.0), 4, "neumann").toarray()
    # curl-curl alone is singular (gradients); its null space has the dimension of the gradients
    ev = np.linalg.eigvalsh(Kn)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == S.V1.ndof - 1


def _n1_field_at(space, u, xi):
    """E_h at the mapped reference points xi of every element: sum_e u_e s_e phi_e (Whitney)."""
    J, adet, Jinv = fe.jacobians(space.elem_X)
    G = np.einsum("eji,aj->eai", Jinv, fe.GRAD_BARY)                  # grad lambda_a, (E, 4, 3)
    lam = fe.bary(xi)                                                  # (nq, 4)
    ue = u[space.elem_dofs] * space.elem_sign                          # (E, 6)
    out = np.zeros((len(space.elem_X), len(xi), 3))
    for e, (a, b) in enumerate(M.P2_EDGES):
        phi = lam[None, :, a, None] * G[:, None, b, :] - lam[None, :, b, None] * G[:, None, a, :]
        out += ue[:, e, None, None] * phi
    return out, J, adet


def test_n1_solution_converges_first_order():
    """Section 7.3 checks that the Nedelec FMG solution converges as O(h) in L2.  Pinned here on the
    oracle with a manufactured field on the unit cube: E = (sin pi y sin pi z, sin pi x sin pi z,
    sin pi x sin pi y) has zero tangential trace on the boundary and div E = 0, so with
    alpha = beta = 1, curl curl E + E = (2 pi^2 + 1) E.  The Galerkin solution (Dirichlet
    tangential trace, exact sparse solve) must approach E with ratio about 1/2 per level."""
    import scipy.sparse.linalg as spla
    from oracle import quadrature

    def E(p):
        s = np.sin(np.pi * p)
        return np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], axis=1)

    mm = M.MacroMesh(*W.cube6())
    xi, w = quadrature.rule(5)
    errs = []
    for level in (1, 2, 3, 4):
        S = A.EdgeSpace(mm, level)
        K = A.n1_matrix(S, ("const", 1.0), ("const", 1.0), 4, "dirichlet")
        # load vector b_e = int f . phi_e, f = (2 pi^2 + 1) E, element by element
        unit = np.zeros(S.ndof)
        b = np.zeros(S.ndof)
        _, J, adet = _n1_field_at(S, unit, xi)
        pts = fe.map_points(S.elem_X, J, xi)
        fq = (2 * np.pi ** 2 + 1) * E(pts.reshape(-1, 3)).reshape(len(S.elem_X), len(w), 3)
        G = np.einsum("eji,aj->eai", fe.jacobians(S.elem_X)[2], fe.GRAD_BARY)
        lam = fe.bary(xi)
        for e, (a, c) in enumerate(M.P2_EDGES):
            phi = lam[None, :, a, None] * G[:, None, c, :] - lam[None, :, c, None] * G[:, None, a, :]
            be = np.einsum("k,q,kqd,kqd->k", adet, w, fq, phi) * S.elem_sign[:, e]
            np.add.at(b, S.elem_dofs[:, e], be)
        b[S.boundary] = 0.0
        u = spla.spsolve(K.tocsc(), b)
        Eh, _, _ = _n1_field_at(S, u, xi)
        err = Eh - E(pts.reshape(-1, 3)).reshape(Eh.shape)
        errs.append(np.sqrt(np.einsum("k,q,kqd->", adet, w, err ** 2)))
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.all(ratios < 0.62) and ratios[-1] > 0.4, (errs, ratios)
