"""Pins of the oracle's global operators (Eq. 4.1) and coefficient adjoint."""
import numpy as np
import pytest

import workloads as W
from oracle import assemble as A, mesh as M, layout as L

RNG = np.random.default_rng(11)


def _space(meshname, level, degree):
    v, t = getattr(W, meshname)()
    return A.Space(M.MacroMesh(v, t), level, degree)


COEFFS = [("const", 1.0), ("sin3",), ("func", lambda p: 1.0 + 0.5 * p[:, 0] - 0.25 * p[:, 1] * p[:, 2])]


@pytest.mark.parametrize("meshname,level", [("reference_tet", 2), ("cube6", 1), ("cube48", 0)])
@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("ci", range(3))
def test_symmetry_and_constants(meshname, level, degree, ci):
    S = _space(meshname, level, degree)
    qd = 2 if degree == 1 else 4
    An = A.diffusion_matrix(S, COEFFS[ci], qd, "neumann")
    Ad = A.diffusion_matrix(S, COEFFS[ci], qd, "dirichlet")
    x, y = RNG.standard_normal(S.ndof), RNG.standard_normal(S.ndof)
    for Mx in (An, Ad):
        assert abs(x @ (Mx @ y) - y @ (Mx @ x)) <= 1e-13 * np.abs(Mx).sum() * 10
    assert np.abs(An @ np.ones(S.ndof)).max() < 1e-13 * abs(An).max()
    # Dirichlet rows of boundary DoFs are identity; interior rows ignore boundary columns
    xb = np.where(S.boundary, x, 0.0)
    assert np.allclose((Ad @ xb)[S.boundary], x[S.boundary])
    assert np.abs((Ad @ xb)[~S.boundary]).max() < 1e-15


def test_config1_counts():
    S = _space("reference_tet", 4, 1)
    assert S.ndof == 969 and S.interior.sum() == 455


@pytest.mark.parametrize("degree", [1, 2])
def test_energy_identities(degree):
    """x^T A x = integral of k |grad u|^2 for u in the space (u linear for P1, quadratic for P2)."""
    sympy = pytest.importorskip("sympy")
    S = _space("cube6", 2, degree)
    xs, ys, zs = sympy.symbols("x y z")
    if degree == 1:
        u = 0.3 * xs - 1.1 * ys + 0.7 * zs + 0.2
    else:
        u = 0.3 * xs ** 2 - 1.1 * xs * ys + 0.7 * zs ** 2 + 0.4 * ys * zs - zs + 0.1
    for kexpr in (sympy.Integer(1), 1 + xs / 2 - ys / 4):
        integrand = kexpr * sum(sympy.diff(u, v) ** 2 for v in (xs, ys, zs))
        exact = float(sympy.integrate(integrand, (xs, 0, 1), (ys, 0, 1), (zs, 0, 1)))
        f = sympy.lambdify((xs, ys, zs), u, "numpy")
        kf = sympy.lambdify((xs, ys, zs), kexpr, "numpy")
        uh = S.interpolate(lambda p: f(p[:, 0], p[:, 1], p[:, 2]) + 0 * p[:, 0])
        coeff = ("func", lambda p: kf(p[:, 0], p[:, 1], p[:, 2]) + 0 * p[:, 0])
        K = A.diffusion_matrix(S, coeff, 2 if degree == 1 else 4, "neumann")
        assert abs(uh @ (K @ uh) - exact) < 1e-12 * max(1.0, abs(exact))


@pytest.mark.parametrize("degree", [1, 2])
def test_dirichlet_spd(degree):
    S = _space("cube6", 1, degree)
    Ad = A.diffusion_matrix(S, ("sin3",), 2 if degree == 1 else 4, "dirichlet").toarray()
    ev = np.linalg.eigvalsh(Ad)
    assert ev.min() > 0


def test_level1_single_macro_by_hand():
    """Reference macro at level 1 (8 micro-tets, 10 P1 DoFs): sum of cotangent-formula element matrices."""
    S = _space("reference_tet", 1, 1)
    K = A.diffusion_matrix(S, ("const", 1.0), 1, "neumann").toarray()
    ref = np.zeros((10, 10))
    for X, d in zip(S.elem_X, S.elem_dofs):
        vol = abs(np.linalg.det((X[1:] - X[0]).T)) / 6
        for i in range(4):
            for j in range(4):
                if i == j:
                    continue
                k, l = [v for v in range(4) if v not in (i, j)]
                e = X[l] - X[k]
                ni, nj = np.cross(e, X[i] - X[k]), np.cross(e, X[j] - X[k])
                cot = np.dot(ni, nj) / np.linalg.norm(np.cross(ni, nj))
                ref[d[i], d[j]] += -np.linalg.norm(e) * cot / 6
    ref[np.diag_indices(10)] = -ref.sum(axis=1)
    assert np.allclose(K, ref, atol=1e-14)


def test_epsilon_operator():
    S = _space("cube6", 1, 2)
    mu = ("func", W.viscosity_mu)
    K = A.epsilon_matrix(S, mu, 4, "neumann")
    # the six rigid-body modes are in the null space
    for r in [np.tile(np.eye(3)[c], S.ndof) for c in range(3)] + \
             [np.cross(w[None, :], S.coords).reshape(-1) for w in np.eye(3)]:
        assert np.abs(K @ r).max() < 1e-12 * abs(K).max()
    x, y = RNG.standard_normal(3 * S.ndof), RNG.standard_normal(3 * S.ndof)
    assert abs(x @ (K @ y) - y @ (K @ x)) < 1e-11
    Kd = A.epsilon_matrix(S, mu, 4, "dirichlet").toarray()
    assert np.linalg.eigvalsh(Kd).min() > 0


@pytest.mark.parametrize("degree,kdeg", [(1, 1), (2, 2)])
def test_coefficient_adjoint(degree, kdeg):
    S = _space("cube6", 1, degree)
    KS = S if kdeg == degree else _space("cube6", 1, kdeg)
    qd = 2 if degree == 1 else 4
    k = np.exp(W.fourier_field(KS.coords, seed=0))
    u, g = RNG.uniform(-1, 1, S.ndof), RNG.uniform(-1, 1, S.ndof)
    for bc in ("dirichlet", "neumann"):
        dk = A.diffusion_coeff_adjoint(S, KS, u, g, qd, bc)
        Ak = A.diffusion_matrix(S, ("field", KS, k), qd, bc)
        A0 = A.diffusion_matrix(S, ("field", KS, np.zeros(KS.ndof)), qd, bc)
        # linearity: sum_m k_m dk_m = g^T (A(k) - A(0)) u  (A(0) holds only the Dirichlet identity rows)
        assert np.isclose(k @ dk, g @ ((Ak - A0) @ u), rtol=1e-12)
        # central differences along random directions
        for _ in range(3):
            d = RNG.standard_normal(KS.ndof)
            h = 1e-6
            fp = g @ (A.diffusion_matrix(S, ("field", KS, k + h * d), qd, bc) @ u)
            fm = g @ (A.diffusion_matrix(S, ("field", KS, k - h * d), qd, bc) @ u)
            assert abs((fp - fm) / (2 * h) - d @ dk) < 1e-6 * max(1, abs(d @ dk))


def test_p1_field_adjoint_closed_form():
    """P1 operator with P1 field: dk_v = sum over T containing v of (1/4) g_T^T A0_T u_T."""
    S = _space("reference_tet", 2, 1)
    u, g = RNG.uniform(-1, 1, S.ndof), RNG.uniform(-1, 1, S.ndof)
    dk = A.diffusion_coeff_adjoint(S, S, u, g, 2, "neumann")
    from oracle import fe
    A0 = fe.diffusion_local(S.elem_X, 1, 1)
    ref = np.zeros(S.ndof)
    for e, d in enumerate(S.elem_dofs):
        ref[d] += 0.25 * (g[d] @ A0[e] @ u[d])
    assert np.allclose(dk, ref, atol=1e-14)


def test_epsilon_adjoint_linearity():
    S = _space("cube6", 0, 2)
    mu = W.viscosity_mu(S.coords)
    u, g = RNG.uniform(-1, 1, 3 * S.ndof), RNG.uniform(-1, 1, 3 * S.ndof)
    dmu = A.epsilon_coeff_adjoint(S, u, g, 4, "neumann")
    K = A.epsilon_matrix(S, ("field", S, mu), 4, "neumann")
    assert np.isclose(mu @ dmu, g @ (K @ u), rtol=1e-12)


@pytest.mark.parametrize("degree,coeff", [(1, ("const", 1.0)), (1, ("sin3",)), (2, ("sin3",)), (2, ("const", 2.0))])
def test_sampled_rows_match_assembled(degree, coeff):
    S = _space("reference_tet", 2, degree)
    qd = 2 if degree == 1 else 4
    K = A.diffusion_matrix(S, coeff, qd, "dirichlet")
    x = RNG.uniform(-1, 1, S.ndof)
    xp = L.to_packed(S, x)
    y = L.to_packed(S, K @ x)
    sample = np.arange(0, len(S.pts), 3)
    ys = A.sampled_diffusion_rows(S.mesh.vertices[S.mesh.tets[0]], 2, degree, coeff, qd, "dirichlet", xp, S.pts[sample])
    assert np.allclose(ys, y[sample], rtol=1e-13, atol=1e-14)


def test_layout_roundtrip():
    S = _space("cube6", 1, 2)
    x = RNG.standard_normal(S.ndof)
    xp = L.to_packed(S, x)
    assert len(xp) == 6 * M.lattice_size(4)
    assert L.copies_spread(S, xp) == 0.0
    assert np.array_equal(L.from_packed(S, xp), x)


def test_epsilon_solution_is_third_order():
    """The P2 vector epsilon operator (Section 7.4 names it) with a manufactured displacement on the
    unit cube: u = phi (1, 1, 1), phi = sin pi x sin pi y sin pi z (zero on the boundary),
    mu = 1 + x/2, f = -div(2 mu eps(u)) = -mu (Lap u + grad div u) - 2 eps(u) grad mu in closed
    form.  The Galerkin solution (exact sparse solve) must approach u as O(h^3) in L2."""
    import scipy.sparse.linalg as spla
    from oracle import mg

    p = np.pi

    def parts(x):
        s, c = np.sin(p * x), np.cos(p * x)
        phi = s[:, 0] * s[:, 1] * s[:, 2]
        d1 = p * np.stack([c[:, 0] * s[:, 1] * s[:, 2], s[:, 0] * c[:, 1] * s[:, 2], s[:, 0] * s[:, 1] * c[:, 2]], 1)
        d2 = np.empty((len(x), 3, 3))                                 # second derivatives of phi
        for i in range(3):
            for j in range(3):
                if i == j:
                    d2[:, i, j] = -p * p * phi
                else:
                    k = 3 - i - j
                    d2[:, i, j] = p * p * c[:, i] * c[:, j] * s[:, k]
        return phi, d1, d2

    def f_comp(comp):
        def f(x):
            phi, d1, d2 = parts(x)
            mu = 1.0 + 0.5 * x[:, 0]
            lap = -3.0 * p * p * phi                                    # Lap u_c, every component
            graddiv = d2[:, comp, :].sum(axis=1)                        # d_c (phi_x + phi_y + phi_z)
            eps_c0 = 0.5 * (d1[:, comp] + d1[:, 0])                     # eps(u)_{c,x}
            return -mu * (lap + graddiv) - 2.0 * eps_c0 * 0.5           # grad mu = (1/2, 0, 0)
        return f

    mm = M.MacroMesh(*W.cube6())
    errs = []
    for level in (1, 2, 3):
        S = A.Space(mm, level, 2)
        K = A.epsilon_matrix(S, ("func", lambda x: 1.0 + 0.5 * x[:, 0]), 4, "dirichlet")
        b = np.zeros(3 * S.ndof)
        for comp in range(3):
            b[comp::3] = mg.load_vector(S, f_comp(comp))
        u = spla.spsolve(K.tocsc(), b)
        e2 = sum(mg.l2_error(S, u[comp::3], lambda x: parts(x)[0]) ** 2 for comp in range(3))
        errs.append(np.sqrt(e2))
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert 0.09 < ratios[-1] < 0.16 and ratios[0] < 0.2, (errs, ratios)


def _keyed(mesh, N, nrhs, seed):
    """x_at(m, pts) from the counter-based keyed generator: equal values at every copy of a point."""
    def at(m, pts):
        keys = M.point_keys(mesh.tets[m], np.asarray(pts), N)
        return W.uniform_keyed(keys, 3 * nrhs, seed).reshape(-1, 3, nrhs)
    return at


def _interface_samples(S, rng, count):
    """Lattice points of every kind: inside a macro, on shared and boundary faces, edges, vertices."""
    N = S.N
    w = np.stack([N - S.pts.sum(axis=1), S.pts[:, 0], S.pts[:, 1], S.pts[:, 2]], axis=1)
    zeros = (w == 0).sum(axis=1)
    out = []
    for m in rng.choice(S.mesh.nmacro, size=count):
        for z in (0, 1, 2, 3):
            cand = np.nonzero(zeros == z)[0]
            if len(cand):
                out.append((int(m), S.pts[rng.choice(cand)]))
    return out


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("meshname,level", [("cube48", 1), ("cube6", 2)])
def test_sampled_epsilon_rows_match_assembled(meshname, level, bc):
    """The sampled epsilon rows and mu-adjoint (every macro that stores a point, every micro-tet
    around it) against the assembled operator and adjoint, on points of every kind."""
    S = _space(meshname, level, 2)
    nrhs = 3
    mu = W.viscosity_mu(S.coords)
    mu_p = L.to_packed(S, mu)
    K = A.epsilon_matrix(S, ("field", S, mu), 4, bc)
    xat, gat = _keyed(S.mesh, S.N, nrhs, 7), _keyed(S.mesh, S.N, nrhs, 8)
    P = M.lattice_size(S.N)
    xp = np.concatenate([xat(m, S.pts) for m in range(S.mesh.nmacro)])       # packed, consistent copies
    gp = np.concatenate([gat(m, S.pts) for m in range(S.mesh.nmacro)])
    assert L.copies_spread(S, xp.reshape(-1), 3, nrhs) == 0.0
    X = L.from_packed(S, xp.reshape(-1), 3, nrhs).reshape(S.ndof * 3, nrhs)
    G = L.from_packed(S, gp.reshape(-1), 3, nrhs).reshape(S.ndof * 3, nrhs)
    Y = (K @ X).reshape(S.ndof, 3, nrhs)
    dmu = sum(A.epsilon_coeff_adjoint(S, X[:, r], G[:, r], 4, bc) for r in range(nrhs))
    samples = _interface_samples(S, np.random.default_rng(3), 6)
    ys = A.sampled_epsilon_rows(S.mesh, level, mu_p, xat, samples, 4, bc)
    ds = A.sampled_epsilon_adjoint(S.mesh, level, xat, gat, samples, 4, bc)
    gids = [S.gid[m, M.packed_position(p[None], S.N)[0]] for m, p in samples]
    assert np.allclose(ys, Y[gids], rtol=1e-13, atol=1e-13 * np.abs(Y).max())
    assert np.allclose(ds, dmu[gids], rtol=1e-13, atol=1e-13 * np.abs(dmu).max())
    assert P * S.mesh.nmacro == len(xp)
