"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each one."""
import numpy as np

import workloads as W
from oracle import assemble as A, fe, mesh as M


def _p1_closed_form_ok():
    rng = np.random.default_rng(1)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)[None] + 0.3 * rng.standard_normal((5, 4, 3))
    Aq = fe.diffusion_local(X, 1, 1)
    G = np.array([np.linalg.inv(np.hstack([np.ones((4, 1)), x]))[1:, :].T for x in X])
    vol = np.abs(np.linalg.det(np.transpose(X[:, 1:] - X[:, :1], (0, 2, 1)))) / 6
    return np.allclose(Aq, vol[:, None, None] * np.einsum("eia,eja->eij", G, G), rtol=1e-10)


def test_transposed_jacobian_is_caught(monkeypatch):
    assert _p1_closed_form_ok()
    monkeypatch.setattr(fe, "phys_grads", lambda Jinv, g: np.einsum("eij,qnj->eqni", Jinv, g))
    assert not _p1_closed_form_ok()


def test_dropped_epsilon_cross_term_is_caught(monkeypatch):
    S = A.Space(M.MacroMesh(*W.cube6()), 0, 2)
    K = A.epsilon_matrix(S, ("const", 1.0), 2, "neumann")
    r = np.cross(np.array([0, 0, 1.0])[None, :], S.coords).reshape(-1)
    assert np.abs(K @ r).max() < 1e-12

    def bad(X, qd, mu):
        # grad u : grad v in place of eps(u) : eps(v) -- the transpose part is lost
        lap = fe.diffusion_local(X, 2, qd, mu)
        return np.einsum("eab,cd->eacbd", lap, np.eye(3)).reshape(len(X), 30, 30)
    monkeypatch.setattr(fe, "epsilon_local", bad)
    K = A.epsilon_matrix(S, ("const", 1.0), 2, "neumann")
    assert np.abs(K @ r).max() > 1e-6


def test_wrong_octahedron_split_is_caught(monkeypatch):
    bad = M.CLASS_OFFSETS.copy()
    bad[1] = [[0, 1, 0], [1, 0, 1], [1, 0, 0], [0, 0, 1]]     # duplicates a tet of another class
    monkeypatch.setattr(M, "CLASS_OFFSETS", bad)
    n = 4
    cls, tv = M.micro_tets(n)
    faces = {}
    for t in tv:
        for a in range(4):
            f = tuple(sorted(tuple(p) for idx, p in enumerate(t) if idx != a))
            faces[f] = faces.get(f, 0) + 1
    assert max(faces.values()) > 2        # conformity pin fails


def test_dropped_p2_gradient_term_is_caught(monkeypatch):
    S = A.Space(M.MacroMesh(*W.cube6()), 1, 2)
    u = S.interpolate(lambda p: p[:, 0] * p[:, 1])       # grad = (y, x, 0): |grad|^2 integrates to 2/3
    K = A.diffusion_matrix(S, ("const", 1.0), 4, "neumann")
    assert np.isclose(u @ K @ u, 2.0 / 3.0, rtol=1e-12)
    orig = fe.basis_grad

    def bad(degree, xi):
        g = orig(degree, xi)
        if degree == 2:
            g[:, 4:, :] *= 0.5      # edge functions lose half of their gradient
        return g
    monkeypatch.setattr(fe, "basis_grad", bad)
    K = A.diffusion_matrix(S, ("const", 1.0), 4, "neumann")
    assert not np.isclose(u @ K @ u, 2.0 / 3.0, rtol=1e-6)
