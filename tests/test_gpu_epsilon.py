"""P2 vector epsilon operator 2 div(mu eps(u)) through the C-ABI against the oracle, batched over
right-hand sides, and its adjoint in a P2 viscosity field mu = 10^(3(z - 0.5))."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import assemble as OA, layout as OL

pytestmark = pytest.mark.gpu


def _case(meshname, level):
    from gpu_helpers import Case
    c = Case(meshname, level, 2)
    mu = c.S.interpolate(W.viscosity_mu)
    return c, mu


@pytest.mark.parametrize("meshname,level", [("reference_tet", 1), ("reference_tet", 2), ("cube6", 1), ("cube48", 0),
                                            ("cube48", 1)])
@pytest.mark.parametrize("nrhs", [1, 3, 16])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_epsilon_apply_parity(meshname, level, nrhs, bc, dtype):
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    c, mu = _case(meshname, level)
    if dtype == torch.float32:
        mu = mu.astype(np.float32).astype(np.float64)
    op = hhg.Operator(c.mesh, kind="epsilon", degree=2, coeff=("field_p2", c.packed(mu, dtype)), bc=bc, quad_degree=4)
    K = OA.epsilon_matrix(c.S, ("field", c.S, mu), 4, bc)
    X = np.stack([W.uniform(3 * c.S.ndof, seed=s) for s in range(nrhs)], axis=1)   # (3*ndof, nrhs)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    xg = X.reshape(c.S.ndof, 3, nrhs)
    xp = torch.tensor(OL.to_packed(c.S, xg, 3, nrhs), dtype=dtype, device="cuda")
    y = op.apply(xp, nrhs=nrhs)
    ref = (K @ X).reshape(c.S.ndof, 3, nrhs)
    got_p = y.cpu().double().numpy()
    got = OL.from_packed(c.S, got_p, 3, nrhs).reshape(c.S.ndof, 3, nrhs)
    assert rel_err(got, ref) <= (1e-12 if dtype == torch.float64 else 1e-5), rel_err(got, ref)
    assert OL.copies_spread(c.S, got_p, 3, nrhs) == 0.0


@pytest.mark.parametrize("meshname,level", [("reference_tet", 2), ("cube6", 1), ("cube48", 1)])
@pytest.mark.parametrize("nrhs", [1, 16])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_epsilon_adjoint_parity(meshname, level, nrhs, bc):
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    c, mu = _case(meshname, level)
    op = hhg.Operator(c.mesh, kind="epsilon", degree=2, coeff=("field_p2", c.packed(mu)), bc=bc, quad_degree=4)
    U = np.stack([W.uniform(3 * c.S.ndof, seed=s) for s in range(nrhs)], axis=1)
    G = np.stack([W.uniform(3 * c.S.ndof, seed=100 + s) for s in range(nrhs)], axis=1)
    up = torch.tensor(OL.to_packed(c.S, U.reshape(c.S.ndof, 3, nrhs), 3, nrhs), device="cuda")
    gp = torch.tensor(OL.to_packed(c.S, G.reshape(c.S.ndof, 3, nrhs), 3, nrhs), device="cuda")
    dmu = op.adjoint_coeff(up, gp, nrhs=nrhs)
    ref = sum(OA.epsilon_coeff_adjoint(c.S, U[:, r], G[:, r], 4, bc) for r in range(nrhs))
    got, spread = c.unpack(dmu)
    assert rel_err(got, ref) <= 1e-12 and spread == 0.0
    # linearity in mu: sum_m mu_m dmu_m = sum_r g_r^T (A(mu) - A(0)) u_r
    K = OA.epsilon_matrix(c.S, ("field", c.S, mu), 4, bc)
    K0 = OA.epsilon_matrix(c.S, ("field", c.S, np.zeros_like(mu)), 4, bc)
    assert np.isclose(mu @ got, np.sum(G * ((K - K0) @ U)), rtol=1e-11)


def test_epsilon_rigid_body_modes_neumann():
    """A r = 0 for the six rigid-body motions (Neumann), through the batched apply."""
    import paper_2404_08371_gb300 as hhg
    c, mu = _case("cube48", 1)
    op = hhg.Operator(c.mesh, kind="epsilon", degree=2, coeff=("field_p2", c.packed(mu)), bc="neumann", quad_degree=4)
    modes = [np.tile(np.eye(3)[a], c.S.ndof) for a in range(3)] + \
            [np.cross(w[None, :], c.S.coords).reshape(-1) for w in np.eye(3)]
    X = np.stack(modes, axis=1)
    xp = torch.tensor(OL.to_packed(c.S, X.reshape(c.S.ndof, 3, 6), 3, 6), device="cuda")
    y = op.apply(xp, nrhs=6).cpu().numpy()
    K = OA.epsilon_matrix(c.S, ("field", c.S, mu), 4, "neumann")
    scale = abs(K).max() * np.abs(X).max()
    assert np.abs(y).max() <= 1e-12 * scale * 10


def test_epsilon_batch_sizes_on_one_operator():
    """One operator applied with 3, 16 and again 3 right-hand sides (the task lists are built at the
    first call of each batch size and kept); more than 256 right-hand sides are refused."""
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    c, mu = _case("cube6", 1)
    op = hhg.Operator(c.mesh, kind="epsilon", degree=2, coeff=("field_p2", c.packed(mu)), bc="dirichlet",
                      quad_degree=4)
    K = OA.epsilon_matrix(c.S, ("field", c.S, mu), 4, "dirichlet")
    for nrhs in (3, 16, 3):
        X = np.stack([W.uniform(3 * c.S.ndof, seed=40 + s) for s in range(nrhs)], axis=1)
        xp = torch.tensor(OL.to_packed(c.S, X.reshape(c.S.ndof, 3, nrhs), 3, nrhs), device="cuda")
        got = OL.from_packed(c.S, op.apply(xp, nrhs=nrhs).cpu().numpy(), 3, nrhs).reshape(c.S.ndof, 3, nrhs)
        assert rel_err(got, (K @ X).reshape(c.S.ndof, 3, nrhs)) <= 1e-12
    xb = torch.zeros(c.mesh.vec_size(2) * 3 * 257, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="256"):
        op.apply(xb, nrhs=257)


@pytest.mark.parametrize("level", [2, 3])
@pytest.mark.parametrize("nrhs", [1, 16])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_epsilon_cube48_assembled(level, nrhs, bc):
    """The 48-macro cube of the batched epsilon workload at levels 2 and 3 (4 and 8 cubes per
    macro edge, ragged parity passes and several CTAs per macro), every point against the
    assembled operator, and the mu-adjoint summed over the right-hand sides."""
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    c, mu = _case("cube48", level)
    op = hhg.Operator(c.mesh, kind="epsilon", degree=2, coeff=("field_p2", c.packed(mu)), bc=bc, quad_degree=4)
    X = np.stack([W.uniform(3 * c.S.ndof, seed=20 + s) for s in range(nrhs)], axis=1)
    G = np.stack([W.uniform(3 * c.S.ndof, seed=60 + s) for s in range(nrhs)], axis=1)
    xp = torch.tensor(OL.to_packed(c.S, X.reshape(c.S.ndof, 3, nrhs), 3, nrhs), device="cuda")
    gp = torch.tensor(OL.to_packed(c.S, G.reshape(c.S.ndof, 3, nrhs), 3, nrhs), device="cuda")
    K = OA.epsilon_matrix(c.S, ("field", c.S, mu), 4, bc)
    y = op.apply(xp, nrhs=nrhs).cpu().numpy()
    got = OL.from_packed(c.S, y, 3, nrhs).reshape(c.S.ndof, 3, nrhs)
    assert rel_err(got, (K @ X).reshape(c.S.ndof, 3, nrhs)) <= 1e-12
    assert OL.copies_spread(c.S, y, 3, nrhs) == 0.0
    dmu, spread = c.unpack(op.adjoint_coeff(xp, gp, nrhs=nrhs))
    ref = OA.epsilon_coeff_adjoint(c.S, X, G, 4, bc)
    assert rel_err(dmu, ref) <= 1e-12 and spread == 0.0


@pytest.fixture(scope="module")
def eps_full():
    """The batched epsilon workload at its full size: unit cube as 48 macros at level 6 (64 cubes
    per macro edge, 17.6 M stored P2 points), 16 right-hand sides, mu = 10^(3(z - 0.5)) as a P2
    field.  Inputs come from the keyed counter-based generator (equal values at every copy of a
    shared point), so the oracle regenerates x and g at the few points it needs."""
    import paper_2404_08371_gb300 as hhg
    from oracle import mesh as OM
    level, nrhs = 6, 16
    v, t = W.cube48()
    mm = OM.MacroMesh(v, t)
    N = 2 ** (level + 1)
    pts = OM.lattice_points(N)
    P = len(pts)
    mesh = hhg.Mesh(v, t, level)
    assert mesh.vec_size(2) == P * len(t)
    x = torch.empty((len(t) * P, 3 * nrhs), dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    mu_p = np.empty(len(t) * P)
    for m in range(len(t)):
        keys = OM.point_keys(mm.tets[m], pts, N)
        x[m * P:(m + 1) * P] = torch.from_numpy(W.uniform_keyed(keys, 3 * nrhs, 1))
        g[m * P:(m + 1) * P] = torch.from_numpy(W.uniform_keyed(keys, 3 * nrhs, 2))
        mu_p[m * P:(m + 1) * P] = W.viscosity_mu(OM.physical(v[t[m]], pts, N))

    def at(seed):
        def f(m, q):
            return W.uniform_keyed(OM.point_keys(mm.tets[m], np.asarray(q), N), 3 * nrhs, seed).reshape(-1, 3, nrhs)
        return f

    rng = np.random.default_rng(11)
    w = np.stack([N - pts.sum(axis=1), pts[:, 0], pts[:, 1], pts[:, 2]], axis=1)
    zeros = (w == 0).sum(axis=1)
    samples = [(int(m), pts[rng.integers(P)]) for m in rng.integers(len(t), size=60)]
    for z in (1, 2, 3):                      # faces (shared or boundary), edges, vertices
        cand = np.nonzero(zeros == z)[0]
        samples += [(int(m), pts[rng.choice(cand)]) for m in rng.integers(len(t), size=12)]
    pos = torch.tensor([m * P + int(OM.packed_position(p[None], N)[0]) for m, p in samples], device="cuda")
    return dict(level=level, nrhs=nrhs, mm=mm, mesh=mesh, x=x.view(-1), g=g.view(-1), mu_p=mu_p,
                xat=at(1), gat=at(2), samples=samples, pos=pos)


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_epsilon_full_size_sampled(eps_full, bc):
    """The bench's epsilon launch configuration (48 macros, level 6, 16 right-hand sides, FP64):
    the apply at sampled points of every kind and the mu-adjoint at the same points against the
    oracle's point-by-point sums over the micro-tets of every macro that stores the point."""
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    F = eps_full
    nrhs = F["nrhs"]
    mu_t = torch.from_numpy(F["mu_p"]).to("cuda")
    op = hhg.Operator(F["mesh"], kind="epsilon", degree=2, coeff=("field_p2", mu_t), bc=bc, quad_degree=4)
    y = op.apply(F["x"], nrhs=nrhs)
    got = y.view(-1, 3, nrhs)[F["pos"]].cpu().numpy()
    del y
    ref = OA.sampled_epsilon_rows(F["mm"], F["level"], F["mu_p"], F["xat"], F["samples"], 4, bc)
    assert rel_err(got, ref) <= 1e-12, rel_err(got, ref)
    dmu = op.adjoint_coeff(F["x"], F["g"], nrhs=nrhs)
    got_d = dmu[F["pos"]].cpu().numpy()
    ref_d = OA.sampled_epsilon_adjoint(F["mm"], F["level"], F["xat"], F["gat"], F["samples"], 4, bc)
    assert rel_err(got_d, ref_d) <= 1e-12, rel_err(got_d, ref_d)
