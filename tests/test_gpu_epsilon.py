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
    """One operator applied with 3, 16 and again 3 right-hand sides (the per-launch task lists are
    rebuilt when the batch size changes); more than 256 right-hand sides are refused."""
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
