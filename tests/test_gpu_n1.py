"""Lowest-order Nedelec curl-curl + mass operator (Eq. N1) through the C-ABI against the oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import assemble as OA, layout as OL, mesh as OM

pytestmark = pytest.mark.gpu
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _coeffs(S, kind, dtype):
    """(library alpha, library beta, oracle alpha, oracle beta)."""
    if kind == "const":
        return ("const", 1.3), ("const", 0.7), ("const", 1.3), ("const", 0.7)
    a = 1.0 + 0.5 * np.sin(3.0 * S.V1.coords[:, 0]) * np.cos(2.0 * S.V1.coords[:, 2])
    b = np.exp(W.fourier_field(S.V1.coords, seed=3))
    if dtype == torch.float32:
        a = a.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    ap = torch.tensor(OL.to_packed(S.V1, a), dtype=dtype, device="cuda")
    bp = torch.tensor(OL.to_packed(S.V1, b), dtype=dtype, device="cuda")
    return ("field_p1", ap), ("field_p1", bp), ("field", S.V1, a), ("field", S.V1, b)


@pytest.mark.parametrize("meshname,level", [("reference_tet", 0), ("reference_tet", 1), ("reference_tet", 3),
                                            ("cube6", 1), ("cube6", 2), ("cube48", 1), ("cuboid36", 1)])
@pytest.mark.parametrize("kind", ["const", "field"])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_n1_apply_parity(meshname, level, kind, bc, dtype):
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    v, t = getattr(W, meshname)()
    mesh = hhg.Mesh(v, t, level)
    S = OA.EdgeSpace(OM.MacroMesh(v, t), level)
    la, lb, oa, ob = _coeffs(S, kind, dtype)
    op = hhg.CurlCurl(mesh, la, lb, bc=bc)
    xg = W.uniform(S.ndof, seed=0)
    if dtype == torch.float32:
        xg = xg.astype(np.float32).astype(np.float64)
    xp = torch.tensor(OL.n1_to_packed(S, xg), dtype=dtype, device="cuda")
    y = op.apply(xp).double().cpu().numpy()
    ref = OA.n1_matrix(S, oa, ob, 4, bc) @ xg
    assert rel_err(OL.n1_from_packed(S, y), ref) <= TOL[dtype]
    assert OL.n1_copies_spread(S, y) <= 1e-13 * np.abs(ref).max() * (1 if dtype == torch.float64 else 1e7)
    # vertex entries stay zero
    N2 = 2 * 2 ** level
    vert = np.ones(OM.lattice_size(N2), dtype=bool)
    vert[S.edge_pos] = False
    assert np.all(y.reshape(len(t), -1)[:, vert] == 0.0)


def test_n1_apply_parity_atomic_tiles():
    """Level 6 (64 cubes per edge): the marching tiles add the points on their i- and j-faces
    atomically; every edge checked."""
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, 6)
    S = OA.EdgeSpace(OM.MacroMesh(v, t), 6)
    la, lb, oa, ob = _coeffs(S, "field", torch.float64)
    op = hhg.CurlCurl(mesh, la, lb, bc="dirichlet")
    xg = W.uniform(S.ndof, seed=0)
    xp = torch.tensor(OL.n1_to_packed(S, xg), dtype=torch.float64, device="cuda")
    y = op.apply(xp).cpu().numpy()
    ref = OA.n1_matrix(S, oa, ob, 4, "dirichlet") @ xg
    assert rel_err(OL.n1_from_packed(S, y), ref) <= TOL[torch.float64]


def test_n1_gradients_in_kernel_level3():
    """curl-curl on discrete gradients vanishes through the GPU apply (Neumann, beta = 0)."""
    import paper_2404_08371_gb300 as hhg
    v, t = W.cube6()
    level = 3
    mesh = hhg.Mesh(v, t, level)
    S = OA.EdgeSpace(OM.MacroMesh(v, t), level)
    op = hhg.CurlCurl(mesh, ("const", 1.0), ("const", 0.0), bc="neumann")
    p = W.uniform(S.V1.ndof, seed=4)
    gp = OA.n1_gradient(S) @ p
    y = op.apply(torch.tensor(OL.n1_to_packed(S, gp), device="cuda")).cpu().numpy()
    K = OA.n1_matrix(S, ("const", 1.0), ("const", 0.0), 4, "neumann")
    assert np.abs(OL.n1_from_packed(S, y)).max() <= 1e-12 * abs(K).max() * np.abs(gp).max() * 10


@pytest.mark.parametrize("meshname,level", [("reference_tet", 3), ("cube6", 2), ("cuboid36", 1)])
@pytest.mark.parametrize("kind", ["const", "field"])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_n1_stored_element_matrices_parity(meshname, level, kind, bc, dtype):
    """Precomputed variant of the Nedelec operator: the 21 entries per micro-tet stored once, then
    applied; the same operator as the matrix-free apply."""
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    v, t = getattr(W, meshname)()
    mesh = hhg.Mesh(v, t, level)
    S = OA.EdgeSpace(OM.MacroMesh(v, t), level)
    la, lb, oa, ob = _coeffs(S, kind, dtype)
    op = hhg.CurlCurl(mesh, la, lb, bc=bc)
    xg = W.uniform(S.ndof, seed=2)
    if dtype == torch.float32:
        xg = xg.astype(np.float32).astype(np.float64)
    xp = torch.tensor(OL.n1_to_packed(S, xg), dtype=dtype, device="cuda")
    y_free = op.apply(xp)
    op.store_element_matrices(dtype)
    y = op.apply(xp)
    ref = OA.n1_matrix(S, oa, ob, 4, bc) @ xg
    assert rel_err(OL.n1_from_packed(S, y.double().cpu().numpy()), ref) <= TOL[dtype]
    assert torch.allclose(y, y_free, rtol=0, atol=(1e-13 if dtype == torch.float64 else 2e-6) * y_free.abs().max().item())
    op.drop_element_matrices()
    assert torch.equal(op.apply(xp), y_free)
