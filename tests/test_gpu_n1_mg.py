"""The Nedelec multigrid of Section 8 on the GPU (Hiptmair's hybrid smoother, Eq. N1) through the
C-ABI, step by step against the oracle (oracle/mg_n1.py): edge prolongation and restriction, the
discrete gradient and its transpose, the diagonal, and the FMG solve against the direct solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import workloads as W
from oracle import assemble as OA, layout as OL, mesh as OM, mg_n1

pytestmark = pytest.mark.gpu

MESHES = [("reference_tet", 2), ("cube6", 2), ("cube48", 1), ("cuboid36", 1)]


def _setup(meshname, level):
    import paper_2404_08371_gb300 as hhg
    v, t = getattr(W, meshname)()
    mesh = hhg.Mesh(v, t, level)
    mm = OM.MacroMesh(v, t)
    return hhg, mesh, mm


@pytest.mark.parametrize("meshname,level", MESHES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_edge_prolongation(meshname, level, dtype):
    from gpu_helpers import rel_err
    hhg, mesh, mm = _setup(meshname, level)
    Sc, Sf = OA.EdgeSpace(mm, level - 1), OA.EdgeSpace(mm, level)
    P = mg_n1.edge_prolongation(Sc, Sf)
    xc = W.uniform(Sc.ndof, seed=3)
    if dtype == torch.float32:
        xc = xc.astype(np.float32).astype(np.float64)
    xf = mesh.prolongate_edges(torch.tensor(OL.n1_to_packed(Sc, xc), dtype=dtype, device="cuda"), level)
    got = xf.double().cpu().numpy()
    assert rel_err(OL.n1_from_packed(Sf, got), P @ xc) <= (1e-13 if dtype == torch.float64 else 1e-6)
    assert OL.n1_copies_spread(Sf, got) == 0.0


@pytest.mark.parametrize("meshname,level", MESHES)
def test_edge_restriction(meshname, level):
    """rc = P^T rf over distinct fine edges (rf with zero tangential boundary entries, as the
    V-cycle's residuals have), coarse boundary entries zero."""
    from gpu_helpers import rel_err
    hhg, mesh, mm = _setup(meshname, level)
    Sc, Sf = OA.EdgeSpace(mm, level - 1), OA.EdgeSpace(mm, level)
    P = mg_n1.edge_prolongation(Sc, Sf)
    rf = W.uniform(Sf.ndof, seed=4)
    rf[Sf.boundary] = 0.0
    ref = P.T @ rf
    ref[Sc.boundary] = 0.0
    rc = mesh.restrict_edges(torch.tensor(OL.n1_to_packed(Sf, rf), device="cuda"), level).cpu().numpy()
    assert rel_err(OL.n1_from_packed(Sc, rc), ref) <= 1e-13
    assert OL.n1_copies_spread(Sc, rc) == 0.0


@pytest.mark.parametrize("meshname,level", MESHES)
def test_gradient_and_transpose(meshname, level):
    """e = G p (tangential integrals of grad p) and p = G^T e over the interior vertices."""
    from gpu_helpers import rel_err
    hhg, mesh, mm = _setup(meshname, level)
    S = OA.EdgeSpace(mm, level)
    G = OA.n1_gradient(S)
    p = W.uniform(S.V1.ndof, seed=5)
    p[S.V1.boundary] = 0.0
    e = mesh.gradient(torch.tensor(OL.to_packed(S.V1, p), device="cuda")).cpu().numpy()
    assert rel_err(OL.n1_from_packed(S, e), G @ p) <= 1e-14
    assert OL.n1_copies_spread(S, e) == 0.0
    r = W.uniform(S.ndof, seed=6)
    ref = G.T @ r
    ref[S.V1.boundary] = 0.0
    q = mesh.gradient_transpose(torch.tensor(OL.n1_to_packed(S, r), device="cuda")).cpu().numpy()
    assert rel_err(OL.from_packed(S.V1, q), ref) <= 1e-13
    assert OL.copies_spread(S.V1, q) == 0.0


@pytest.mark.parametrize("meshname,level", MESHES + [("cube6", 6)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_n1_diagonal(meshname, level, bc):
    """diag(A) of the curl-curl + mass operator (orientation-free), Dirichlet rows 1; level 6 uses the
    marching tiles' shared faces."""
    from gpu_helpers import rel_err
    hhg, mesh, mm = _setup(meshname, level)
    S = OA.EdgeSpace(mm, level)
    xyz1 = mesh.coordinates(1)
    a_t, b_t = (1.0 + xyz1[:, 0] / 3.0).contiguous(), (1.0 + xyz1[:, 2]).contiguous()
    op = hhg.CurlCurl(mesh, ("field_p1", a_t), ("field_p1", b_t), bc=bc)
    a = S.V1.interpolate(lambda x: 1.0 + x[:, 0] / 3.0)
    b = S.V1.interpolate(lambda x: 1.0 + x[:, 2])
    K = OA.n1_matrix(S, ("field", S.V1, a), ("field", S.V1, b), 4, bc)
    d = op.diagonal(torch.float64).cpu().numpy()
    assert rel_err(np.abs(OL.n1_from_packed(S, d)), K.diagonal()) <= 1e-12


def _field(p):
    s = np.sin(np.pi * p)
    return (2 * np.pi ** 2 + 1) * np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], axis=1)


@pytest.mark.parametrize("meshname,level", [("cube6", 3), ("cuboid36", 2)])
@pytest.mark.parametrize("mixed", [0, 1])
def test_n1_fmg_matches_direct_solution(meshname, level, mixed):
    """FMG + V(2,2) with the hybrid smoother (FP64, or FP32 cycles inside FP64 refinement) reaches a
    relative residual of 1e-10 and the oracle's direct solution of the same system."""
    hhg, mesh, mm = _setup(meshname, level)
    S = OA.EdgeSpace(mm, level)
    b = mg_n1.load_vector(S, _field)
    K = OA.n1_matrix(S, ("const", 1.0), ("const", 1.0), 4, "dirichlet")
    xd = spla.spsolve(K.tocsc(), b)
    op = hhg.CurlCurl(mesh, ("const", 1.0), ("const", 1.0), bc="dirichlet")
    bp = torch.tensor(OL.n1_to_packed(S, b), device="cuda")
    x, st = op.mg_solve(bp, torch.zeros_like(bp), mixed=mixed)
    assert st["rel_residual"] <= 1e-10 and st["iterations"] <= 30, st
    got = OL.n1_from_packed(S, x.cpu().numpy())
    assert np.abs(got - xd).max() <= 1e-8 * np.abs(xd).max()
    assert OL.n1_copies_spread(S, x.cpu().numpy()) <= 1e-12 * np.abs(xd).max()
