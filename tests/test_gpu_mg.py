"""Multigrid pieces through the C-ABI against the oracle (Section 8): transfers, smoother, power
iteration, load vector, L2 error, and full FMG / iterative-refinement solves."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import workloads as W
from oracle import assemble as OA, layout as OL, mesh as OM, mg as OMG

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _spaces(meshname, level, degree):
    v, t = getattr(W, meshname)()
    mm = OM.MacroMesh(v, t)
    return mm, OA.Space(mm, level - 1, degree), OA.Space(mm, level, degree)


@pytest.mark.parametrize("meshname,level", [("reference_tet", 1), ("reference_tet", 3), ("cube6", 2), ("cube48", 1),
                                            ("cuboid36", 1)])
@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_transfer_parity(meshname, level, degree, dtype):
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import rel_err
    mm, Sc, Sf = _spaces(meshname, level, degree)
    v, t = getattr(W, meshname)()
    mesh = hhg.Mesh(v, t, level)
    P = OMG.prolongation(Sc, Sf)
    xc = W.uniform(Sc.ndof, seed=0)
    rf = W.uniform(Sf.ndof, seed=1)
    if dtype == torch.float32:
        xc = xc.astype(np.float32).astype(np.float64)
        rf = rf.astype(np.float32).astype(np.float64)
    xf = mesh.prolongate(torch.tensor(OL.to_packed(Sc, xc), dtype=dtype, device="cuda"), degree, level)
    got = xf.cpu().double().numpy()
    assert OL.copies_spread(Sf, got) == 0.0
    assert rel_err(OL.from_packed(Sf, got), P @ xc) <= TOL[dtype]
    rc = mesh.restrict(torch.tensor(OL.to_packed(Sf, rf), dtype=dtype, device="cuda"), degree, level)
    ref = P.T @ rf
    ref[Sc.boundary] = 0.0
    got = rc.cpu().double().numpy()
    assert OL.copies_spread(Sc, got) == 0.0
    assert rel_err(OL.from_packed(Sc, got), ref) <= TOL[dtype]


def _op_and_oracle(meshname, level, degree, coeff, dtype=torch.float64):
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import Case
    c = Case(meshname, level, degree)
    qd = 2 if degree == 1 else 4
    op = hhg.Operator(c.mesh, degree=degree, coeff=coeff, bc="dirichlet", quad_degree=qd)
    A = OA.diffusion_matrix(c.S, coeff, qd, "dirichlet")
    return c, op, A


@pytest.mark.parametrize("meshname,level,degree,coeff", [("reference_tet", 3, 1, ("const", 1.0)),
                                                         ("cube6", 2, 2, ("sin3",)), ("cube48", 1, 2, ("const", 1.0)),
                                                         ("cube6", 3, 1, ("sin3",))])
@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_chebyshev_parity(meshname, level, degree, coeff, order, dtype):
    from gpu_helpers import rel_err
    c, op, A = _op_and_oracle(meshname, level, degree, coeff)
    dinv = 1.0 / A.diagonal()
    b = W.uniform(c.S.ndof, seed=3)
    x = W.uniform(c.S.ndof, seed=4)
    if dtype == torch.float32:
        b, x, dinv = (a.astype(np.float32).astype(np.float64) for a in (b, x, dinv))
    lam = 1.7
    ref = OMG.chebyshev(A, dinv, b, x, lam, order)
    xt = c.packed(x, dtype)
    op.cheb_smooth(c.packed(b, dtype), xt, c.packed(dinv, dtype), lam, 0.1, 1.1, order)
    got, spread = c.unpack(xt)
    assert rel_err(got, ref) <= (TOL[dtype] if dtype == torch.float64 else 5e-5)
    # a second call continues from the first one's result
    ref2 = OMG.chebyshev(A, dinv, b, ref, lam, order)
    op.cheb_smooth(c.packed(b, dtype), xt, c.packed(dinv, dtype), lam, 0.1, 1.1, order)
    got2, _ = c.unpack(xt)
    assert rel_err(got2, ref2) <= (TOL[dtype] if dtype == torch.float64 else 1e-4)


@pytest.mark.parametrize("meshname,level,degree,coeff", [("cube6", 2, 1, ("const", 1.0)), ("cube6", 2, 2, ("sin3",)),
                                                         ("reference_tet", 3, 2, ("const", 1.0))])
def test_power_iteration_parity(meshname, level, degree, coeff):
    c, op, A = _op_and_oracle(meshname, level, degree, coeff)
    dinv = 1.0 / A.diagonal()
    v0 = W.uniform(c.S.ndof, seed=5)
    v0[c.S.boundary] = 0.0
    lam_ref = OMG.power_iteration(A, dinv, v0, 15)
    v = c.packed(v0)
    lam = op.power_iteration(c.packed(dinv), v, 15)
    assert abs(lam - lam_ref) <= 1e-12 * lam_ref


@pytest.mark.parametrize("meshname,level", [("cube6", 1), ("cube6", 2), ("cube48", 1), ("reference_tet", 3)])
@pytest.mark.parametrize("degree", [1, 2])
def test_rhs_and_l2_error_parity(meshname, level, degree):
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import Case, rel_err
    c = Case(meshname, level, degree)
    b = c.mesh.rhs_sin3_poisson(degree)
    got, spread = c.unpack(b)
    ref = OMG.load_vector(c.S, W.manufactured_f, 5)
    assert spread == 0.0 and rel_err(got, ref) <= 1e-12
    uh = W.uniform(c.S.ndof, seed=6) * 0.1 + c.S.interpolate(W.manufactured_u)
    e = c.mesh.l2_error_sin3(c.packed(uh), degree)
    e_ref = OMG.l2_error(c.S, uh, W.manufactured_u, 5)
    assert abs(e - e_ref) <= 1e-12 * e_ref


@pytest.mark.parametrize("degree,level", [(1, 4), (2, 3)])
@pytest.mark.parametrize("mixed", [0, 1])
def test_mg_solve_matches_direct_solution(degree, level, mixed):
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import Case
    c = Case("cube6", level, degree)
    op = hhg.Operator(c.mesh, degree=degree, coeff=("const", 1.0), bc="dirichlet", quad_degree=2 if degree == 1 else 4)
    b = c.mesh.rhs_sin3_poisson(degree)
    x = torch.zeros_like(b)
    x, st = op.mg_solve(b, x, mixed=mixed, tol=1e-10)
    assert st["rel_residual"] <= 1e-10 and st["iterations"] <= 15
    hist = st["history"]
    assert all(hist[i + 1] < hist[i] for i in range(len(hist) - 1))
    A = OA.diffusion_matrix(c.S, ("const", 1.0), 2 if degree == 1 else 4, "dirichlet")
    bg, _ = c.unpack(b)
    xs = spla.spsolve(A.tocsc(), bg)
    got, spread = c.unpack(x)
    assert spread == 0.0
    assert np.abs(got - xs).max() <= 1e-8 * np.abs(xs).max()
    # V-cycle contraction well below one
    rates = [hist[i + 1] / hist[i] for i in range(1, len(hist) - 1)]
    assert max(rates) < 0.3, rates


def test_mg_solve_discretisation_order_and_status():
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import Case
    errs = []
    for level in (1, 2, 3):
        c = Case("cube6", level, 2)
        op = hhg.Operator(c.mesh, degree=2, coeff=("const", 1.0), bc="dirichlet", quad_degree=4)
        b = c.mesh.rhs_sin3_poisson(2)
        x, st = op.mg_solve(b, torch.zeros_like(b), mixed=1, tol=1e-10)
        errs.append(c.mesh.l2_error_sin3(x, 2))
    r = errs[-1] / errs[-2]
    assert 0.09 < r < 0.16, errs     # O(h^3) in L2 for P2
    # not converged within the iteration cap: status and last iterate returned
    with pytest.raises(hhg.HHGError) as ei:
        op.mg_solve(b, torch.zeros_like(b), max_iters=1, tol=1e-14)
    assert ei.value.code == hhg._lib.HHG_E_NOT_CONVERGED
    # unsupported operator
    opn = hhg.Operator(c.mesh, degree=2, coeff=("const", 1.0), bc="neumann", quad_degree=4)
    with pytest.raises(hhg.HHGError) as ei:
        opn.mg_solve(b, torch.zeros_like(b))
    assert ei.value.code == hhg._lib.HHG_E_UNSUPPORTED
