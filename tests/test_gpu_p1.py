"""P1 constant-coefficient apply through the C-ABI against the oracle (Eq. P1, Eq. 4.1)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import assemble as OA, layout as OL, mesh as OM

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@pytest.mark.parametrize("meshname,level", [("reference_tet", 0), ("reference_tet", 1), ("reference_tet", 4),
                                            ("reference_tet", 5), ("reference_tet", 6), ("cube6", 2), ("cube6", 3),
                                            ("cube6", 5), ("cube48", 2), ("cuboid36", 1), ("cuboid36", 4)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_p1_const_apply_parity(meshname, level, bc, dtype):
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, 1)
    op = hhg.Operator(c.mesh, degree=1, coeff=("const", 1.7), bc=bc)
    xg = W.uniform(c.S.ndof, seed=0)
    xg32 = xg.astype(np.float32).astype(np.float64) if dtype == torch.float32 else xg
    y = op.apply(c.packed(xg, dtype))
    ref = OA.diffusion_matrix(c.S, ("const", 1.7), 2, bc) @ xg32
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= TOL[dtype]
    assert spread == 0.0          # output is consistent: every copy of a shared point agrees


def test_config1_repeated_applies_bitwise():
    """Reference macro at level 4 (969 DoFs), zero Dirichlet, seed 0: 10 applies, identical results."""
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case("reference_tet", 4, 1)
    assert c.mesh.dof_count(1) == (969, 455)
    op = hhg.Operator(c.mesh, degree=1, coeff=("const", 1.0), bc="dirichlet")
    xg = W.uniform(c.S.ndof, seed=0)
    x = c.packed(xg)
    ref = OA.diffusion_matrix(c.S, ("const", 1.0), 2, "dirichlet") @ xg
    ys = [op.apply(x).cpu().numpy() for _ in range(10)]
    for y in ys:
        assert np.array_equal(y, ys[0])
    assert rel_err(OL.from_packed(c.S, ys[0]), ref) <= 1e-12


@pytest.mark.parametrize("meshname,level,degree", [("reference_tet", 3, 1), ("cube6", 2, 1), ("cube48", 1, 2),
                                                   ("cube6", 2, 2), ("cuboid36", 1, 1)])
def test_dof_counts(meshname, level, degree):
    from gpu_helpers import Case
    c = Case(meshname, level, degree)
    assert c.mesh.dof_count(degree) == (c.S.ndof, int(c.S.interior.sum()))


@pytest.mark.parametrize("meshname,level,degree", [("cube6", 2, 1), ("cube48", 1, 2)])
def test_make_consistent_and_dot(meshname, level, degree):
    from gpu_helpers import Case
    c = Case(meshname, level, degree)
    n = c.mesh.vec_size(degree)
    raw = torch.tensor(W.uniform(n, seed=3), device="cuda")
    x = c.mesh.make_consistent(raw.clone(), degree)
    xp = x.cpu().numpy()
    assert OL.copies_spread(c.S, xp) == 0.0
    # owner copy (lowest macro) kept
    assert np.array_equal(OL.from_packed(c.S, xp), OL.from_packed(c.S, raw.cpu().numpy()))
    y = c.mesh.make_consistent(torch.tensor(W.uniform(n, seed=4), device="cuda"), degree)
    d = c.mesh.dot(x, y, degree)
    ref = OL.from_packed(c.S, xp) @ OL.from_packed(c.S, y.cpu().numpy())
    assert abs(d - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("meshname,level", [("reference_tet", 3), ("cube6", 2)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_p1_const_diagonal(meshname, level, bc):
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, 1)
    op = hhg.Operator(c.mesh, degree=1, coeff=("const", 1.0), bc=bc)
    d = op.diagonal(torch.float64)
    ref = OA.diffusion_matrix(c.S, ("const", 1.0), 2, bc).diagonal()
    got, spread = c.unpack(d)
    assert rel_err(got, ref) <= 1e-12 and spread == 0.0


def test_p1_const_level8_sampled():
    """Full-size single macro (level 8, 2,862,209 DoFs): sampled rows against the oracle's per-point sum."""
    import paper_2404_08371_gb300 as hhg
    v, t = W.reference_tet()
    level = 8
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=1, coeff=("const", 1.0), bc="dirichlet")
    N = 2 ** level
    n = mesh.vec_size(1)
    assert n == 2862209
    xp = W.uniform(n, seed=0)
    y = op.apply(torch.tensor(xp, device="cuda")).cpu().numpy()
    pts = OM.lattice_points(N)
    rng = np.random.default_rng(1)
    sample = np.concatenate([rng.choice(n, 300, replace=False), [0, n - 1, n // 2]])
    # include points next to every face
    near = np.nonzero((pts.min(axis=1) == 1) | (pts.sum(axis=1) == N - 1))[0]
    sample = np.concatenate([sample, rng.choice(near, 100, replace=False)])
    ref = OA.sampled_diffusion_rows(v[t[0]], level, 1, ("const", 1.0), 2, "dirichlet", xp, pts[sample])
    assert np.abs(y[sample] - ref).max() <= 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("meshname,level,degree", [("cube48", 1, 2), ("reference_tet", 3, 1), ("cuboid36", 1, 1)])
def test_coordinates(meshname, level, degree):
    from gpu_helpers import Case
    c = Case(meshname, level, degree)
    xyz = c.mesh.coordinates(degree).cpu().numpy()
    ref = np.concatenate([OM.physical(c.v[c.t[m]], c.S.pts, c.S.N) for m in range(len(c.t))])
    assert np.abs(xyz - ref).max() <= 1e-15


@pytest.mark.parametrize("level", [7, 8])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_p1_const_f32_matches_f64_full_vector(level, bc):
    """Every point of the FP32 apply (register-climbing kernel + face blocks) at sizes with many
    k-chunks and row blocks, against the FP64 apply of the same FP32-representable input; the FP64
    apply is itself checked against the oracle's rows at level 8 (test_p1_const_level8_sampled), and
    the FP32 apply directly at level 9 (test_p1_const_f32_level9_sampled)."""
    import paper_2404_08371_gb300 as hhg
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=1, coeff=("const", 1.3), bc=bc)
    x32 = torch.tensor(W.uniform(mesh.vec_size(1), seed=4), device="cuda").float()
    y32 = op.apply(x32).double()
    y64 = op.apply(x32.double())
    assert torch.isfinite(y32).all()
    assert (y32 - y64).abs().max().item() <= 1e-5 * y64.abs().max().item()


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_p1_const_f32_level9_sampled(bc):
    """The bench's FP32 P1 constant-coefficient leg (reference macro, level 9, 22.6 M points, climbing
    kernel): sampled rows against the oracle's per-point sum on the FP32-rounded input (FP64)."""
    import paper_2404_08371_gb300 as hhg
    v, t = W.reference_tet()
    level = 9
    N = 2 ** level
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=1, coeff=("const", 1.0), bc=bc)
    n = mesh.vec_size(1)
    xp = W.uniform(n, seed=2).astype(np.float32)
    x = torch.from_numpy(xp).to("cuda")
    y = op.apply(x).cpu().numpy().astype(np.float64)
    pts = OM.lattice_points(N)
    rng = np.random.default_rng(5)
    near = np.nonzero((pts.min(axis=1) <= 1) | (pts.sum(axis=1) >= N - 1) | (pts[:, 2] >= N - 5))[0]
    sample = np.concatenate([rng.choice(n, 400, replace=False), rng.choice(near, 200, replace=False), [0, n - 1]])
    ref = OA.sampled_diffusion_rows(v[t[0]], level, 1, ("const", 1.0), 2, bc, xp.astype(np.float64), pts[sample])
    assert np.abs(y[sample] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_p1_const_f32_unaligned_view():
    """Vectors that do not start on a 16-byte boundary (a view one float in) give the same result."""
    import paper_2404_08371_gb300 as hhg
    from gpu_helpers import Case, rel_err
    c = Case("cube6", 5, 1)
    op = hhg.Operator(c.mesh, degree=1, coeff=("const", 1.0), bc="dirichlet")
    xg = W.uniform(c.S.ndof, seed=9)
    n = c.mesh.vec_size(1)
    buf = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    buf[1:] = c.packed(xg, torch.float32)
    ybuf = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    op.apply(buf[1:], out=ybuf[1:])
    ref = OA.diffusion_matrix(c.S, ("const", 1.0), 2, "dirichlet") @ xg.astype(np.float32).astype(np.float64)
    got, spread = c.unpack(ybuf[1:])
    assert rel_err(got, ref) <= 1e-5 and spread == 0.0


@pytest.mark.parametrize("meshname,level", [("reference_tet", 4), ("reference_tet", 6), ("cube6", 3), ("cube48", 2),
                                            ("cuboid36", 2)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_p1_const_double_float_parity(meshname, level, bc):
    """FP64 vectors with the arithmetic in FP32 pairs (48 significant bits) meet the FP64 tolerance
    against the oracle; switching back to native FP64 gives the FP64 kernel's result again."""
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, 1)
    op = hhg.Operator(c.mesh, degree=1, coeff=("const", 1.7), bc=bc)
    xg = W.uniform(c.S.ndof, seed=7)
    x = c.packed(xg)
    y_native = op.apply(x).clone()
    y = op.set_fp64_arith("double_float").apply(x)
    ref = OA.diffusion_matrix(c.S, ("const", 1.7), 2, bc) @ xg
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= 1e-12, rel_err(got, ref)
    assert spread == 0.0
    assert torch.equal(op.set_fp64_arith("native").apply(x), y_native)


def test_p1_const_double_float_level9_sampled():
    """The double-float apply at the bench's size (level 9, 22.6 M points): sampled rows against the
    oracle at the FP64 tolerance."""
    import paper_2404_08371_gb300 as hhg
    v, t = W.reference_tet()
    level = 9
    N = 2 ** level
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=1, coeff=("const", 1.0), bc="dirichlet").set_fp64_arith("double_float")
    n = mesh.vec_size(1)
    xp = W.uniform(n, seed=11)
    y = op.apply(torch.tensor(xp, device="cuda")).cpu().numpy()
    pts = OM.lattice_points(N)
    rng = np.random.default_rng(12)
    near = np.nonzero((pts.min(axis=1) <= 1) | (pts.sum(axis=1) >= N - 1))[0]
    sample = np.concatenate([rng.choice(n, 400, replace=False), rng.choice(near, 200, replace=False)])
    ref = OA.sampled_diffusion_rows(v[t[0]], level, 1, ("const", 1.0), 2, "dirichlet", xp, pts[sample])
    assert np.abs(y[sample] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_double_float_refused_for_other_operators():
    import paper_2404_08371_gb300 as hhg
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, 2)
    op = hhg.Operator(mesh, degree=2, coeff=("sin3",), bc="dirichlet", quad_degree=4)
    with pytest.raises(RuntimeError, match="P1 and P2 constant"):
        op.set_fp64_arith("double_float")
