"""Variable-coefficient and P2 operators through the C-ABI against the oracle (Eq. P2V, Eq. 6.1, Algorithm 1)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import assemble as OA, layout as OL

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
QD = {1: 2, 2: 4}


def _coeff(case, kind, dtype):
    """(library coefficient, oracle coefficient, rounded-input flag)."""
    if kind == "const":
        return ("const", 1.3), ("const", 1.3)
    if kind == "sin3":
        return ("sin3",), ("sin3",)
    kg = np.exp(W.fourier_field(case.S.coords, seed=0))
    if dtype == torch.float32:
        kg = kg.astype(np.float32).astype(np.float64)
    field = case.packed(kg, dtype)
    return ("field_p%d" % case.degree, field), ("field", case.S, kg)


CASES = [("reference_tet", 0), ("reference_tet", 1), ("reference_tet", 3), ("cube6", 2), ("cube48", 1), ("cuboid36", 1)]


@pytest.mark.parametrize("meshname,level", CASES)
@pytest.mark.parametrize("degree,kind", [(1, "sin3"), (1, "field"), (2, "const"), (2, "sin3"), (2, "field")])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_apply_parity(meshname, level, degree, kind, bc, dtype):
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, degree)
    lc, oc = _coeff(c, kind, dtype)
    op = hhg.Operator(c.mesh, degree=degree, coeff=lc, bc=bc, quad_degree=QD[degree])
    xg = W.uniform(c.S.ndof, seed=0)
    if dtype == torch.float32:
        xg = xg.astype(np.float32).astype(np.float64)
    y = op.apply(c.packed(xg, dtype))
    ref = OA.diffusion_matrix(c.S, oc, QD[degree], bc) @ xg
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= TOL[dtype], rel_err(got, ref)
    assert spread == 0.0


@pytest.mark.parametrize("meshname,level", [("reference_tet", 5), ("cube6", 4), ("cube6", 5), ("cuboid36", 3)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_p2_const_parity_large(meshname, level, bc, dtype):
    """P2 constant coefficient (stencil rows per node parity) at sizes with many interior rows; from 64
    intervals per edge on, FP32 runs the plane-tile kernel launched once per macro (cube6 level 5)."""
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, 2)
    op = hhg.Operator(c.mesh, degree=2, coeff=("const", 0.8), bc=bc, quad_degree=QD[2])
    xg = W.uniform(c.S.ndof, seed=4)
    if dtype == torch.float32:
        xg = xg.astype(np.float32).astype(np.float64)
    y = op.apply(c.packed(xg, dtype))
    ref = OA.diffusion_matrix(c.S, ("const", 0.8), QD[2], bc) @ xg
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= TOL[dtype], rel_err(got, ref)
    assert spread == 0.0


@pytest.mark.parametrize("meshname,level", [("reference_tet", 3), ("reference_tet", 5), ("cube6", 5), ("cuboid36", 3)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_p2_const_double_float_parity(meshname, level, bc):
    """P2 constant coefficient with FP64 vectors and the arithmetic in FP32 pairs (the two-plane kernel
    from 64 intervals per edge on, FP64 below) meets the FP64 tolerance against the oracle; switching
    back to native FP64 gives the FP64 kernel's result again."""
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, 2)
    op = hhg.Operator(c.mesh, degree=2, coeff=("const", 0.8), bc=bc, quad_degree=QD[2])
    xg = W.uniform(c.S.ndof, seed=5)
    x = c.packed(xg)
    y_native = op.apply(x).clone()
    y = op.set_fp64_arith("double_float").apply(x)
    ref = OA.diffusion_matrix(c.S, ("const", 0.8), QD[2], bc) @ xg
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= TOL[torch.float64], rel_err(got, ref)
    assert spread == 0.0
    assert torch.equal(op.set_fp64_arith("native").apply(x), y_native)


@pytest.mark.parametrize("meshname,level", [("reference_tet", 2), ("cube6", 1), ("cube48", 1)])
@pytest.mark.parametrize("degree,kind", [(1, "sin3"), (1, "field"), (2, "const"), (2, "sin3"), (2, "field")])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_diagonal_parity(meshname, level, degree, kind, bc):
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, degree)
    lc, oc = _coeff(c, kind, torch.float64)
    op = hhg.Operator(c.mesh, degree=degree, coeff=lc, bc=bc, quad_degree=QD[degree])
    d = op.diagonal(torch.float64)
    ref = OA.diffusion_matrix(c.S, oc, QD[degree], bc).diagonal()
    got, spread = c.unpack(d)
    assert rel_err(got, ref) <= 1e-12 and spread == 0.0


@pytest.mark.parametrize("meshname,level", [("reference_tet", 0), ("reference_tet", 3), ("cube6", 2), ("cube48", 1)])
@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_adjoint_parity(meshname, level, degree, bc, dtype):
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, degree)
    lc, oc = _coeff(c, "field", dtype)
    op = hhg.Operator(c.mesh, degree=degree, coeff=lc, bc=bc, quad_degree=QD[degree])
    u = W.uniform(c.S.ndof, seed=1)
    g = W.uniform(c.S.ndof, seed=2)
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
        g = g.astype(np.float32).astype(np.float64)
    dk = op.adjoint_coeff(c.packed(u, dtype), c.packed(g, dtype))
    ref = OA.diffusion_coeff_adjoint(c.S, c.S, u, g, QD[degree], bc)
    got, spread = c.unpack(dk)
    assert rel_err(got, ref) <= (1e-12 if dtype == torch.float64 else 2e-5), rel_err(got, ref)
    assert spread == 0.0


# Level 6 (64 cubes per edge) is the smallest lattice on which the marching tiles own every column
# of cubes and the points on their i- and j-faces collect the partial sums of the neighbouring
# tiles through the per-operator face scratch; every point checked here.
@pytest.mark.parametrize("meshname,degree,kind,bc,dtype", [
    ("reference_tet", 2, "sin3", "dirichlet", torch.float64),
    ("reference_tet", 2, "sin3", "dirichlet", torch.float32),
    ("reference_tet", 1, "sin3", "neumann", torch.float64),
    ("cube6", 1, "sin3", "dirichlet", torch.float64),
    ("cube6", 1, "field", "neumann", torch.float64),
])
def test_apply_parity_atomic_tiles(meshname, degree, kind, bc, dtype):
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, 6, degree)
    lc, oc = _coeff(c, kind, dtype)
    op = hhg.Operator(c.mesh, degree=degree, coeff=lc, bc=bc, quad_degree=QD[degree])
    xg = W.uniform(c.S.ndof, seed=0)
    if dtype == torch.float32:
        xg = xg.astype(np.float32).astype(np.float64)
    y = op.apply(c.packed(xg, dtype))
    ref = OA.diffusion_matrix(c.S, oc, QD[degree], bc) @ xg
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= TOL[dtype], rel_err(got, ref)
    assert spread == 0.0


def test_diagonal_and_adjoint_atomic_tiles():
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case("reference_tet", 6, 1)
    lc, oc = _coeff(c, "field", torch.float64)
    op = hhg.Operator(c.mesh, degree=1, coeff=lc, bc="dirichlet", quad_degree=QD[1])
    d = op.diagonal(torch.float64)
    got, _ = c.unpack(d)
    assert rel_err(got, OA.diffusion_matrix(c.S, oc, QD[1], "dirichlet").diagonal()) <= 1e-12
    u = W.uniform(c.S.ndof, seed=1)
    g = W.uniform(c.S.ndof, seed=2)
    dk = op.adjoint_coeff(c.packed(u, torch.float64), c.packed(g, torch.float64))
    got, _ = c.unpack(dk)
    assert rel_err(got, OA.diffusion_coeff_adjoint(c.S, c.S, u, g, QD[1], "dirichlet")) <= 1e-12


def test_field_dtype_mismatch_rejected():
    from gpu_helpers import Case
    import paper_2404_08371_gb300 as hhg
    c = Case("reference_tet", 1, 1)
    lc, _ = _coeff(c, "field", torch.float64)
    op = hhg.Operator(c.mesh, degree=1, coeff=lc)
    with pytest.raises(hhg.HHGError):
        op.apply(torch.zeros(c.mesh.vec_size(1), dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("degree", [1, 2])
def test_level8_sampled_sin3(degree):
    """The level-8 workload: sampled rows of the analytic-coefficient apply against the oracle's per-point sums."""
    import paper_2404_08371_gb300 as hhg
    from oracle import mesh as OM
    v, t = W.reference_tet()
    level = 8
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=degree, coeff=("sin3",), bc="dirichlet", quad_degree=QD[degree])
    N = degree * 2 ** level
    n = mesh.vec_size(degree)
    xp = W.uniform(n, seed=0)
    y = op.apply(torch.tensor(xp, device="cuda")).cpu().numpy()
    rng = np.random.default_rng(2)
    sample = rng.choice(n, 200, replace=False)
    pts = np.empty((len(sample), 3), dtype=np.int64)
    # lattice points of the sampled packed positions (from the layout definition)
    allpos = OM.packed_position
    planes = np.array([OM.lattice_size(N) - OM.lattice_size(N - k) for k in range(N + 2)])
    for e, p in enumerate(sample):
        k = np.searchsorted(planes, p, side="right") - 1
        q = p - planes[k]
        s = N - k
        j = 0
        while (j + 1) * (s + 1) - (j + 1) * j // 2 <= q:
            j += 1
        i = q - (j * (s + 1) - j * (j - 1) // 2)
        pts[e] = (i, j, k)
        assert allpos(pts[e:e + 1], N)[0] == p
    ref = OA.sampled_diffusion_rows(v[t[0]], level, degree, ("sin3",), QD[degree], "dirichlet", xp, pts)
    assert np.abs(y[sample] - ref).max() <= 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("meshname,level", [("reference_tet", 3), ("cube6", 2), ("cube48", 1)])
@pytest.mark.parametrize("kind", ["sin3", "field"])
@pytest.mark.parametrize("qd", [1, 2])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_p2_under_integration_parity(meshname, level, kind, qd, dtype):
    """P2 variable coefficient with a rule of degree 2 (4 points) or 1: the paper's under-integration (U)."""
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, 2)
    lc, oc = _coeff(c, kind, dtype)
    op = hhg.Operator(c.mesh, degree=2, coeff=lc, bc="dirichlet", quad_degree=qd)
    xg = W.uniform(c.S.ndof, seed=0)
    if dtype == torch.float32:
        xg = xg.astype(np.float32).astype(np.float64)
    y = op.apply(c.packed(xg, dtype))
    ref = OA.diffusion_matrix(c.S, oc, qd, "dirichlet") @ xg
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= TOL[dtype] and spread == 0.0


@pytest.mark.parametrize("meshname,level", [("reference_tet", 0), ("reference_tet", 3), ("cube6", 2), ("cuboid36", 1)])
@pytest.mark.parametrize("degree,kind", [(1, "sin3"), (1, "field"), (2, "sin3"), (2, "field")])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_stored_element_matrices_parity(meshname, level, degree, kind, bc, dtype):
    """Precomputed variant: local matrices integrated once and stored, then applied; the same
    operator as the matrix-free apply (oracle parity), other dtypes keep the matrix-free path."""
    from gpu_helpers import Case, rel_err
    import paper_2404_08371_gb300 as hhg
    c = Case(meshname, level, degree)
    lc, oc = _coeff(c, kind, dtype)
    op = hhg.Operator(c.mesh, degree=degree, coeff=lc, bc=bc, quad_degree=QD[degree])
    xg = W.uniform(c.S.ndof, seed=5)
    if dtype == torch.float32:
        xg = xg.astype(np.float32).astype(np.float64)
    xp = c.packed(xg, dtype)
    y_free = op.apply(xp)
    op.store_element_matrices(dtype)
    y = op.apply(xp)
    ref = OA.diffusion_matrix(c.S, oc, QD[degree], bc) @ xg
    got, spread = c.unpack(y)
    assert rel_err(got, ref) <= TOL[dtype], rel_err(got, ref)
    assert spread == 0.0
    assert torch.allclose(y, y_free, rtol=0, atol=(1e-13 if dtype == torch.float64 else 2e-6) * y_free.abs().max().item())
    other = torch.float32 if dtype == torch.float64 else torch.float64
    if kind == "sin3":   # the other dtype still takes the matrix-free path
        y_other = op.apply(xp.to(other))
        assert rel_err(c.unpack(y_other)[0], ref) <= 1e-5
    op.drop_element_matrices()
    assert torch.equal(op.apply(xp), y_free)


def _sampled_points(N, n, rng, count=300):
    """Sampled packed positions of a single-macro lattice of resolution N (plus points next to every
    face and the first / last positions) and their lattice points."""
    from oracle import mesh as OM
    pts = OM.lattice_points(N)
    near = np.nonzero((pts.min(axis=1) == 1) | (pts.sum(axis=1) == N - 1))[0]
    sample = np.unique(np.concatenate([rng.choice(n, count, replace=False), rng.choice(near, 100, replace=False),
                                       [0, n - 1, n // 2]]))
    return sample, pts[sample]


@pytest.mark.parametrize("degree,coeff,level,stored", [(1, "sin3", 8, False), (2, "sin3", 8, False),
                                                        (1, "const", 9, False), (2, "const", 8, False),
                                                        (2, "sin3", 8, True), (1, "sin3", 8, True)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_bench_legs_full_size_sampled(degree, coeff, level, stored, dtype):
    """The bench's legs at full size, in the launch configuration it times (single macro, Dirichlet,
    the leg's rule; constant-coefficient legs at their levels 8 / 9; the precomputed variant):
    sampled rows against the oracle's per-point sums."""
    import paper_2404_08371_gb300 as hhg
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, level)
    lc = ("sin3",) if coeff == "sin3" else ("const", 1.0)
    op = hhg.Operator(mesh, degree=degree, coeff=lc, bc="dirichlet", quad_degree=QD[degree])
    if stored:
        op.store_element_matrices(dtype)
    N = degree * 2 ** level
    n = mesh.vec_size(degree)
    xp = W.uniform(n, seed=3)
    if dtype == torch.float32:
        xp = xp.astype(np.float32).astype(np.float64)
    y = op.apply(torch.tensor(xp, dtype=dtype, device="cuda")).double().cpu().numpy()
    sample, pts = _sampled_points(N, n, np.random.default_rng(level + 10 * degree))
    ref = OA.sampled_diffusion_rows(v[t[0]], level, degree, lc, QD[degree], "dirichlet", xp, pts)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.abs(y[sample] - ref).max() <= tol * np.abs(y).max(), np.abs(y[sample] - ref).max() / np.abs(y).max()


def test_p2_const_double_float_level8_sampled():
    """The double-float P2 constant-coefficient apply at the bench's size (level 8, 22.6 M points):
    sampled rows against the oracle's per-point sums at the FP64 tolerance."""
    import paper_2404_08371_gb300 as hhg
    v, t = W.reference_tet()
    level, degree = 8, 2
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=2, coeff=("const", 1.0), bc="dirichlet", quad_degree=QD[2])
    op.set_fp64_arith("double_float")
    n = mesh.vec_size(2)
    xp = W.uniform(n, seed=13)
    y = op.apply(torch.tensor(xp, device="cuda")).cpu().numpy()
    sample, pts = _sampled_points(degree * 2 ** level, n, np.random.default_rng(14))
    ref = OA.sampled_diffusion_rows(v[t[0]], level, degree, ("const", 1.0), QD[2], "dirichlet", xp, pts)
    assert np.abs(y[sample] - ref).max() <= 1e-12 * np.abs(y).max(), np.abs(y[sample] - ref).max() / np.abs(y).max()


@pytest.mark.parametrize("arith", ["f32", "double_float"])
def test_p2_const_multi_macro_level7_sampled(arith):
    """The two-plane P2 kernel on the cube of 6 macros at level 7 (256 intervals per edge), one launch
    per macro on the op's streams: sampled rows off the macro faces of every macro against the
    oracle's per-point sums on that macro alone (Neumann, so an interior row sums only its own
    macro's micro-tets and reads only its own copy of the face points)."""
    import paper_2404_08371_gb300 as hhg
    from oracle import mesh as OM
    v, t = W.cube6()
    level, degree = 7, 2
    N = degree * 2 ** level
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=2, coeff=("const", 1.3), bc="neumann", quad_degree=QD[2])
    dtype = torch.float32 if arith == "f32" else torch.float64
    if arith == "double_float":
        op.set_fp64_arith("double_float")
    n = mesh.vec_size(2)
    V = n // len(t)
    xp = W.uniform(n, seed=21)
    if dtype == torch.float32:
        xp = xp.astype(np.float32).astype(np.float64)
    y = op.apply(torch.tensor(xp, dtype=dtype, device="cuda")).double().cpu().numpy()
    pts = OM.lattice_points(N)
    inner = np.nonzero((pts.min(axis=1) >= 1) & (pts.sum(axis=1) <= N - 1))[0]
    rng = np.random.default_rng(22)
    tol = 1e-12 if arith == "double_float" else 1e-5
    for m in range(len(t)):
        sample = rng.choice(inner, 150, replace=False)
        ref = OA.sampled_diffusion_rows(v[t[m]], level, degree, ("const", 1.3), QD[2], "neumann",
                                        xp[m * V:(m + 1) * V], pts[sample])
        got = y[m * V + sample]
        scale = np.abs(y[m * V:(m + 1) * V]).max()
        assert np.abs(got - ref).max() <= tol * scale, (m, np.abs(got - ref).max() / scale)


@pytest.mark.parametrize("case", ["p2_sin3_f64_level8_apply", "p1_sin3_f32_level8_apply", "p1_field_f64_level7_adjoint",
                                  "p2_sin3_f64_level7_diag", "n1_cube6_level6_apply"])
def test_march_bitwise_repeatable(case):
    """On lattices whose marching tiles share faces (64 cubes per edge and more), two calls give
    bit-identical results: the shared points are summed in a fixed order, without atomics."""
    import paper_2404_08371_gb300 as hhg
    if case.startswith("n1"):
        v, t = W.cube6()
        mesh = hhg.Mesh(v, t, 6)
        xyz = mesh.coordinates(1)
        op = hhg.CurlCurl(mesh, ("field_p1", (1.0 + xyz[:, 0] / 3.0).contiguous()),
                          ("field_p1", (1.0 + xyz[:, 2]).contiguous()), bc="dirichlet")
        x = torch.tensor(W.uniform(mesh.vec_size(2), seed=3), device="cuda")
        a, b = op.apply(x), op.apply(x)
    else:
        v, t = W.reference_tet()
        degree = int(case[1])
        level = int(case.split("level")[1][0])
        dtype = torch.float64 if "f64" in case else torch.float32
        mesh = hhg.Mesh(v, t, level)
        n = mesh.vec_size(degree)
        if "field" in case:
            k = torch.exp(torch.tensor(W.fourier_field(mesh.coordinates(degree).cpu().numpy()), device="cuda"))
            op = hhg.Operator(mesh, degree=degree, coeff=("field_p%d" % degree, k.to(dtype)), bc="dirichlet",
                              quad_degree=QD[degree])
        else:
            op = hhg.Operator(mesh, degree=degree, coeff=("sin3",), bc="dirichlet", quad_degree=QD[degree])
        x = torch.tensor(W.uniform(n, seed=1), device="cuda").to(dtype)
        if case.endswith("adjoint"):
            g = torch.tensor(W.uniform(n, seed=2), device="cuda").to(dtype)
            a, b = op.adjoint_coeff(x, g), op.adjoint_coeff(x, g)
        elif case.endswith("diag"):
            a, b = op.diagonal(dtype), op.diagonal(dtype)
        else:
            a, b = op.apply(x), op.apply(x)
    assert torch.isfinite(a).all()
    assert torch.equal(a, b)
