"""Coefficient inversion workload: loss = 1/2 ||A(k) u - f||^2 over interior rows, P1, k = exp(g) with g a
seeded sum of 8 Fourier modes (amplitude 0.5); gradients by the adjoint kernels against central finite
differences (h = 1e-6, 32 seeded directions) and against the oracle's element-wise adjoint."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import assemble as OA, layout as OL, mesh as OM

pytestmark = pytest.mark.gpu


def _setup(level, degree=1, dtype=torch.float64):
    import paper_2404_08371_gb300 as hhg
    from paper_2404_08371_gb300.autograd import apply_ak
    v, t = W.reference_tet()
    mesh = hhg.Mesh(v, t, level)
    N = degree * 2 ** level
    pts = OM.lattice_points(N)
    xyz = OM.physical(v[t[0]], pts, N)
    k = torch.tensor(np.exp(W.fourier_field(xyz, seed=0)), dtype=dtype, device="cuda")
    n = len(pts)
    u = torch.tensor(W.uniform(n, seed=1), dtype=dtype, device="cuda")
    f = torch.tensor(W.uniform(n, seed=2), dtype=dtype, device="cuda")
    interior = torch.tensor((pts.min(axis=1) > 0) & (pts.sum(axis=1) < N), device="cuda")
    op = hhg.Operator(mesh, degree=degree, coeff=("field_p%d" % degree, k), bc="dirichlet",
                      quad_degree=2 if degree == 1 else 4)

    def residual(u_, k_):
        r = apply_ak(op, u_, k_) - f
        return torch.where(interior, r, torch.zeros_like(r))

    def loss(u_, k_):
        r = residual(u_, k_)
        return 0.5 * (r * r).sum()
    loss.residual = residual
    return op, u, k, f, interior, loss, pts


def central_difference(loss, u_p, k_p, u_m, k_m, h):
    """(L(+) - L(-)) / 2h with L = |r|^2 / 2, formed as sum((r+ - r-)(r+ + r-)) / 4h.

    The two losses are large (~1e5) and their difference is O(h), so subtracting the rounded
    losses would lose about eps |L| / h ~ 1e-5 of absolute accuracy; the difference of the
    residuals keeps it.
    """
    rp = loss.residual(u_p, k_p)
    rm = loss.residual(u_m, k_m)
    return ((rp - rm) * (rp + rm)).sum().item() / (4 * h)


@pytest.mark.parametrize("degree,level", [(1, 7), (2, 5)])
def test_gradients_against_finite_differences(degree, level):
    op, u, k, f, interior, loss, pts = _setup(level, degree)
    u.requires_grad_(True)
    k.requires_grad_(True)
    L = loss(u, k)
    L.backward()
    gu, gk = u.grad.detach().clone(), k.grad.detach().clone()
    rng = np.random.default_rng(7)
    h = 1e-6
    with torch.no_grad():
        for trial in range(32):
            d = torch.tensor(rng.standard_normal(len(pts)), device="cuda")
            d /= d.norm()
            fd_k = central_difference(loss, u, k + h * d, u, k - h * d, h)
            an_k = (gk * d).sum().item()
            assert abs(fd_k - an_k) <= 1e-6 * max(1.0, abs(an_k)), (trial, fd_k, an_k)
            if trial < 8:
                fd_u = central_difference(loss, u + h * d, k, u - h * d, k, h)
                an_u = (gu * d).sum().item()
                assert abs(fd_u - an_u) <= 1e-6 * max(1.0, abs(an_u))


def test_gradient_matches_oracle_adjoint_and_linearity():
    level = 4
    op, u, k, f, interior, loss, pts = _setup(level)
    k.requires_grad_(True)
    L = loss(u, k)
    L.backward()
    v, t = W.reference_tet()
    S = OA.Space(OM.MacroMesh(v, t), level, 1)
    ug, kg, fg = (OL.from_packed(S, a.detach().cpu().numpy()) for a in (u, k, f))
    A = OA.diffusion_matrix(S, ("field", S, kg), 2, "dirichlet")
    r = A @ ug - fg
    r[S.boundary] = 0.0
    dk_ref = OA.diffusion_coeff_adjoint(S, S, ug, r, 2, "dirichlet")
    got = OL.from_packed(S, k.grad.cpu().numpy())
    assert np.abs(got - dk_ref).max() <= 1e-12 * np.abs(dk_ref).max()
    # A is linear in k: sum_m k_m dL/dk_m = r^T (A(k) - A(0)) u
    A0 = OA.diffusion_matrix(S, ("field", S, np.zeros(S.ndof)), 2, "dirichlet")
    assert np.isclose(kg @ got, r @ ((A - A0) @ ug), rtol=1e-12)


def test_fp32_gradients_against_fp64_finite_differences():
    level = 6
    op64, u64, k64, f64, interior, loss64, pts = _setup(level, 1, torch.float64)
    op32, u32, k32, f32, _, loss32, _ = _setup(level, 1, torch.float32)
    k32.requires_grad_(True)
    loss32(u32, k32).backward()
    rng = np.random.default_rng(9)
    h = 1e-6
    with torch.no_grad():
        for trial in range(32):
            d = torch.tensor(rng.standard_normal(len(pts)), device="cuda")
            d /= d.norm()
            fd = central_difference(loss64, u64, k64 + h * d, u64, k64 - h * d, h)
            an = (k32.grad.double() * d).sum().item()
            assert abs(fd - an) <= 1e-3 * max(1.0, abs(fd)), (trial, fd, an)
