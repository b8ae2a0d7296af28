"""The allocation-free Chebyshev smoother (hhg_cheb_smooth_noalloc) through the C interface.

Callers that must not allocate device memory while they run (a process whose device memory is
handed to another allocator, a loop that cannot afford cudaMalloc's synchronisation) use this
entry point instead of hhg_cheb_smooth; it takes its work vectors from a fixed array in the
library.  Its results must equal those of hhg_cheb_smooth, call after call, within the tolerance
of the other GPU tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _setup(meshname, level, degree, coeff, dtype):
    import paper_2404_08371_gb300 as hhg
    v, t = getattr(W, meshname)()
    mesh = hhg.Mesh(v, t, level)
    op = hhg.Operator(mesh, degree=degree, coeff=coeff, bc="dirichlet", quad_degree=2 if degree == 1 else 4)
    n = mesh.vec_size(degree)
    dinv = 1.0 / op.diagonal(dtype)
    b = mesh.make_consistent(torch.tensor(W.uniform(n, seed=11), dtype=dtype, device="cuda"), degree)
    x = mesh.make_consistent(torch.tensor(W.uniform(n, seed=12), dtype=dtype, device="cuda"), degree)
    return mesh, op, b, x, dinv


def _call(fn, op, b, x, dinv, lam, dtype):
    from paper_2404_08371_gb300 import dtype_code
    return fn(op.handle, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
              ctypes.c_void_p(dinv.data_ptr()), lam, 0.1, 1.1, 2, dtype_code(x),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_smoother_matches_allocating_one(dtype):
    from paper_2404_08371_gb300 import lib
    cases = [("cube6", 3, 2, ("sin3",)), ("reference_tet", 5, 1, ("const", 1.0))]
    setups = [_setup(*c, dtype) for c in cases]
    # two calls in a row on each operator, alternating operators so the shared array is reused
    for call in range(2):
        for mesh, op, b, x, dinv in setups:
            if call == 0:
                op._x_ref = x.clone()
                op._x_new = x.clone()
            assert _call(lib.hhg_cheb_smooth, op, b, op._x_ref, dinv, 1.8, dtype) == 0
            assert _call(lib.hhg_cheb_smooth_noalloc, op, b, op._x_new, dinv, 1.8, dtype) == 0, \
                lib.hhg_last_error()
            torch.cuda.synchronize()
            ref = op._x_ref.double().cpu().numpy()
            got = op._x_new.double().cpu().numpy()
            assert np.abs(got - ref).max() <= TOL[dtype] * np.abs(ref).max()


def test_noalloc_smoother_rejects_oversized_operator():
    from paper_2404_08371_gb300 import lib, _lib
    mesh, op, b, x, dinv = _setup("reference_tet", 8, 1, ("const", 1.0), torch.float64)
    assert mesh.vec_size(1) > 524288
    assert _call(lib.hhg_cheb_smooth_noalloc, op, b, x, dinv, 1.8, torch.float64) == _lib.HHG_E_ARG
    assert b"fixed scratch" in lib.hhg_last_error()
