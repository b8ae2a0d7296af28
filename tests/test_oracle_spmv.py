"""The oracle's OpenMP CSR apply equals scipy's product bit for bit, for any thread count."""
import numpy as np

import workloads as W
from oracle import assemble as A, mesh as M, spmv


def test_openmp_spmv_equals_scipy():
    S = A.Space(M.MacroMesh(*W.cube6()), 2, 2)
    K = A.diffusion_matrix(S, ("sin3",), 4, "dirichlet")
    x = W.uniform(S.ndof, seed=5)
    ref = K @ x
    op = spmv.CsrSpmv(K)
    for threads in (1, 3, spmv.max_threads()):
        assert np.array_equal(op(x, threads), ref)
