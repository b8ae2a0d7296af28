"""FP64 CPU oracle for the matrix-free operator apply on hybrid tetrahedral grids.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline leg and ``--impl reference``) may import this
package.  It shares no code with the CUDA path and the CUDA path never calls it.

What it computes is the plain definition of the discrete operator
(Section 4, Eq. 4.1): every micro-tetrahedron of every uniformly refined
macro-tetrahedron is enumerated in the sawtooth order of Algorithm 2, its local
matrix is formed by quadrature directly from its physical vertex coordinates
(Algorithm 1, no per-class hoisting), and the local matrices are summed into a
global sparse matrix keyed by exact integer DoF keys.  The apply is then a
sparse matrix-vector product.  Multigrid pieces (prolongation by evaluation of
the coarse function, restriction as its transpose, Chebyshev smoothing, V-cycle,
FMG, iterative refinement; Section 8) are written on top of those matrices.

Modules:
  mesh        macro mesh, refinement lattice, six micro-tet classes, DoF keys
  quadrature  quadrature rules on the reference tetrahedron
  fe          P1 / P2 bases and local matrices (diffusion, epsilon)
  assemble    global matrices, Dirichlet handling, diagonal, coefficient adjoint
  mg          transfers, Chebyshev smoother, V-cycle, FMG, iterative refinement
  layout      the packed per-macro vector layout of the library (for tests)

Parity status of each function is stated in its docstring ("pinned by" lists
the independent checks in tests/test_oracle_*.py).
"""
