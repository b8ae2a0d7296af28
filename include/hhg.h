/*
 * hhg.h -- C interface of the GB300 matrix-free finite-element library for
 * hybrid tetrahedral grids (Boehm et al., "Code Generation and Performance
 * Engineering for Matrix-Free Finite Element Methods on Hybrid Tetrahedral
 * Grids").
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Status: every call returns HHG_OK (0) or a negative HHG_E_* code;
 *   hhg_last_error() then gives a message (per calling thread).  A failed
 *   call leaves its outputs unspecified but the handles valid.
 * Handles: hhg_mesh_t and hhg_op_t are opaque, owned by the library, freed
 *   by their *_destroy call.  A mesh must outlive the operators made on it.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Unless stated otherwise a call only enqueues work on that
 *   stream and returns; its device outputs are ready when the stream is.
 * Vectors: device pointers owned by the caller, contiguous, of dtype
 *   HHG_F32 (float) or HHG_F64 (double) as the call's `dtype` says.  The
 *   library never keeps a vector pointer beyond the call (coefficient fields
 *   are the one exception, see hhg_coeff_t).
 *
 * Packed vector layout ("level l, degree p")
 * ------------------------------------------
 * Each macro-tetrahedron (P0,P1,P2,P3) refined l times has n = 2^l intervals
 * per edge (Section 2).  A degree-p vector stores, for macro 0, 1, ..., all
 * lattice points (i,j,k), i,j,k >= 0, i+j+k <= N with N = p*n (P2 nodes are
 * the vertices of the grid refined once more), at position
 *     macro*V(N) + V(N) - V(N-k) + j*(N-k+1) - j*(j-1)/2 + i,
 *     V(s) = (s+1)(s+2)(s+3)/6,
 * i.e. k slowest, i fastest.  Point (i,j,k) sits at P0 + (i/N)(P1-P0) +
 * (j/N)(P2-P0) + (k/N)(P3-P0).  Points on faces, edges and vertices of a
 * macro are stored once per macro containing them; a vector is
 * "consistent" when all copies of a point hold the same value.  Inputs
 * must be consistent and outputs are consistent.  Vector-valued fields
 * (HHG_EPSILON) store 3 components per point, and a batch of nrhs vectors
 * stores the batch index fastest: element ((point*ncomp + c)*nrhs + r).
 *
 * Boundary conditions: HHG_DIRICHLET applies A_D = [[A_II, 0], [0, I]] --
 * rows of interior points use interior columns only and boundary rows return
 * their input; HHG_NEUMANN applies the full matrix.  Boundary points are the
 * points on macro faces that belong to exactly one macro.
 */
#ifndef HHG_H
#define HHG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HHG_OK 0
#define HHG_E_ARG (-1)           /* invalid argument: null pointer, size, enum out of range */
#define HHG_E_DEGENERATE (-2)    /* a macro-tetrahedron has (numerically) zero volume */
#define HHG_E_NONMANIFOLD (-3)   /* a macro face is shared by more than two macros */
#define HHG_E_OOM (-4)           /* host or device allocation failed */
#define HHG_E_CUDA (-5)          /* a CUDA call or a kernel launch failed */
#define HHG_E_NOT_CONVERGED (-6) /* mg_solve reached max_iters above its tolerance */
#define HHG_E_NAN (-7)           /* a NaN or Inf appeared in a residual norm */
#define HHG_E_UNSUPPORTED (-8)   /* valid but not implemented combination */

enum { HHG_F32 = 0, HHG_F64 = 1 };
enum { HHG_DIFFUSION = 0, HHG_EPSILON = 1, HHG_CURLCURL = 2 };
enum { HHG_DIRICHLET = 0, HHG_NEUMANN = 1 };
enum {
  HHG_COEFF_CONST = 0,    /* k(x) = value */
  HHG_COEFF_SIN3 = 1,     /* k(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z), at quadrature points */
  HHG_COEFF_FIELD_P1 = 2, /* k = sum_v k_v phi_v, a P1 field (packed degree-1 vector at the op's level) */
  HHG_COEFF_FIELD_P2 = 3  /* k = sum_m k_m psi_m, a P2 field (packed degree-2 vector at the op's level) */
};

typedef struct hhg_mesh hhg_mesh_t;
typedef struct hhg_op hhg_op_t;

/* Coefficient of an operator.  For FIELD types `field` is a device pointer
 * of dtype `field_dtype` that the operator BORROWS: it is read at every
 * apply, so the caller keeps it alive and may change its values between
 * applies.  Applies must use dtype == field_dtype. */
typedef struct {
  int type;
  double value;
  const void* field;
  int field_dtype;
} hhg_coeff_t;

/* Message of the last failed call on this thread ("" if none). */
const char* hhg_last_error(void);

/* Build the refined hierarchy of a macro mesh (Section 2).
 * macro_vertices: host, nv x 3 doubles (copied).  macro_tets: host, nt x 4
 * vertex indices (copied), either orientation.  level: finest refinement
 * level, 0..10; levels 0..level are all available.
 * Errors: HHG_E_ARG (sizes, indices), HHG_E_DEGENERATE, HHG_E_NONMANIFOLD,
 * HHG_E_OOM, HHG_E_CUDA (device set-up).  The current CUDA device at this
 * call is the mesh's device. */
int hhg_mesh_create(const double* macro_vertices, int64_t nv, const int32_t* macro_tets, int64_t nt,
                    int level, hhg_mesh_t** out);
int hhg_mesh_destroy(hhg_mesh_t* mesh);

/* Number of packed entries of a degree-p scalar vector at `level`
 * (nmacro * V(p * 2^level)); multiply by ncomp * nrhs for batched or vector fields. */
int hhg_vec_size(const hhg_mesh_t* mesh, int level, int degree, int64_t* n);

/* Number of distinct points (DoFs) of a degree-p scalar space at `level`,
 * and how many of them are not Dirichlet boundary points. */
int hhg_dof_count(const hhg_mesh_t* mesh, int level, int degree, int64_t* total, int64_t* interior);

/* Create a matrix-free operator (Eq. 4.1) at `level` (-1 = finest).
 * kind HHG_DIFFUSION: a(u,v) = int k grad u . grad v, degree 1 or 2
 *   (Eq. P1, Eq. P2V).  kind HHG_EPSILON: a(u,v) = int 2 mu eps(u):eps(v),
 *   eps(u) = (grad u + grad u^T)/2, degree 2, vector valued.
 * quad_degree: degree of the quadrature rule for variable coefficients
 *   (1: centroid, 2: 4-point, 4: 14-point rule exact to degree 5); for
 *   constant coefficients the local matrices are exact whatever its value.
 * Errors: HHG_E_ARG, HHG_E_UNSUPPORTED, HHG_E_OOM, HHG_E_CUDA. */
int hhg_op_create(hhg_mesh_t* mesh, int level, int kind, int degree, const hhg_coeff_t* coeff, int bc,
                  int quad_degree, hhg_op_t** out);
int hhg_op_destroy(hhg_op_t* op);

/* Create the lowest-order Nedelec (first kind) operator
 *     a(u, v) = int alpha curl u . curl v + beta u . v        (Eq. N1)
 * at `level` (-1 = finest).  alpha, beta: HHG_COEFF_CONST or HHG_COEFF_FIELD_P1
 * (a P1 packed vector at the op's level, borrowed as for hhg_coeff_t).  The
 * DoFs are the micro-edges, stored in the degree-2 packed layout: the entry of
 * the edge midpoint holds the tangential integral of u along the macro's
 * canonical index direction of that edge -- (1,0,0), (0,1,0), (0,0,1),
 * (1,-1,0), (1,0,-1), (0,1,-1) or (1,-1,1) for midpoints whose doubled
 * coordinates have the odd entries (i), (j), (k), (i,j), (i,k), (j,k), (i,j,k)
 * -- and vertex entries are zero.  A point shared by macros holds the value
 * of its own macro's orientation (copies may differ in sign).  DIRICHLET
 * fixes the tangential trace: edges on boundary faces return their input.
 * Apply with hhg_op_apply (nrhs = 1).  Errors: HHG_E_ARG, HHG_E_UNSUPPORTED,
 * HHG_E_OOM, HHG_E_CUDA. */
int hhg_op_create_curlcurl(hhg_mesh_t* mesh, int level, const hhg_coeff_t* alpha, const hhg_coeff_t* beta, int bc,
                           hhg_op_t** out);

/* Arithmetic of FP64 applies (no counterpart in the paper, whose FP64 runs
 * on CPU FMA units).  HHG_FP64_NATIVE (the default): FP64 operations.
 * HHG_FP64_DOUBLE_FLOAT: FP64 vectors in and out, the arithmetic in pairs
 * of FP32 numbers (hi + lo, 48 significant bits: relative errors of a few
 * 1e-15 per operation, within the 1e-12 tolerance of FP64 applies), for
 * GPUs whose FP64 rate is a small fraction of their FP32 rate (GB300:
 * 1/64).  Available for P1 and P2 constant-coefficient DIFFUSION operators
 * (P2: lattices of more than 32 intervals per edge; smaller ones keep FP64
 * operations); it allocates a device vector of 8 bytes per point for the
 * split input (freed when the mode returns to native or with the operator).
 * The operator's other calls (diagonal, multigrid) use its applies as set;
 * a multigrid hierarchy built while the mode is set (the first
 * hhg_mg_solve) gives its coarse operators the same mode.
 * Errors: HHG_E_UNSUPPORTED (other operators), HHG_E_OOM, HHG_E_ARG. */
enum { HHG_FP64_NATIVE = 0, HHG_FP64_DOUBLE_FLOAT = 1 };
int hhg_op_set_fp64_arith(hhg_op_t* op, int mode);

/* Replace the borrowed coefficient field pointer of a FIELD operator. */
int hhg_op_set_field(hhg_op_t* op, const void* field, int field_dtype);

/* y = A x (Eq. 4.1, Algorithm 1 summed over all micro-tets).  x, y: packed
 * vectors of the op's space (ncomp = 3 for EPSILON), nrhs right-hand sides
 * (nrhs >= 1; > 1 only for EPSILON, at most 256, else HHG_E_UNSUPPORTED).
 * y is overwritten; x and y must not overlap.  The apply computes every
 * local matrix on the fly.  Results repeat bit for bit from call to call:
 * on lattices of 64 or more cubes per edge the points on the faces between
 * GPU tiles collect their partial sums (at most four) in a fixed order,
 * through a scratch array allocated with the operator. */
int hhg_op_apply(hhg_op_t* op, const void* x, void* y, int dtype, int nrhs, void* stream);

/* Adjoint in the coefficient of a FIELD operator (A is linear in k):
 * dk_m = g^T (dA/dk_m) u, summed over the nrhs pairs (u_r, g_r).  Under
 * HHG_DIRICHLET only interior rows and columns of A depend on k, so the
 * boundary entries of u and g do not contribute.  dk: packed vector of the
 * coefficient space, overwritten.  The gradient of L(u) with respect to u
 * is A^T g = A g (A symmetric) -- use hhg_op_apply.
 * Errors: HHG_E_UNSUPPORTED for non-FIELD coefficients. */
int hhg_op_apply_adjoint_coeff(hhg_op_t* op, const void* u, const void* g, void* dk, int dtype, int nrhs,
                               void* stream);

/* d = diag(A) (Dirichlet rows: 1), packed, overwritten.  Scalar DIFFUSION
 * operators and CURLCURL operators (Eq. N1; the diagonal of an edge does not
 * depend on its orientation; vertex points of the doubled lattice, which
 * carry no DoF, get 0). */
int hhg_op_diagonal(hhg_op_t* op, void* d, int dtype, void* stream);

/* Precomputed variant of Eq. 4.1 for a variable-coefficient DIFFUSION op
 * (HHG_COEFF_SIN3 or a FIELD of the op's degree) or a CURLCURL op (Eq. N1):
 * the local matrices A_T of all micro-tets are integrated once with the op's
 * rule and kept in device memory owned by the op (P2: the 55 entries of the
 * symmetric 10 x 10 matrix, P1: the element mean of k, A_T = mean(k) A0, N1:
 * the 21 entries of the symmetric 6 x 6 matrix); later hhg_op_apply calls in
 * `dtype` read them instead of integrating (the paper's precomputed element
 * matrices, Section 6.6).  Memory: 6 V(2^level - 1) (55 for P2, 1 for P1, 21
 * for N1) entries per macro of `dtype`; coefficient fields must have `dtype`.  Applies in the other dtype, the diagonal and
 * the adjoint keep the matrix-free path.  hhg_op_set_field drops the stored
 * matrices.  Errors: HHG_E_UNSUPPORTED (other kinds or coefficients),
 * HHG_E_ARG, HHG_E_OOM, HHG_E_CUDA. */
int hhg_op_store_element_matrices(hhg_op_t* op, int dtype, void* stream);

/* Drops the matrices of hhg_op_store_element_matrices (no-op if none). */
int hhg_op_drop_element_matrices(hhg_op_t* op);

/* Physical coordinates of every packed point of a degree-p space at `level`:
 * xyz (device, FP64) receives 3 values per point, (x, y, z), in the packed
 * order (nmacro * V(p * 2^level) points), overwritten.  Use it to sample
 * coefficient fields or initial data. */
int hhg_vec_coordinates(const hhg_mesh_t* mesh, int level, int degree, double* xyz, void* stream);

/* Make a packed vector consistent: every copy of a shared point takes the
 * value of its copy in the lowest-numbered macro.  n_per_point = ncomp*nrhs. */
int hhg_vec_make_consistent(const hhg_mesh_t* mesh, int level, int degree, void* x, int dtype,
                            int n_per_point, void* stream);

/* Inner product over distinct points (each shared point counted once) of
 * two consistent packed vectors; synchronous, result on the host. */
int hhg_vec_dot(const hhg_mesh_t* mesh, int level, int degree, const void* x, const void* y, int dtype,
                int n_per_point, double* result, void* stream);

/* Grid transfers between level l-1 and level l (Section 8; the spaces are
 * nested).  Prolongation xf = P xc evaluates the coarse FE function at the
 * fine points.  Restriction rc = P^T rf sums over distinct fine points and
 * leaves the coarse Dirichlet boundary entries zero.  Both overwrite their
 * output. */
int hhg_prolongate(const hhg_mesh_t* mesh, int level_fine, int degree, const void* xc, void* xf, int dtype,
                   void* stream);
int hhg_restrict(const hhg_mesh_t* mesh, int level_fine, int degree, const void* rf, void* rc, int dtype,
                 void* stream);

/* Grid transfers of Nedelec edge vectors (Eq. N1 space, Section 8's
 * multigrid for the curl-curl problem).  xf = P xc: the tangential integral
 * along every fine edge of the coarse Whitney field (the spaces are nested);
 * rc = P^T rf over distinct fine edges, coarse Dirichlet (tangential
 * boundary) entries zero.  Vectors in the packed Nedelec layout of
 * hhg_op_create_curlcurl (doubled lattice, each copy in its macro's
 * orientation, vertex points zero); both outputs consistent, overwritten. */
int hhg_prolongate_edges(const hhg_mesh_t* mesh, int level_fine, const void* xc, void* xf, int dtype, void* stream);
int hhg_restrict_edges(const hhg_mesh_t* mesh, int level_fine, const void* rf, void* rc, int dtype, void* stream);

/* Discrete gradient of the Nedelec space (the nodal part of Hiptmair's
 * hybrid smoother, Section 8).  hhg_gradient: e = G p, the tangential
 * integral of grad p along every edge of level `level`, p a consistent P1
 * packed vector of that level, e a packed Nedelec vector (vertex points 0).
 * hhg_gradient_transpose: p = G^T e over distinct edges, Dirichlet vertices
 * zero, consistent.  Outputs overwritten; errors HHG_E_ARG, HHG_E_CUDA. */
int hhg_gradient(const hhg_mesh_t* mesh, int level, const void* p, void* e, int dtype, void* stream);
int hhg_gradient_transpose(const hhg_mesh_t* mesh, int level, const void* e, void* p, int dtype, void* stream);

/* Load vector b_i = int f phi_i for f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
 * (the manufactured Poisson right-hand side), by the 14-point rule per
 * micro-tet; Dirichlet entries zero.  FP64 output, packed, overwritten. */
int hhg_rhs_sin3_poisson(const hhg_mesh_t* mesh, int level, int degree, double* b, void* stream);

/* || u_h - u ||_L2 for u = sin(pi x) sin(pi y) sin(pi z), 14-point rule
 * per micro-tet; synchronous. */
int hhg_l2_error_sin3(const hhg_mesh_t* mesh, int level, int degree, const double* uh, double* err,
                      void* stream);

/* One Chebyshev smoothing step of order `order` on D^{-1} A over
 * [lo*lam, hi*lam] (Section 8): x <- x + p(D^{-1}A) D^{-1}(b - A x).
 * dinv: packed inverse diagonal.  x updated in place. */
int hhg_cheb_smooth(hhg_op_t* op, const void* b, void* x, const void* dinv, double lam, double lo, double hi,
                    int order, int dtype, void* stream);

/* The smoothing step of hhg_cheb_smooth, for callers that must not allocate
 * device memory while they run.  (The paper has no counterpart: this is an
 * interface variant, not part of the method.)  hhg_cheb_smooth allocates two
 * work vectors on its first call for an operator; processes that hand all
 * device memory to their own allocator, or loops that cannot afford the
 * device synchronisation of cudaMalloc, can call this entry point instead.
 * It calls no cudaMalloc / cudaFree: its two work vectors live in one fixed
 * 8 MiB array in the library's device image (2 x 524288 entries), held by
 * every GPU that loads the library until the process exits.
 * Limits and rules:
 *  - the operator's vectors may have at most 524288 entries
 *    (hhg_vec_size); larger operators get HHG_E_ARG;
 *  - the array's device address is looked up (cudaGetSymbolAddress, which
 *    can load the library's device image) when an operator is created on
 *    the device, so the call itself triggers no module loading; create the
 *    operator before any stream capture begins;
 *  - all calls share the one array, which keeps the last call's contents
 *    (nothing in it needs to start at zero); calls that overlap on the GPU,
 *    e.g. on two streams at once, race with each other;
 *  - the operator must have been created beforehand (hhg_op_create allocates).
 * Arguments, results and errors are otherwise those of hhg_cheb_smooth. */
int hhg_cheb_smooth_noalloc(hhg_op_t* op, const void* b, void* x, const void* dinv, double lam, double lo,
                            double hi, int order, int dtype, void* stream);

/* Power iteration for the largest eigenvalue of D^{-1} A from start vector
 * v (consistent, overwritten by the last iterate): iters steps of
 * v <- D^{-1} A v / ||D^{-1} A v||; returns the last norm.  Synchronous. */
int hhg_power_iteration(hhg_op_t* op, const void* dinv, void* v, int iters, int dtype, double* lam,
                        void* stream);

typedef struct {
  int nu1, nu2;          /* pre / post smoothing steps per V-cycle (each a Chebyshev step) */
  int cheb_order;        /* Chebyshev polynomial order (applications of A per step) */
  int power_iters;       /* power-iteration steps for lambda_max of D^{-1}A per level */
  double cheb_lo, cheb_hi; /* smoothing interval [lo*lam, hi*lam] */
  double tol;            /* stop when ||b - A x||_2 / ||b||_2 <= tol */
  int max_iters;         /* maximum number of outer iterations after FMG */
  int mixed;             /* 0: all FP64; 1: FP32 cycles inside FP64 iterative refinement */
  int fmg;               /* 1: start from full multigrid; 0: start from the given x */
  int coarse_level;      /* level solved exactly (dense Cholesky in FP64) */
} hhg_mg_opts_t;

typedef struct {
  int iterations;        /* outer iterations after FMG */
  double rel_residual;   /* final ||b - A x||_2 / ||b||_2 (FP64) */
  double residual_history[64]; /* relative residual after FMG and after each outer iteration */
  double setup_ms;       /* hierarchy set-up time (first call on an op only) */
  double solve_ms;       /* FMG + iterations, device time */
} hhg_mg_stats_t;

/* Fill `opts` with the defaults: V(2,2), order 2, 15 power iterations,
 * [0.1, 1.1], tol 1e-10, 50 iterations, FP64, FMG on, coarse level 0. */
int hhg_mg_default_opts(hhg_mg_opts_t* opts);

/* Solve A x = b with geometric multigrid (Section 8): FMG, then outer
 * iterations x <- x + V(b - A x) until the relative residual reaches tol.
 * op: a scalar DIFFUSION operator with DIRICHLET boundary and a CONST or
 * SIN3 coefficient; the hierarchy (coarser operators, inverse diagonals,
 * eigenvalue estimates, coarse factor) is built on the first call and kept
 * with op.  b, x: FP64 packed vectors; x is the initial guess when fmg = 0
 * and is overwritten with the solution.  In mixed mode smoothing,
 * restriction and prolongation run in FP32; the outer residual, the update
 * of x and the coarse solve are FP64.  Synchronous.
 * Errors: HHG_E_NOT_CONVERGED (x holds the last iterate), HHG_E_NAN,
 * HHG_E_UNSUPPORTED, HHG_E_ARG, HHG_E_CUDA. */
int hhg_mg_solve(hhg_op_t* op, const double* b, double* x, const hhg_mg_opts_t* opts, hhg_mg_stats_t* stats,
                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HHG_H */
