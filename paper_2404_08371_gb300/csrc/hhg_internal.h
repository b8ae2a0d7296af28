// Internal declarations of the hhg library (not part of the public C interface).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <vector>

#include "hhg.h"

namespace hhg {

int fail(int code, const char* fmt, ...);
void clear_error();

#define HHG_CUDA_TRY(call)                                                                       \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return ::hhg::fail(HHG_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define HHG_TRY(call)          \
  do {                         \
    int s_ = (call);           \
    if (s_ != HHG_OK) return s_; \
  } while (0)

// Number of lattice points with i+j+k <= s.
__host__ __device__ inline int64_t lattice_size(int64_t s) { return (s + 1) * (s + 2) * (s + 3) / 6; }

// Index-space vertex offsets of the six micro-tet classes in the cube at origin c
// (white up, four octahedron tets split along (0,1,0)-(1,0,1), white down; Section 2, Fig. 3).
extern const int kClassOffsets[6][4][3];
// B(o, m) = m - kClassShrink[o] (Section 5.1).
extern const int kClassShrink[6];
// P2 local node order: 4 vertices then edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).
extern const int kP2Edges[6][2];

// Geometry and boundary description of one macro-tetrahedron.
struct MacroGeom {
  double p0[3];
  double e[3][3];        // e[a] = P_{a+1} - P_0
  int32_t vid[4];
  uint32_t bnd_table;    // bit z set: a point whose zero-weight set is z lies on the domain boundary
  uint32_t own_table;    // bit z set: this macro is the lowest-numbered macro holding such a point
};

// Interface groups of one (level, degree): the copies of every point shared by several macros.
struct TileTasks {
  int4* d = nullptr;
  int64_t n = 0;
  int kchunk = 32;
};

// Task list of the epsilon kernels for one number of cubes per CTA: tasks of colour c at
// d[off[c] .. off[c+1]); the host copy stays alive while the asynchronous upload may read it.
struct EpsTasks {
  int4* d = nullptr;
  int64_t off[9] = {0};
  std::vector<int4> host;
  ~EpsTasks() { cudaFree(d); }
};

struct Interface {
  int64_t ngroups = 0;
  int64_t nmembers = 0;
  int64_t* d_ptr = nullptr;    // ngroups + 1 offsets into d_idx
  int64_t* d_idx = nullptr;    // scalar packed positions, sorted (the first is the owner copy)
  uint8_t* d_bnd = nullptr;    // 1 if the point is a Dirichlet boundary point
  int64_t ndof_total = 0;
  int64_t ndof_interior = 0;
  std::vector<int64_t> h_ptr, h_idx;   // host copies of the groups (set-up code)
  std::vector<uint8_t> h_bnd;
  // degree-2 data: orientation of each copy of an edge point relative to the group's first copy
  // (+1 / -1; +1 for vertex points), used by the Nedelec operator
  int8_t* d_sign = nullptr;
  // launch tables of the gather kernels: CTAs of 256 points never cross a plane
  int64_t ncta = 0;
  int* d_cta_plane = nullptr;   // plane of each CTA
  int* d_cta_start = nullptr;   // first CTA of each plane (N + 2 entries)
  int* d_pstart = nullptr;      // first packed position of each plane (N + 2 entries)
  // task list of the marching kernels: (i-tile, j-tile, k-chunk, macro), heaviest first
  int4* d_march_tasks = nullptr;
  int64_t n_march_tasks = 0;
  int march_kchunk = 32;
  // task lists of the plane-tile kernels: (i-chunk, row group, k-chunk, macro), heaviest first;
  // tile[0]: chunks of 128 points along i on one macro (launched once per macro), tile[1]: chunks
  // of 64 on all macros (one launch), tile[2]: chunks of 64 on one macro
  TileTasks tile[3];
  ~Interface();
};

// Tile shape of the marching kernels (march.cu): 32 lanes along i, kMarchWarps warps along j,
// march_kchunk cube layers along k.  Below kMarchJAtomicN cubes per edge the tiles overlap their
// neighbours below by one cube in i and j (31 x (kMarchWarps - 1) owned) and every point is stored
// once; from kMarchJAtomicN on all 32 x kMarchWarps columns of cubes are the tile's own (no cube is
// integrated twice along i or j) and the points on the tile's i- and j-faces get partial sums from
// two or four tiles, added in a fixed order by march_finish_kernel (march_kernel.cuh).
constexpr int kMarchWarps = 8;
constexpr int kMarchJAtomicN = 64;
__host__ __device__ constexpr int march_iw(int n) { return n >= kMarchJAtomicN ? 32 : 31; }
__host__ __device__ constexpr int march_jw(int n) { return n >= kMarchJAtomicN ? kMarchWarps : kMarchWarps - 1; }
// Rows j of the plane-tile tasks (ops.cu): one per warp of an 8-warp CTA.
constexpr int kStencilWarps = 8;

// Quadrature rule on the reference tetrahedron (volume 1/6).
struct QuadRule {
  std::vector<double> xi;   // nq x 3
  std::vector<double> w;    // nq
  int nq() const { return (int)w.size(); }
};
int quad_rule(int degree, QuadRule* out);

}  // namespace hhg

struct hhg_mesh {
  int level = 0;            // finest level
  int device = 0;
  std::vector<double> vertices;
  std::vector<int32_t> tets;
  std::vector<hhg::MacroGeom> macros;
  hhg::MacroGeom* d_macros = nullptr;
  std::map<int, std::unique_ptr<hhg::Interface>> iface;   // key: level * 8 + degree
  void* d_scratch = nullptr;   // reduction scratch, grown on demand (set-up time, not in applies)
  size_t scratch_bytes = 0;
  int nmacro() const { return (int)macros.size(); }
  int interface(int level, int degree, const hhg::Interface** out);
  int build_tile_tasks(int64_t N, int64_t iw, int64_t jw, int copies, int64_t min_tasks, hhg::TileTasks* out) const;
  int scratch_reserve(size_t bytes);
  ~hhg_mesh();
};

namespace hhg {

constexpr int kMaxQ = 14;
struct MGHierarchy;
struct OpWork;
void destroy_mg(MGHierarchy* h);
void destroy_work(OpWork* w);

// Per-macro constants of an operator, in the compute type T (one block per macro, in device memory).
template <typename T>
struct alignas(16) OpConst {
  int64_t base;          // offset of the macro in a packed scalar vector
  int64_t kbase;         // offset of the macro in the packed coefficient vector
  uint32_t bnd_table;
  int N;                 // lattice resolution of the space (degree * 2^level)
  int n;                 // cubes per edge (2^level)
  T A[6][10][10];        // hoisted constant-coefficient local matrices per class (P1 uses [4][4])
  T S[15];               // P1 interior 15-point stencil (offset order kStencil)
  T Sface[4][15];        // P1 stencil of a point inside macro face a (the face with weight a = 0)
  T M[6][6];             // per class |det J| J^{-1} J^{-T} (xx, yy, zz, xy, xz, yz)
  T adet[6];             // per class |det J| of the micro-tet map
  T Jinv[6][9];          // per class J^{-1}, row-major
  uint32_t own_table;    // see MacroGeom
  double x0[3];          // physical position of lattice point (0,0,0)
  double h[3][3];        // h[a] = e[a] / n: physical step of one cube along index axis a
  // quadrature (variable coefficients): nq points, weights, barycentric coordinates,
  // P2 basis values psi_m(xi_q), and for the analytic coefficient the cosine / sine of
  // 2 pi delta, delta = H (off_o[0] + D_o xi_q): the offset of point q of class o from the cube origin.
  int nq;
  T w[kMaxQ];
  T lam[kMaxQ][4];
  T lam4[kMaxQ][4];      // 4 lambda_a and 4 lambda_a - 1 at the points (P2 gradients)
  T lam4m1[kMaxQ][4];
  T psi[kMaxQ][10];
  T cs[6][kMaxQ][3][2];
  T qoff[6][kMaxQ][3];   // physical offset delta of point q of class o from the cube origin
  T rot[3][2];           // cos / sin of 2 pi H[2][d]: rotation of (sin, cos)(2 pi x_d) per k step
  T X0[3];               // x0 and H in the compute type
  T H[3][3];             // H[a][d]: component d of the step along index axis a
};

extern const int kStencil[15][3];

// Launchers (ops.cu).
template <typename T>
int launch_apply(const struct ::hhg_op* op, const T* x, T* y, cudaStream_t s);
template <typename T>
int launch_interface_sum(const Interface* itf, T* y, int per_point, bool dirichlet, cudaStream_t s);
template <typename T>
int launch_make_consistent(const Interface* itf, T* x, int per_point, cudaStream_t s);
// Element-centric kernels (march.cu); mode 0 apply, 1 diagonal, 2 coefficient adjoint,
// 3 load vector of f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z).
// Scratch of the marching kernels' shared tile faces for an operator on lattices of at least
// kMarchJAtomicN cubes per edge (march.cu); allocated at operator creation.
int alloc_face_scratch(struct ::hhg_op* op);
// Device address of the allocation-free smoother's scratch array on the current device (mg.cu),
// looked up at operator creation.
int noalloc_prepare();
// Precomputed variant (march.cu): local matrices of all micro-tets into elem, and applies from them.
template <typename T>
int launch_elem_store(const struct ::hhg_op* op, T* elem, cudaStream_t s);
template <typename T>
int launch_march_stored(const struct ::hhg_op* op, const T* x, T* y, cudaStream_t s);
template <typename T>
int launch_elem_store_n1(const struct ::hhg_op* op, T* elem, cudaStream_t s);
template <typename T>
int launch_march(const struct ::hhg_op* op, const OpConst<T>* cst, int mode, const T* x, const T* g, const T* kf,
                 T* out, cudaStream_t s);
// Nedelec curl-curl + mass apply (march.cu, R = 2 traversal of the doubled lattice).
template <typename T>
int launch_n1(const struct ::hhg_op* op, const T* x, T* y, cudaStream_t s);
template <typename T>
int launch_n1_diag(const struct ::hhg_op* op, T* d, cudaStream_t s);
// Interface sum with orientation signs (edge points of the doubled lattice).
template <typename T>
int launch_interface_sum_signed(const Interface* itf, T* y, bool dirichlet, cudaStream_t s);
// Nedelec vectors: every copy of a shared edge set from the owner copy with its orientation sign.
template <typename T>
int launch_make_consistent_signed(const Interface* itf, T* x, cudaStream_t s);
// P2 vector epsilon operator (eps.cu): mode 0 apply to nrhs right-hand sides, 2 adjoint in mu.
template <typename T>
int launch_eps(const struct ::hhg_op* op, const OpConst<T>* cst, int mode, int nrhs, const T* x, const T* g,
               const T* mu, T* out, cudaStream_t s);
// Squared L2 error of u_h against sin(pi x) sin(pi y) sin(pi z): per-CTA partial sums.
int64_t launch_l2_blocks(const struct ::hhg_op* op);
int launch_l2_error(const struct ::hhg_op* op, const double* uh, double* partial, cudaStream_t s);

}  // namespace hhg

namespace hhg {
// P2 constant-coefficient stencils: the row of a point of the doubled lattice is fixed by the
// parity (I & 1, J & 1, K & 1) of its coordinates and by the macro faces it lies on (zero mask z).
// The 8 parities have 65, 27, 19, 27, 27, 19, 27, 19 structural neighbours (230 in all); entry d of
// parity p (start[p] <= d < start[p + 1]) is the offset off[d] (packed (dx+2) | (dy+2) << 4 |
// (dz+2) << 8) with weight w[z][d] (zero for neighbours outside the macro).
constexpr int kP2StTotal = 230;
struct P2StencilIndex {
  int start[9];
  int off[kP2StTotal];
};
template <typename T>
struct alignas(16) P2Stencil {
  T w[16][kP2StTotal];
};
// The weights of the rows off the macro faces (mask 0) of one macro, passed by value to the
// two-plane kernel so that its FMAs read them from the kernel's parameter bank: in FP32, and as FP32
// pairs (hi, lo) for double-float arithmetic.
struct P2ParamW {
  float w[kP2StTotal];
};
struct P2ParamWDF {
  float2 w[kP2StTotal];
};

// Hoisted per-class data of the Nedelec operator (one block per macro), in the macro's canonical
// edge orientation (the local orientation a -> b times s_e = +-1, folded into the entries) and
// stored as the upper triangle e <= f (index n1_sym(e, f)):
//   C[o][.] = s_e s_f |T| curl phi_e . curl phi_f   (curl phi_e = 2 grad l_a x grad l_b, constant)
//   M[o][v][.] = s_e s_f int_T lambda_v phi_e . phi_f  (exact)
constexpr int kN1Sym = 21;
__host__ __device__ constexpr int n1_sym(int e, int f) { return e * 6 - e * (e - 1) / 2 + (f - e); }
template <typename T>
struct alignas(16) N1Const {
  T C[6][kN1Sym];
  T M[6][4][kN1Sym];
  int64_t vbase;     // offset of the macro in a packed P1 vector (coefficient fields)
};
}  // namespace hhg

struct hhg_op {
  hhg_mesh* mesh = nullptr;
  int level = 0, kind = 0, degree = 1, bc = 0, quad_degree = 2;
  hhg_coeff_t coeff{};
  hhg_coeff_t coeff2{};      // second coefficient (beta of the Nedelec operator)
  void* d_p2st64 = nullptr;  // P2Stencil<double>[nmacro] (P2 constant-coefficient diffusion)
  void* d_p2st32 = nullptr;
  void* d_p2idx = nullptr;   // P2StencilIndex (structural neighbour lists)
  std::vector<hhg::P2ParamW> h_p2w32;   // per macro: FP32 weights of the rows off the faces
  std::vector<hhg::P2ParamWDF> h_p2wdf; // the same as FP32 pairs (double-float FP64 applies, if set)
  // several macros: their per-macro launches run on these streams side by side, forked from and
  // joined back into the caller's stream by the events (created with the op; no apply allocates)
  std::vector<cudaStream_t> aux_streams;
  std::vector<cudaEvent_t> aux_events;   // [0]: fork, [1 + i]: join of stream i
  // stored local matrices (hhg_op_store_element_matrices): [macro][class][entry][cube], cube =
  // packed index of its origin in the lattice of resolution 2^level - 1; entries 55 (P2) or 1 (P1)
  void* d_elem = nullptr;
  int elem_dtype = -1;
  // epsilon operator: per colour, the CTAs of live cubes (ci/2 start, cj/2, ck/2, macro), built on
  // the first use of each number of cubes per CTA (256 / nrhs) and kept
  mutable std::map<int, std::unique_ptr<hhg::EpsTasks>> eps_tasks;
  void* d_n1_64 = nullptr;   // N1Const<double>[nmacro]
  void* d_n1_32 = nullptr;
  int N = 0, n = 0;
  int64_t npts = 0;          // packed scalar entries of the space
  void* d_const64 = nullptr; // OpConst<double>[nmacro]
  void* d_const32 = nullptr; // OpConst<float>[nmacro]
  hhg::QuadRule rule;
  std::vector<hhg::OpConst<double>> h_const;
  const hhg::Interface* itf = nullptr;   // per-level data of the op's space (owned by the mesh)
  // FP64 vectors in double-float arithmetic (ops.cu): the P1 stencil weights as FP32 pairs
  // (float2[16] per macro) and the split input vector of P1 or P2 applies (float2[npts])
  void* d_p1df = nullptr;
  void* d_dfx = nullptr;
  // partial sums of the points shared by marching tiles (lattices of at least kMarchJAtomicN cubes
  // per edge; march_kernel.cuh, FaceScratch): FP64-sized, per macro face_S slots
  void* d_face = nullptr;
  int64_t face_S = 0, face_Si = 0, face_Sj = 0;
  int face_Ti = 0, face_Tj = 0;
  hhg::MGHierarchy* mg = nullptr;         // multigrid hierarchy, built by the first mg_solve
  hhg::OpWork* work = nullptr;            // work vectors of the standalone smoother calls
  ~hhg_op();
};
