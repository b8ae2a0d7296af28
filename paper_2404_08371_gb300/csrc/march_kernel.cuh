#pragma once
// Element-centric "marching" kernels: apply, diagonal and coefficient adjoint of the
// variable-coefficient and P2 operators.
//
// Eq. 4.1 / Algorithm 1 per micro-tet, traversed in the spirit of the cubes loop
// strategy (Section 5.2, Algorithm 3): one thread owns one cube of the index-space
// lattice and evaluates all six micro-tets in it, so every DoF of the cube is
// loaded once per cube and stays in registers.  A CTA of 32 lanes (i) x kWarps
// warps (j) marches upward through the cube layers k.  Element results are summed
// into points without atomics:
//   i: a lane adds the low-i face of its right neighbour (warp shuffle);
//   j: a warp adds the low-j face of the warp above it (shared memory);
//   k: the top face of a cube is carried in registers to the next layer.
// On small lattices adjacent CTAs overlap by one cube in i and j; the overlapping cube's points
// are written by exactly one of them.  On lattices of at least kMarchJAtomicN cubes per edge the
// tiles do not overlap in i or j: a point on a face between tiles is stored by the lowest of them,
// the others store their partial sums into a per-operator scratch (FaceScratch), and
// march_finish_kernel adds those in a fixed order and writes the Dirichlet rows; no atomics, so
// every apply is bitwise repeatable.
//
// Local matrices are never stored: the quadrature is fused with the local apply
// (Remark 4.1): grad u at each point from the 10 nodal values, scaled by
// k w |det J| J^{-1} J^{-T} (the hoisted per-class metric, Section 6.1), tested
// against the basis gradients.  Gradients of the P2 basis are written through the
// barycentric coordinates, so grad u = sum_a grad lambda_a s_a with
// s_a = u_a (4 lambda_a - 1) + 4 sum_b u_ab lambda_b.
#include <type_traits>

#include "hhg_internal.h"
#include "lattice.cuh"

namespace hhg {

constexpr int kWarps = kMarchWarps;   // warps per CTA along j

enum { MODE_APPLY = 0, MODE_DIAG = 1, MODE_ADJ = 2, MODE_RHS = 3, MODE_N1 = 4, MODE_N1D = 5 };
// the Nedelec modes: apply (MODE_N1) and diagonal (MODE_N1D)
__host__ __device__ constexpr bool is_n1_mode(int m) { return m == MODE_N1 || m == MODE_N1D; }

// Extra inputs of the Nedelec mode (unused otherwise).
template <typename T>
struct N1Args {
  const N1Const<T>* n1 = nullptr;
  const T* alpha = nullptr;   // P1 fields (packed degree-1 vectors) or null for constants
  const T* beta = nullptr;
  T alpha_c = T(0), beta_c = T(0);
  int n = 0;                  // cubes per edge (P1 lattice resolution)
};

// Partial sums of the points that neighbouring marching tiles share (lattices of at least
// kMarchJAtomicN cubes per edge).  Tiles own 32 x kWarps columns of cubes; a point on the face
// between two tiles along i (pi = Fi t, Fi = 32 R) or along j (pj = Fj t', Fj = kWarps R) gets a
// partial sum from each side, a point on both from four tiles.  The lowest tile stores its partial
// into the output; the others store theirs into this per-op scratch, one slot each: per macro the
// i-face points [0, Si) (faces t = 1..Ti, triangle (pj, pk) by rows pk), the j-face points
// [Si, Si + Sj) (faces t' = 1..Tj, triangle (pi, pk)) and the corner lines [Si + Sj, S)
// ((t, t') dense, pk = 0..N).  march_finish_kernel adds them in a fixed order.
template <typename T>
struct FaceScratch {
  T* d = nullptr;
  int64_t S = 0, Si = 0, Sj = 0;   // per macro: all slots, i-face slots, j-face slots
  int Ti = 0, Tj = 0;              // tile faces along i and j (pi = Fi t <= N, pj = Fj t' <= N)
};

// sum_{u=1}^{T} tri(N - F u), tri(m) = (m+1)(m+2)/2, in closed form
__host__ __device__ inline int64_t face_tri_sum(int64_t F, int64_t T, int64_t N) {
  const int64_t a = N + 1;
  return (T * a * (a + 1) - F * (2 * a + 1) * (T * (T + 1) / 2) + F * F * (T * (T + 1) * (2 * T + 1) / 6)) / 2;
}
__host__ __device__ inline int64_t face_tri_row(int64_t m, int64_t r) { return r * (2 * m + 3 - r) / 2; }

__host__ __device__ constexpr int coff(int o, int v, int d) {
  constexpr int t[6][4][3] = {
      {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {1, 1, 0}},
      {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {0, 1, 1}}, {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {0, 0, 1}},
      {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {1, 0, 0}}, {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}}};
  return t[o][v][d];
}
__host__ __device__ constexpr int edge_end(int e, int s) {
  constexpr int t[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  return t[e][s];
}
__host__ __device__ constexpr int class_shrink(int o) { return o == 0 ? 0 : (o == 5 ? 2 : 1); }

// Coefficient tag of the precomputed variant: local matrices read from device memory (kf points to
// them, layout [macro][class][entry][cube]); entries of the symmetric 10 x 10 P2 matrix a <= b.
constexpr int kCoefStored = 4;
__host__ __device__ constexpr int p2_sym(int a, int b) { return a * 10 - a * (a - 1) / 2 + (b - a); }
// Position (0..R per axis) of local node `node` of class o inside the cube block, linearised.
template <int R>
__host__ __device__ constexpr int node_slot(int o, int node) {
  int p[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    if (R == 1 || node < 4)
      p[d] = R * coff(o, node, d);
    else
      p[d] = coff(o, edge_end(node - 4, 0), d) + coff(o, edge_end(node - 4, 1), d);
  }
  return p[0] + (R + 1) * (p[1] + (R + 1) * p[2]);
}

template <typename T>
__device__ __forceinline__ T shfl_down(T v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}

// grad_ref u at a quadrature point from the 10 P2 nodal values, and y_i += r . grad_ref phi_i, with
// 4 lambda and 4 lambda - 1 tabulated per quadrature point (19 FP64 operations each); used for rules
// of few points, where the per-element set-up of the affine form below does not pay.
template <typename T>
__device__ __forceinline__ void p2_ref_grad_q(const T* u, const T* L4, const T* L4m1, T g[3]) {
  T s[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) s[a] = u[a] * L4m1[a];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = edge_end(e, 0), b = edge_end(e, 1);
    s[a] = fma(u[4 + e], L4[b], s[a]);
    s[b] = fma(u[4 + e], L4[a], s[b]);
  }
  g[0] = s[1] - s[0];
  g[1] = s[2] - s[0];
  g[2] = s[3] - s[0];
}

template <typename T>
__device__ __forceinline__ void p2_ref_test_q(const T r[3], const T* L4, const T* L4m1, T* y) {
  const T rho[4] = {-(r[0] + r[1] + r[2]), r[0], r[1], r[2]};   // r . grad lambda_a
#pragma unroll
  for (int a = 0; a < 4; ++a) y[a] = fma(L4m1[a], rho[a], y[a]);
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = edge_end(e, 0), b = edge_end(e, 1);
    y[4 + e] = fma(L4[a], rho[b], fma(L4[b], rho[a], y[4 + e]));
  }
}

// The reference gradient of a P2 function is affine in the barycentric coordinates:
// grad_ref u(lambda) = W0 + lambda_1 W1 + lambda_2 W2 + lambda_3 W3, with W formed once per
// micro-tet from W'_c = 4 u_c g_c + 4 sum_{edges (c, b)} u_(c,b) g_b - sum_a u_a g_a (g_a = grad_ref
// lambda_a), W0 = W'_0 and Wc = W'_c - W'_0; a quadrature point then costs 9 FMA.
template <int B, typename T>
__device__ __forceinline__ void add_gref(T v[3], T f) {
  if (B == 0) {
    v[0] -= f;
    v[1] -= f;
    v[2] -= f;
  } else {
    v[B - 1] += f;
  }
}

template <typename T>
__device__ __forceinline__ void p2_grad_affine(const T* u, T W[4][3]) {
  const T U[3] = {u[1] - u[0], u[2] - u[0], u[3] - u[0]};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) W[a][d] = -U[d];
  add_gref<0>(W[0], T(4) * u[0]);
  add_gref<1>(W[1], T(4) * u[1]);
  add_gref<2>(W[2], T(4) * u[2]);
  add_gref<3>(W[3], T(4) * u[3]);
  // edges (0,1) (0,2) (0,3) (1,2) (1,3) (2,3): W'_a += 4 u_e g_b, W'_b += 4 u_e g_a
  {
    const T f = T(4) * u[4];
    add_gref<1>(W[0], f);
    add_gref<0>(W[1], f);
  }
  {
    const T f = T(4) * u[5];
    add_gref<2>(W[0], f);
    add_gref<0>(W[2], f);
  }
  {
    const T f = T(4) * u[6];
    add_gref<3>(W[0], f);
    add_gref<0>(W[3], f);
  }
  {
    const T f = T(4) * u[7];
    add_gref<2>(W[1], f);
    add_gref<1>(W[2], f);
  }
  {
    const T f = T(4) * u[8];
    add_gref<3>(W[1], f);
    add_gref<1>(W[3], f);
  }
  {
    const T f = T(4) * u[9];
    add_gref<3>(W[2], f);
    add_gref<2>(W[3], f);
  }
#pragma unroll
  for (int c = 1; c < 4; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) W[c][d] -= W[0][d];
}

template <typename T>
__device__ __forceinline__ void p2_grad_at(const T W[4][3], T l1, T l2, T l3, T g[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) g[d] = fma(l3, W[3][d], fma(l2, W[2][d], fma(l1, W[1][d], W[0][d])));
}

// Testing against the P2 basis over all quadrature points through the moments
// S_ab = sum_q lambda_b rho_a and R_a = sum_q rho_a of rho_a = r . g_a (a, b = 1..3 accumulated):
// y_a += 4 S_aa - R_a for a vertex, y_(a,b) += 4 (S_ab + S_ba) for an edge.
template <typename T>
__device__ __forceinline__ void p2_test_moments(const T S3[3][3], const T R3[3], T* y) {
  T S[4][4], R[4];
#pragma unroll
  for (int a = 1; a < 4; ++a) {
    R[a] = R3[a - 1];
#pragma unroll
    for (int b = 1; b < 4; ++b) S[a][b] = S3[a - 1][b - 1];
    S[a][0] = R[a] - S[a][1] - S[a][2] - S[a][3];   // lambda_0 = 1 - lambda_1 - lambda_2 - lambda_3
  }
  R[0] = -(R[1] + R[2] + R[3]);                      // g_0 = -(g_1 + g_2 + g_3)
#pragma unroll
  for (int b = 0; b < 4; ++b) S[0][b] = -(S[1][b] + S[2][b] + S[3][b]);
#pragma unroll
  for (int a = 0; a < 4; ++a) y[a] += T(4) * S[a][a] - R[a];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = edge_end(e, 0), b = edge_end(e, 1);
    y[4 + e] += T(4) * (S[a][b] + S[b][a]);
  }
}

template <typename T>
__device__ __forceinline__ void metric(const T* M, const T g[3], T r[3]) {
  r[0] = M[0] * g[0] + M[3] * g[1] + M[4] * g[2];
  r[1] = M[3] * g[0] + M[1] * g[1] + M[5] * g[2];
  r[2] = M[4] * g[0] + M[5] * g[1] + M[2] * g[2];
}

template <typename T>
__device__ __forceinline__ void sincos2pi(T x, T* s, T* c);
template <>
__device__ __forceinline__ void sincos2pi<double>(double x, double* s, double* c) {
  sincospi(2.0 * x, s, c);
}
template <>
__device__ __forceinline__ void sincos2pi<float>(float x, float* s, float* c) {
  sincospif(2.0f * x, s, c);
}

// AFF (P2, variable coefficient, APPLY): affine gradient + moment test (rules of many points) or the
// tabulated direct form (rules of few points).
// The body of both entry points below.
template <typename T, int R, int COEF, int MODE, bool DIR, bool AFF, bool JATOM>
__device__ __forceinline__ void march_body(const OpConst<T>* __restrict__ cst, const int4* __restrict__ tasks, int kChunk,
                                           const T* __restrict__ x, const T* __restrict__ g,
                                           const T* __restrict__ kf, T* __restrict__ out, N1Args<T> n1a,
                                           FaceScratch<T> fs) {
  constexpr int P = R + 1;
  constexpr int P3 = P * P * P;
  constexpr int NL = R == 1 ? 4 : 10;
  __shared__ OpConst<T> c;
  __shared__ T xch[kWarps][P][R][32];
  __shared__ typename std::conditional<is_n1_mode(MODE), N1Const<T>, char>::type n1c;
  const int4 task = tasks[blockIdx.x];   // (i-tile, j-tile, k-chunk, macro), heaviest first
  const int macro = task.w;
  const int kc = task.z;
  {
    const int4* src = reinterpret_cast<const int4*>(cst + macro);
    int4* dst = reinterpret_cast<int4*>(&c);
    for (int t = threadIdx.x; t < (int)(sizeof(OpConst<T>) / sizeof(int4)); t += blockDim.x) dst[t] = src[t];
    if constexpr (is_n1_mode(MODE)) {
      const int4* s1 = reinterpret_cast<const int4*>(n1a.n1 + macro);
      int4* d1 = reinterpret_cast<int4*>(&n1c);
      for (int t = threadIdx.x; t < (int)(sizeof(N1Const<T>) / sizeof(int4)); t += blockDim.x) d1[t] = s1[t];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = c.n, N = c.N;
  constexpr int IW = JATOM ? 32 : 31, JW = JATOM ? kWarps : kWarps - 1;   // cubes owned along i, j
  const int ti0 = IW * task.x, tj0 = JW * task.y, K0 = kChunk * kc;
  if (ti0 + tj0 + K0 > n) return;   // lowest point owned by the CTA lies outside the macro (uniform)
  const int ci = ti0 + lane - (JATOM ? 0 : 1);
  const int cj = tj0 + warp - (JATOM ? 0 : 1);
  const int ck_last = min(K0 + kChunk - 1, n - ti0 - tj0);
  const int64_t base = c.base;
  const uint32_t table = c.bnd_table;
  // owned local index ranges in i (lanes) and j (warps)
  // (JATOM: lane 0 also owns its low face and lane 31 its high face, shared with the neighbouring
  // tiles through the face scratch)
  const int a_lo = lane == 0 ? (JATOM ? 0 : R) : 1, a_hi = (lane == 31 && !JATOM) ? R - 1 : R;
  const int b_lo = warp == 0 ? (JATOM ? 0 : R) : 1, b_hi = (warp == kWarps - 1 && !JATOM) ? R - 1 : R;

  T carry[P * P];
#pragma unroll
  for (int t = 0; t < P * P; ++t) carry[t] = T(0);
  // analytic coefficient in FP64: sin / cos of 2 pi x at the cube origin, evaluated once per
  // chunk and then rotated by the fixed angle 2 pi h_k of one k step (angle addition)
  constexpr bool kRotate = (COEF == HHG_COEFF_SIN3) && (sizeof(T) == 8);
  T so[3], co[3];
  if (kRotate) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T xd = c.X0[d] + T(ci) * c.H[0][d] + T(cj) * c.H[1][d] + T(K0 - 1) * c.H[2][d];
      sincos2pi<T>(xd, &so[d], &co[d]);
    }
  }

  for (int ck = K0 - 1; ck <= ck_last; ++ck) {
    if (kRotate && ck > K0 - 1) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T sn = so[d] * c.rot[d][0] + co[d] * c.rot[d][1];
        const T cn = co[d] * c.rot[d][0] - so[d] * c.rot[d][1];
        so[d] = sn;
        co[d] = cn;
      }
    }
    T acc[P3];
#pragma unroll
    for (int t = 0; t < P3; ++t) acc[t] = T(0);
    const bool cube_ok = ci >= 0 && cj >= 0 && ck >= 0 && ci + cj + ck <= n - 1;
    if (cube_ok) {
      // gather the cube block (masked: outside the macro or Dirichlet boundary -> 0)
      T xb[P3];
      T gb[MODE == MODE_ADJ ? P3 : 1];
      T kb[COEF == HHG_COEFF_FIELD_P1 || COEF == HHG_COEFF_FIELD_P2 ? P3 : 1];
#pragma unroll
      for (int cz = 0; cz < P; ++cz)
#pragma unroll
        for (int cy = 0; cy < P; ++cy)
#pragma unroll
          for (int cx = 0; cx < P; ++cx) {
            const int s = cx + P * (cy + P * cz);
            const int pi = R * ci + cx, pj = R * cj + cy, pk = R * ck + cz;
            const bool in = pi + pj + pk <= N;
            const int64_t idx = in ? packed_index(N, pi, pj, pk) : 0;
            const bool live = in && !(DIR && on_dirichlet(table, N, pi, pj, pk));
            if (MODE == MODE_APPLY || MODE == MODE_ADJ || MODE == MODE_N1) xb[s] = live ? __ldg(x + base + idx) : T(0);
            if (MODE == MODE_ADJ) gb[s] = live ? __ldg(g + base + idx) : T(0);
            if (COEF == HHG_COEFF_FIELD_P1 || COEF == HHG_COEFF_FIELD_P2) kb[s] = in ? __ldg(kf + c.kbase + idx) : T(0);
          }
      // Nedelec coefficients: P1 alpha / beta at the eight cube corners (inside the macro)
      T ca[is_n1_mode(MODE) ? 8 : 1], cb[is_n1_mode(MODE) ? 8 : 1];
      if constexpr (is_n1_mode(MODE) && COEF != kCoefStored) {
#pragma unroll
        for (int cn = 0; cn < 8; ++cn) {
          const int vi = ci + (cn & 1), vj = cj + ((cn >> 1) & 1), vk = ck + (cn >> 2);
          const bool in = vi + vj + vk <= n1a.n;
          const int64_t vidx = n1c.vbase + (in ? packed_index(n1a.n, vi, vj, vk) : 0);
          ca[cn] = n1a.alpha ? (in ? __ldg(n1a.alpha + vidx) : T(0)) : n1a.alpha_c;
          cb[cn] = n1a.beta ? (in ? __ldg(n1a.beta + vidx) : T(0)) : n1a.beta_c;
        }
      }
      // precomputed variant: the cube's entries in the stored local matrices
      const T* __restrict__ elem = nullptr;
      int64_t ncubes = 0;
      if constexpr (COEF == kCoefStored) {
        ncubes = dV(n - 1);
        elem = kf + (int64_t)macro * 6 * (is_n1_mode(MODE) ? kN1Sym : (R == 1 ? 1 : 55)) * ncubes +
               packed_index(n - 1, ci, cj, ck);
      }
      // analytic coefficient in FP32: sin / cos of 2 pi x at the cube origin, per coordinate
      if (COEF == HHG_COEFF_SIN3 && !kRotate) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T xd = c.X0[d] + T(ci) * c.H[0][d] + T(cj) * c.H[1][d] + T(ck) * c.H[2][d];
          sincos2pi<T>(xd, &so[d], &co[d]);
        }
      }
#pragma unroll
      for (int o = 0; o < 6; ++o) {
        if (ci + cj + ck > n - 1 - class_shrink(o)) continue;
        T ul[NL], yl[NL];
#pragma unroll
        for (int a = 0; a < NL; ++a) {
          ul[a] = (MODE == MODE_APPLY || MODE == MODE_ADJ || MODE == MODE_N1) ? xb[node_slot<R>(o, a)] : T(0);
          yl[a] = T(0);
        }
        if constexpr (is_n1_mode(MODE)) {
          // Nedelec edge element (Eq. N1): the six edge nodes of the P2 numbering carry the DoFs.
          // A_T = mean(alpha) C_o + sum_v beta_v M_o^v (symmetric, canonical orientation), formed
          // once per micro-tet and applied to the six edge values.
          if constexpr (R == 2) {
            T A[kN1Sym];
            if constexpr (COEF == kCoefStored) {
#pragma unroll
              for (int t = 0; t < kN1Sym; ++t) A[t] = __ldg(elem + ((int64_t)o * kN1Sym + t) * ncubes);
            } else {
              T av[4], bv[4];
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                const int cn = coff(o, v, 0) + 2 * coff(o, v, 1) + 4 * coff(o, v, 2);
                av[v] = ca[cn];
                bv[v] = cb[cn];
              }
              const T abar = T(0.25) * (av[0] + av[1] + av[2] + av[3]);
#pragma unroll
              for (int t = 0; t < kN1Sym; ++t)
                A[t] = abar * n1c.C[o][t] + bv[0] * n1c.M[o][0][t] + bv[1] * n1c.M[o][1][t] +
                       bv[2] * n1c.M[o][2][t] + bv[3] * n1c.M[o][3][t];
            }
            if constexpr (MODE == MODE_N1D) {
#pragma unroll
              for (int e = 0; e < 6; ++e) yl[4 + e] = A[n1_sym(e, e)];
            } else {
#pragma unroll
              for (int e = 0; e < 6; ++e) {
                T s = T(0);
#pragma unroll
                for (int f = 0; f < 6; ++f) s += A[e <= f ? n1_sym(e, f) : n1_sym(f, e)] * ul[4 + f];
                yl[4 + e] = s;
              }
            }
          }
        } else if (MODE == MODE_RHS) {
          // b_a += sum_q w_q |det J| f(x_q) phi_a(xi_q), f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
          for (int q = 0; q < c.nq; ++q) {
            T xq[3];
#pragma unroll
            for (int d = 0; d < 3; ++d)
              xq[d] = c.X0[d] + T(ci) * c.H[0][d] + T(cj) * c.H[1][d] + T(ck) * c.H[2][d] + c.qoff[o][q][d];
            const T f = T(3.0 * M_PI * M_PI) * sinpi(xq[0]) * sinpi(xq[1]) * sinpi(xq[2]);
            const T s = c.w[q] * c.adet[o] * f;
#pragma unroll
            for (int a = 0; a < NL; ++a) yl[a] += s * (R == 1 ? c.lam[q][a] : c.psi[q][a]);
          }
        } else if (R == 1) {
          // ---- P1: A_T = kbar_T A0_o with A0_o the hoisted constant matrix ----
          T kbar = T(1);
          if (COEF == HHG_COEFF_SIN3) {
            // k_T = 1 + sum_q 3 w_q prod_d sin(2 pi x_q,d), the factor 3 w_q in the x table
            kbar = T(1);
            for (int q = 0; q < c.nq; ++q) {
              T sv[3];
#pragma unroll
              for (int d = 0; d < 3; ++d) sv[d] = so[d] * c.cs[o][q][d][0] + co[d] * c.cs[o][q][d][1];
              kbar = fma(sv[0] * sv[1], sv[2], kbar);
            }
          } else if (COEF == HHG_COEFF_FIELD_P1) {
            kbar = T(0.25) * (kb[node_slot<R>(o, 0)] + kb[node_slot<R>(o, 1)] + kb[node_slot<R>(o, 2)] +
                              kb[node_slot<R>(o, 3)]);
          } else if (COEF == kCoefStored) {
            kbar = __ldg(elem + (int64_t)o * ncubes);
          }
          if (MODE == MODE_APPLY) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              T s = T(0);
#pragma unroll
              for (int b = 0; b < 4; ++b) s += c.A[o][a][b] * ul[b];
              yl[a] = kbar * s;
            }
          } else if (MODE == MODE_DIAG) {
#pragma unroll
            for (int a = 0; a < 4; ++a) yl[a] = kbar * c.A[o][a][a];
          } else {
            // dk_v += (1/4) g_T^T A0 u_T for each vertex v of T (P1 field, exact)
            T t = T(0);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              T s = T(0);
#pragma unroll
              for (int b = 0; b < 4; ++b) s += c.A[o][a][b] * ul[b];
              t += gb[node_slot<R>(o, a)] * s;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) yl[a] = T(0.25) * t;
          }
        } else if (COEF == kCoefStored) {
          // ---- P2 precomputed: the micro-tet's stored symmetric matrix ----
          const T* __restrict__ E = elem + (int64_t)o * 55 * ncubes;
          T Ae[55];
#pragma unroll
          for (int e = 0; e < 55; ++e) Ae[e] = __ldg(E + (int64_t)e * ncubes);
#pragma unroll
          for (int a = 0; a < 10; ++a) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < 10; ++b) s = fma(Ae[a <= b ? p2_sym(a, b) : p2_sym(b, a)], ul[b], s);
            yl[a] = s;
          }
        } else if (COEF == HHG_COEFF_CONST) {
          // ---- P2 constant: hoisted 10x10 matrix ----
          if (MODE == MODE_APPLY) {
#pragma unroll
            for (int a = 0; a < 10; ++a) {
              T s = T(0);
#pragma unroll
              for (int b = 0; b < 10; ++b) s += c.A[o][a][b] * ul[b];
              yl[a] = s;
            }
          } else {
#pragma unroll
            for (int a = 0; a < 10; ++a) yl[a] = c.A[o][a][a];
          }
        } else {
          // ---- P2 variable coefficient: fused quadrature (Remark 4.1) ----
          T gl[10];
          if (MODE == MODE_ADJ) {
#pragma unroll
            for (int a = 0; a < 10; ++a) gl[a] = gb[node_slot<R>(o, a)];
          }
          const T* M = c.M[o];
          constexpr bool affine = AFF;
          T Wu[4][3], Wg[4][3];
          T S3[3][3], R3[3];
          if ((MODE == MODE_APPLY && affine) || MODE == MODE_ADJ) {
            p2_grad_affine<T>(ul, Wu);
            // the metric is linear too: M grad_ref u = M W0 + sum_b lambda_b M Wb
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              T mw[3];
              metric<T>(M, Wu[t], mw);
              Wu[t][0] = mw[0];
              Wu[t][1] = mw[1];
              Wu[t][2] = mw[2];
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              R3[a] = T(0);
#pragma unroll
              for (int b = 0; b < 3; ++b) S3[a][b] = T(0);
            }
          }
          if (MODE == MODE_ADJ) p2_grad_affine<T>(gl, Wg);
#pragma unroll 2
          for (int q = 0; q < c.nq; ++q) {
            // s = w_q k(x_q): analytic, w_q + 0.5 w_q prod_d sin(2 pi x_q,d) with the factor 0.5 w_q
            // in the x table; P2 field, w_q sum_m k_m psi_m(x_q)
            T s;
            if (COEF == HHG_COEFF_SIN3) {
              T sv[3];
#pragma unroll
              for (int d = 0; d < 3; ++d) sv[d] = so[d] * c.cs[o][q][d][0] + co[d] * c.cs[o][q][d][1];
              s = fma(sv[0] * sv[1], sv[2], c.w[q]);
            } else {
              T kq = T(0);
#pragma unroll
              for (int m = 0; m < 10; ++m) kq += c.psi[q][m] * kb[node_slot<R>(o, m)];
              s = kq * c.w[q];
            }
            if (MODE == MODE_APPLY && !affine) {
              T gr[3], r[3];
              p2_ref_grad_q<T>(ul, c.lam4[q], c.lam4m1[q], gr);
              metric<T>(M, gr, r);
                            r[0] *= s;
              r[1] *= s;
              r[2] *= s;
              p2_ref_test_q<T>(r, c.lam4[q], c.lam4m1[q], yl);
            } else if (MODE == MODE_APPLY) {
              const T l1 = c.lam[q][1], l2 = c.lam[q][2], l3 = c.lam[q][3];
              T r[3];
              p2_grad_at<T>(Wu, l1, l2, l3, r);   // M grad_ref u at the point
              #pragma unroll
              for (int a = 0; a < 3; ++a) {
                const T ra = r[a] * s;
                R3[a] += ra;
                S3[a][0] = fma(l1, ra, S3[a][0]);
                S3[a][1] = fma(l2, ra, S3[a][1]);
                S3[a][2] = fma(l3, ra, S3[a][2]);
              }
            } else if (MODE == MODE_DIAG) {
              // grad_ref phi_a . M grad_ref phi_a for every node a
              #pragma unroll
              for (int a = 0; a < 10; ++a) {
                T e[10];
#pragma unroll
                for (int b = 0; b < 10; ++b) e[b] = T(a == b ? 1 : 0);
                T gr[3], r[3];
                p2_ref_grad_q<T>(e, c.lam4[q], c.lam4m1[q], gr);
                metric<T>(M, gr, r);
                yl[a] += s * (gr[0] * r[0] + gr[1] * r[1] + gr[2] * r[2]);
              }
            } else {
              T gg[3], r[3];
              p2_grad_at<T>(Wu, c.lam[q][1], c.lam[q][2], c.lam[q][3], r);   // M grad_ref u
              p2_grad_at<T>(Wg, c.lam[q][1], c.lam[q][2], c.lam[q][3], gg);
              const T t = c.w[q] * (gg[0] * r[0] + gg[1] * r[1] + gg[2] * r[2]);
#pragma unroll
              for (int m = 0; m < 10; ++m) yl[m] += c.psi[q][m] * t;
            }
          }
          if (MODE == MODE_APPLY && affine) p2_test_moments<T>(S3, R3, yl);
        }
#pragma unroll
        for (int a = 0; a < NL; ++a) acc[node_slot<R>(o, a)] += yl[a];
      }
    }
    // k: the bottom face receives the carried top face of the cube below; keep the new top face
#pragma unroll
    for (int t = 0; t < P * P; ++t) {
      acc[t] += carry[t];
      carry[t] = acc[t + R * P * P];
    }
    // i: add the low-i face of the right neighbour (planes 0..R-1)
#pragma unroll
    for (int cz = 0; cz < R; ++cz)
#pragma unroll
      for (int cy = 0; cy < P; ++cy) {
        const T v = shfl_down<T>(acc[0 + P * (cy + P * cz)]);
        if (lane < 31) acc[R + P * (cy + P * cz)] += v;
      }
    // j: add the low-j face of the warp above
#pragma unroll
    for (int cz = 0; cz < R; ++cz)
#pragma unroll
      for (int cx = 0; cx < P; ++cx) xch[warp][cx][cz][lane] = acc[cx + P * (0 + P * cz)];
    __syncthreads();
    if (warp < kWarps - 1) {
#pragma unroll
      for (int cz = 0; cz < R; ++cz)
#pragma unroll
        for (int cx = 0; cx < P; ++cx) acc[cx + P * (R + P * cz)] += xch[warp + 1][cx][cz][lane];
    }
    __syncthreads();
    // write the owned points of planes R*ck .. R*ck + R-1
    if (ck >= K0) {
#pragma unroll
      for (int cz = 0; cz < R; ++cz)
#pragma unroll
        for (int cy = 0; cy < P; ++cy)
#pragma unroll
          for (int cx = 0; cx < P; ++cx) {
            if (cx < a_lo || cx > a_hi || cy < b_lo || cy > b_hi) continue;
            const int pi = R * ci + cx, pj = R * cj + cy, pk = R * ck + cz;
            if (pi < 0 || pj < 0 || pi + pj + pk > N) continue;
            const int64_t idx = base + packed_index(N, pi, pj, pk);
            T v = acc[cx + P * (cy + P * cz)];
            if (JATOM) {
              // Dirichlet rows: written by march_finish_kernel
              if (DIR && MODE != MODE_ADJ && on_dirichlet(table, N, pi, pj, pk)) continue;
              // the tile above the lowest along i (lane 0, point cx = 0) or along j (warp 0, cy = 0)
              // of a shared face point stores its partial sum into the scratch
              const bool si = cx == 0 && lane == 0 && ti0 > 0, sj = cy == 0 && warp == 0 && tj0 > 0;
              if (!si && !sj) {
                out[idx] = v;
              } else {
                int64_t slot;
                if (si && !sj)
                  slot = face_tri_sum(32 * R, task.x - 1, N) + face_tri_row(N - pi, pk) + pj;
                else if (!si)
                  slot = fs.Si + face_tri_sum(kWarps * R, task.y - 1, N) + face_tri_row(N - pj, pk) + pi;
                else
                  slot = fs.Si + fs.Sj + ((int64_t)(task.x - 1) * fs.Tj + (task.y - 1)) * (N + 1) + pk;
                fs.d[(int64_t)macro * fs.S + slot] = v;
              }
              continue;
            }
            if (DIR && MODE != MODE_ADJ && on_dirichlet(table, N, pi, pj, pk))
              v = (MODE == MODE_APPLY || MODE == MODE_N1) ? x[idx] : (MODE == MODE_DIAG || MODE == MODE_N1D ? T(1) : T(0));
            out[idx] = v;
          }
    }
  }
}

// The variants that compute their local matrices: the compiler's own register choice (an explicit
// minimum of one CTA per SM makes it take up to 60% more registers and halves the CTAs of the FP32
// variants).
template <typename T, int R, int COEF, int MODE, bool DIR, bool AFF = true, bool JATOM = false>
__global__ void __launch_bounds__(32 * kWarps) march_kernel(const OpConst<T>* __restrict__ cst,
                                                            const int4* __restrict__ tasks, int kChunk,
                                                            const T* __restrict__ x, const T* __restrict__ g,
                                                            const T* __restrict__ kf, T* __restrict__ out,
                                                            N1Args<T> n1a, FaceScratch<T> fs) {
  march_body<T, R, COEF, MODE, DIR, AFF, JATOM>(cst, tasks, kChunk, x, g, kf, out, n1a, fs);
}

// The stored variant streams its local matrices from HBM: two CTAs per SM (at most 128 registers a
// thread) keep enough loads in flight.
template <typename T, int R, int MODE, bool DIR, bool AFF = true, bool JATOM = false>
__global__ void __launch_bounds__(32 * kWarps, 2) march_stored_kernel(const OpConst<T>* __restrict__ cst,
                                                                      const int4* __restrict__ tasks, int kChunk,
                                                                      const T* __restrict__ x, const T* __restrict__ g,
                                                                      const T* __restrict__ kf, T* __restrict__ out,
                                                                      N1Args<T> n1a, FaceScratch<T> fs) {
  march_body<T, R, kCoefStored, MODE, DIR, AFF, JATOM>(cst, tasks, kChunk, x, g, kf, out, n1a, fs);
}

template <typename T, int R, int COEF, int MODE, bool DIR, bool AFF, bool JATOM>
void launch_march_grid(unsigned grid, cudaStream_t s, const OpConst<T>* cst, const int4* tasks, int kChunk, const T* x,
                       const T* g, const T* kf, T* out, N1Args<T> n1a, FaceScratch<T> fs) {
  if constexpr (COEF == kCoefStored)
    march_stored_kernel<T, R, MODE, DIR, AFF, JATOM><<<grid, 32 * kWarps, 0, s>>>(cst, tasks, kChunk, x, g, kf, out, n1a, fs);
  else
    march_kernel<T, R, COEF, MODE, DIR, AFF, JATOM><<<grid, 32 * kWarps, 0, s>>>(cst, tasks, kChunk, x, g, kf, out, n1a, fs);
}

// Row and position of entry r of a triangle of rows 0..m, row q holding m - q + 1 entries.
__device__ __forceinline__ void tri_decode(int m, int64_t r, int& row, int& pos) {
  const float bq = 2.0f * m + 3.0f;
  int q = (int)(0.5f * (bq - sqrtf(fmaxf(bq * bq - 8.0f * (float)r, 0.0f))));
  q = max(0, min(q, m));
  if (q < m && face_tri_row(m, q + 1) <= r) ++q;
  if (q > 0 && face_tri_row(m, q) > r) --q;
  row = q;
  pos = (int)(r - face_tri_row(m, q));
}

// Largest t in 1..T with face_tri_sum(F, t - 1, N) <= q (the tile face holding compact slot q).
__device__ __forceinline__ int face_of_slot(int64_t F, int T, int64_t N, int64_t q) {
  int lo = 1, hi = T;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (face_tri_sum(F, mid - 1, N) <= q)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Completes a march on lattices of at least kMarchJAtomicN cubes per edge; blockIdx.y = macro.
// Blocks x < nfb: every shared tile-face point adds the partial sums that the tiles above the
// lowest stored in the scratch, in the fixed order ((lowest + i-side) + j-side) + corner, so an
// apply is bitwise repeatable.  Blocks x >= nfb (dir_rows): the Dirichlet rows, y = x (apply,
// Nedelec), 1 (diagonal) or 0 (load vector), one thread per point of each macro face triangle;
// the first part leaves those points alone (skip_dir), so no point is written by both.
template <typename T>
__global__ void march_finish_kernel(const OpConst<T>* __restrict__ cst, int R, int mode, bool dir_rows, bool skip_dir,
                                    const T* __restrict__ x, T* __restrict__ y, FaceScratch<T> fs, int nfb) {
  const OpConst<T>& c = cst[blockIdx.y];
  const int N = c.N;
  const uint32_t table = c.bnd_table;
  if ((int)blockIdx.x < nfb) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= fs.Si + fs.Sj) return;
    const int Fi = 32 * R, Fj = kWarps * R;
    const T* __restrict__ D = fs.d + (int64_t)blockIdx.y * fs.S;
    int pi, pj, pk;
    if (q < fs.Si) {
      const int t = face_of_slot(Fi, fs.Ti, N, q);
      tri_decode(N - Fi * t, q - face_tri_sum(Fi, t - 1, N), pk, pj);
      pi = Fi * t;
    } else {
      const int64_t q2 = q - fs.Si;
      const int t2 = face_of_slot(Fj, fs.Tj, N, q2);
      tri_decode(N - Fj * t2, q2 - face_tri_sum(Fj, t2 - 1, N), pk, pi);
      pj = Fj * t2;
      if (pi > 0 && pi % Fi == 0) return;   // on an i-face too: summed by that face's slot
    }
    if (skip_dir && on_dirichlet(table, N, pi, pj, pk)) return;
    const int64_t idx = c.base + packed_index(N, pi, pj, pk);
    T v = y[idx] + D[q];
    if (q < fs.Si && pj > 0 && pj % Fj == 0) {
      const int t = pi / Fi, t2 = pj / Fj;
      v += D[fs.Si + face_tri_sum(Fj, t2 - 1, N) + face_tri_row(N - pj, pk) + pi];
      v += D[fs.Si + fs.Sj + ((int64_t)(t - 1) * fs.Tj + (t2 - 1)) * (N + 1) + pk];
    }
    y[idx] = v;
    return;
  }
  if (!dir_rows) return;
  const int nb = (int)((((int64_t)N + 1) * (N + 2) / 2 + blockDim.x - 1) / blockDim.x);
  const int b = blockIdx.x - nfb, f = b / nb;
  const int t = (b - f * nb) * blockDim.x + threadIdx.x;
  if (t >= (N + 1) * (N + 2) / 2) return;
  int rowb, a;
  tri_decode(N, t, rowb, a);   // (a, rowb) with a + rowb <= N
  int i, j, k;
  if (f == 0) {
    i = 0; j = a; k = rowb;
  } else if (f == 1) {
    i = a; j = 0; k = rowb;
  } else if (f == 2) {
    i = a; j = rowb; k = 0;
  } else {
    i = N - a - rowb; j = a; k = rowb;
  }
  if (!on_dirichlet(table, N, i, j, k)) return;
  const int64_t idx = c.base + packed_index(N, i, j, k);
  y[idx] = (mode == MODE_DIAG || mode == MODE_N1D) ? T(1) : (mode == MODE_RHS ? T(0) : x[idx]);
}

template <typename T>
FaceScratch<T> face_scratch(const hhg_op* op) {
  FaceScratch<T> f;
  f.d = (T*)op->d_face;
  f.S = op->face_S;
  f.Si = op->face_Si;
  f.Sj = op->face_Sj;
  f.Ti = op->face_Ti;
  f.Tj = op->face_Tj;
  return f;
}

template <typename T, int R, int COEF, int MODE, bool AFF = true>
int launch_march_t(const hhg_op* op, const OpConst<T>* cst, const T* x, const T* g, const T* kf, T* out,
                          cudaStream_t s, N1Args<T> n1a = N1Args<T>()) {
  const Interface* I = op->itf;
  const unsigned grid = (unsigned)I->n_march_tasks;
  const bool dir = op->bc == HHG_DIRICHLET;
  if (march_jw(op->n) == kMarchWarps) {
    if (!op->d_face) return fail(HHG_E_CUDA, "march: the operator has no tile-face scratch");
    const FaceScratch<T> fs = face_scratch<T>(op);
    if (dir)
      launch_march_grid<T, R, COEF, MODE, true, AFF, true>(grid, s, cst, I->d_march_tasks, I->march_kchunk, x, g, kf,
                                                           out, n1a, fs);
    else
      launch_march_grid<T, R, COEF, MODE, false, AFF, true>(grid, s, cst, I->d_march_tasks, I->march_kchunk, x, g, kf,
                                                            out, n1a, fs);
    HHG_CUDA_TRY(cudaGetLastError());
    const bool rows = dir && MODE != MODE_ADJ;
    const int nfb = (int)((fs.Si + fs.Sj + 255) / 256);
    const int nb = rows ? 4 * (int)((((int64_t)op->N + 1) * (op->N + 2) / 2 + 255) / 256) : 0;
    if (nfb + nb > 0) {
      march_finish_kernel<T><<<dim3((unsigned)(nfb + nb), op->mesh->nmacro()), 256, 0, s>>>(
          cst, R, MODE, rows, rows, x, out, fs, nfb);
      HHG_CUDA_TRY(cudaGetLastError());
    }
    return HHG_OK;
  }
  if (dir)
    launch_march_grid<T, R, COEF, MODE, true, AFF, false>(grid, s, cst, I->d_march_tasks, I->march_kchunk, x, g, kf, out,
                                                          n1a, FaceScratch<T>());
  else
    launch_march_grid<T, R, COEF, MODE, false, AFF, false>(grid, s, cst, I->d_march_tasks, I->march_kchunk, x, g, kf, out,
                                                           n1a, FaceScratch<T>());
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

}  // namespace hhg

// The explicit instantiations of launch_march_t are spread over the translation units
// march_inst_<n>.cu so that they compile in parallel; march.cu declares them extern.
#define HHG_MARCH_DECL(T, R, C, M, A)                                                                   \
  int hhg::launch_march_t<T, R, C, M, A>(const hhg_op*, const hhg::OpConst<T>*, const T*, const T*, const T*, \
                                         T*, cudaStream_t, hhg::N1Args<T>)
#define HHG_MARCH_SHARD_0(X)                                                                            \
  X(double, 1, HHG_COEFF_SIN3, hhg::MODE_APPLY, true) X(double, 1, HHG_COEFF_FIELD_P1, hhg::MODE_APPLY, true) \
  X(double, 1, HHG_COEFF_SIN3, hhg::MODE_DIAG, true) X(double, 1, HHG_COEFF_FIELD_P1, hhg::MODE_DIAG, true) \
  X(double, 1, HHG_COEFF_FIELD_P1, hhg::MODE_ADJ, true) X(double, 1, hhg::kCoefStored, hhg::MODE_APPLY, true) \
  X(double, 1, HHG_COEFF_CONST, hhg::MODE_RHS, true)
#define HHG_MARCH_SHARD_1(X)                                                                            \
  X(float, 1, HHG_COEFF_SIN3, hhg::MODE_APPLY, true) X(float, 1, HHG_COEFF_FIELD_P1, hhg::MODE_APPLY, true) \
  X(float, 1, HHG_COEFF_SIN3, hhg::MODE_DIAG, true) X(float, 1, HHG_COEFF_FIELD_P1, hhg::MODE_DIAG, true) \
  X(float, 1, HHG_COEFF_FIELD_P1, hhg::MODE_ADJ, true) X(float, 1, hhg::kCoefStored, hhg::MODE_APPLY, true)
#define HHG_MARCH_SHARD_2(X)                                                                            \
  X(double, 2, HHG_COEFF_SIN3, hhg::MODE_APPLY, true) X(double, 2, HHG_COEFF_SIN3, hhg::MODE_APPLY, false) \
  X(double, 2, HHG_COEFF_FIELD_P2, hhg::MODE_APPLY, true) X(double, 2, HHG_COEFF_FIELD_P2, hhg::MODE_APPLY, false)
#define HHG_MARCH_SHARD_3(X)                                                                            \
  X(float, 2, HHG_COEFF_SIN3, hhg::MODE_APPLY, true) X(float, 2, HHG_COEFF_SIN3, hhg::MODE_APPLY, false) \
  X(float, 2, HHG_COEFF_FIELD_P2, hhg::MODE_APPLY, true) X(float, 2, HHG_COEFF_FIELD_P2, hhg::MODE_APPLY, false)
#define HHG_MARCH_SHARD_4(X)                                                                            \
  X(double, 2, HHG_COEFF_SIN3, hhg::MODE_DIAG, true) X(double, 2, HHG_COEFF_FIELD_P2, hhg::MODE_DIAG, true) \
  X(double, 2, HHG_COEFF_FIELD_P2, hhg::MODE_ADJ, true) X(double, 2, HHG_COEFF_CONST, hhg::MODE_RHS, true)
#define HHG_MARCH_SHARD_5(X)                                                                            \
  X(float, 2, HHG_COEFF_SIN3, hhg::MODE_DIAG, true) X(float, 2, HHG_COEFF_FIELD_P2, hhg::MODE_DIAG, true) \
  X(float, 2, HHG_COEFF_FIELD_P2, hhg::MODE_ADJ, true)
#define HHG_MARCH_SHARD_6(X)                                                                            \
  X(double, 2, HHG_COEFF_CONST, hhg::MODE_APPLY, true) X(double, 2, hhg::kCoefStored, hhg::MODE_APPLY, true) \
  X(double, 2, hhg::kCoefStored, hhg::MODE_N1, true) X(double, 2, HHG_COEFF_CONST, hhg::MODE_N1, true) \
  X(double, 2, HHG_COEFF_CONST, hhg::MODE_N1D, true)
#define HHG_MARCH_SHARD_7(X)                                                                            \
  X(float, 2, HHG_COEFF_CONST, hhg::MODE_APPLY, true) X(float, 2, hhg::kCoefStored, hhg::MODE_APPLY, true) \
  X(float, 2, hhg::kCoefStored, hhg::MODE_N1, true) X(float, 2, HHG_COEFF_CONST, hhg::MODE_N1, true) \
  X(float, 2, HHG_COEFF_CONST, hhg::MODE_N1D, true)
#define HHG_MARCH_INSTANTIATE(T, R, C, M, A) template HHG_MARCH_DECL(T, R, C, M, A);
#define HHG_MARCH_EXTERN(T, R, C, M, A) extern template HHG_MARCH_DECL(T, R, C, M, A);
