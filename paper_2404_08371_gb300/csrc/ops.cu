// Operator set-up and the P1 constant-coefficient apply; interface reconciliation kernels.
//
// Eq. 4.1: A = sum_T P_T A_T R_T.  All micro-tets of one class are translates
// of each other, so their Jacobians -- and, for a constant coefficient, their
// local matrices -- are loop invariants (Section 6.1).  They are computed once
// per macro and class on the host in FP64 ("hoisted") and handed to the kernels.
// For P1 with a constant coefficient the six per-class 4x4 matrices fold into
// one 15-point stencil at points whose incident micro-tets all lie in the
// macro; points next to the macro boundary use the per-class matrices with an
// explicit validity test of each incident micro-tet.  The apply gathers into
// each output point (no atomics); every point is written by exactly one thread.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "hhg_internal.h"
#include "lattice.cuh"

namespace hhg {

// ---------------------------------------------------------------------------
// Host: hoisted per-class invariants (Section 6.1) and local matrices.
// ---------------------------------------------------------------------------
static void inv3(const double J[3][3], double Ji[3][3], double* det) {
  double d = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  *det = d;
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / d;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / d;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / d;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / d;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / d;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / d;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / d;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / d;
}

// Reference gradients of the P1 / P2 basis at a reference point.
static void ref_grads(int degree, const double* xi, double g[10][3]) {
  const double gl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double lam[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
  if (degree == 1) {
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) g[a][d] = gl[a][d];
    return;
  }
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) g[a][d] = (4.0 * lam[a] - 1.0) * gl[a][d];
  for (int e = 0; e < 6; ++e) {
    int a = kP2Edges[e][0], b = kP2Edges[e][1];
    for (int d = 0; d < 3; ++d) g[4 + e][d] = 4.0 * (lam[a] * gl[b][d] + lam[b] * gl[a][d]);
  }
}

static void build_const(hhg_op* op) {
  const hhg_mesh* mesh = op->mesh;
  const int n = op->n;
  const int nloc = op->degree == 1 ? 4 : 10;
  const double kval = op->coeff.type == HHG_COEFF_CONST ? op->coeff.value : 1.0;
  QuadRule r2;
  quad_rule(2, &r2);   // exact for the degree-2 integrand of the constant P2 matrix
  const int Nk = op->coeff.type == HHG_COEFF_FIELD_P2 ? 2 * n : n;
  op->h_const.assign(mesh->nmacro(), OpConst<double>{});
  for (int m = 0; m < mesh->nmacro(); ++m) {
    const MacroGeom& g = mesh->macros[m];
    OpConst<double>& c = op->h_const[m];
    std::memset(&c, 0, sizeof(c));
    c.base = (int64_t)m * lattice_size(op->N);
    c.kbase = (int64_t)m * lattice_size(Nk);
    c.bnd_table = g.bnd_table;
    c.own_table = g.own_table;
    c.N = op->N;
    c.n = n;
    for (int d = 0; d < 3; ++d) c.x0[d] = g.p0[d];
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) c.h[a][d] = g.e[a][d] / n;
    for (int o = 0; o < 6; ++o) {
      // J = H D with H columns h_a and D columns off_b - off_0 (index space)
      double J[3][3], Ji[3][3], det;
      for (int r = 0; r < 3; ++r)
        for (int b = 0; b < 3; ++b) {
          double s = 0;
          for (int a = 0; a < 3; ++a) s += c.h[a][r] * (kClassOffsets[o][b + 1][a] - kClassOffsets[o][0][a]);
          J[r][b] = s;
        }
      inv3(J, Ji, &det);
      const double adet = std::fabs(det);
      double Mm[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double s = 0;
          for (int t = 0; t < 3; ++t) s += Ji[a][t] * Ji[b][t];
          Mm[a][b] = adet * s;
        }
      c.adet[o] = adet;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) c.Jinv[o][a * 3 + b] = Ji[a][b];
      c.M[o][0] = Mm[0][0];
      c.M[o][1] = Mm[1][1];
      c.M[o][2] = Mm[2][2];
      c.M[o][3] = Mm[0][1];
      c.M[o][4] = Mm[0][2];
      c.M[o][5] = Mm[1][2];
      // constant-coefficient local matrix: sum_q w_q grad_ref_i^T M grad_ref_j (times k)
      for (int q = 0; q < r2.nq(); ++q) {
        double gr[10][3];
        ref_grads(op->degree, &r2.xi[3 * q], gr);
        for (int i = 0; i < nloc; ++i)
          for (int j = 0; j < nloc; ++j) {
            double s = 0;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) s += gr[i][a] * Mm[a][b] * gr[j][b];
            c.A[o][i][j] += kval * r2.w[q] * s;
          }
      }
    }
    // quadrature tables for variable coefficients (the op's rule)
    const QuadRule& rq = op->rule;
    c.nq = rq.nq();
    for (int d = 0; d < 3; ++d) {
      c.X0[d] = c.x0[d];
      c.rot[d][0] = std::cos(2.0 * M_PI * c.h[2][d]);
      c.rot[d][1] = std::sin(2.0 * M_PI * c.h[2][d]);
    }
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) c.H[a][d] = c.h[a][d];
    for (int q = 0; q < rq.nq() && q < kMaxQ; ++q) {
      const double* xi = &rq.xi[3 * q];
      const double lam[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
      c.w[q] = rq.w[q];
      for (int a = 0; a < 4; ++a) {
        c.lam[q][a] = lam[a];
        c.psi[q][a] = lam[a] * (2.0 * lam[a] - 1.0);
      }
      for (int e = 0; e < 6; ++e) c.psi[q][4 + e] = 4.0 * lam[kP2Edges[e][0]] * lam[kP2Edges[e][1]];
      for (int o = 0; o < 6; ++o) {
        // index-space offset of the point from the cube origin: off_o[0] + D_o xi
        double ref[3];
        for (int a = 0; a < 3; ++a) {
          ref[a] = kClassOffsets[o][0][a];
          for (int b = 0; b < 3; ++b) ref[a] += (kClassOffsets[o][b + 1][a] - kClassOffsets[o][0][a]) * xi[b];
        }
        for (int d = 0; d < 3; ++d) {
          double delta = 0;
          for (int a = 0; a < 3; ++a) delta += c.h[a][d] * ref[a];
          c.cs[o][q][d][0] = std::cos(2.0 * M_PI * delta);
          c.cs[o][q][d][1] = std::sin(2.0 * M_PI * delta);
          c.qoff[o][q][d] = delta;
        }
      }
    }
    if (op->degree == 1) {
      // stencils of a point inside each macro face: the incident micro-tets that lie in the
      // macro are the same for every such point; found on a probe point of a level-3 macro
      for (int a = 0; a < 4; ++a) {
        const int M = 8;
        const int probe[4][3] = {{3, 3, 2}, {0, 3, 3}, {3, 0, 3}, {3, 3, 0}};
        const int* v = probe[a];
        for (int o = 0; o < 6; ++o)
          for (int la = 0; la < 4; ++la) {
            int cc[3];
            for (int t = 0; t < 3; ++t) cc[t] = v[t] - kClassOffsets[o][la][t];
            bool ok = true;
            for (int lb = 0; lb < 4 && ok; ++lb) {
              int q[3], sum = 0;
              for (int t = 0; t < 3; ++t) {
                q[t] = cc[t] + kClassOffsets[o][lb][t];
                sum += q[t];
                if (q[t] < 0) ok = false;
              }
              if (sum > M) ok = false;
            }
            if (!ok) continue;
            for (int lb = 0; lb < 4; ++lb) {
              int d[3];
              for (int t = 0; t < 3; ++t) d[t] = kClassOffsets[o][lb][t] - kClassOffsets[o][la][t];
              for (int st = 0; st < 15; ++st)
                if (d[0] == kStencil[st][0] && d[1] == kStencil[st][1] && d[2] == kStencil[st][2])
                  c.Sface[a][st] += c.A[o][la][lb];
            }
          }
      }
      // fold the six per-class matrices into the 15-point stencil of a point whose incident tets all exist
      for (int o = 0; o < 6; ++o)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            int d[3];
            for (int t = 0; t < 3; ++t) d[t] = kClassOffsets[o][b][t] - kClassOffsets[o][a][t];
            for (int s = 0; s < 15; ++s)
              if (d[0] == kStencil[s][0] && d[1] == kStencil[s][1] && d[2] == kStencil[s][2]) c.S[s] += c.A[o][a][b];
          }
    }
  }
}

template <typename T>
static OpConst<T> convert_const(const OpConst<double>& c) {
  OpConst<T> o;
  std::memset(&o, 0, sizeof(o));
  o.base = c.base;
  o.kbase = c.kbase;
  o.bnd_table = c.bnd_table;
  o.own_table = c.own_table;
  o.N = c.N;
  o.n = c.n;
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 10; ++b)
      for (int d = 0; d < 10; ++d) o.A[a][b][d] = (T)c.A[a][b][d];
  for (int s = 0; s < 15; ++s) {
    o.S[s] = (T)c.S[s];
    for (int a = 0; a < 4; ++a) o.Sface[a][s] = (T)c.Sface[a][s];
  }
  for (int a = 0; a < 6; ++a) {
    o.adet[a] = (T)c.adet[a];
    for (int b = 0; b < 9; ++b) o.Jinv[a][b] = (T)c.Jinv[a][b];
    for (int b = 0; b < 6; ++b) o.M[a][b] = (T)c.M[a][b];
  }
  std::memcpy(o.x0, c.x0, sizeof(c.x0));
  std::memcpy(o.h, c.h, sizeof(c.h));
  o.nq = c.nq;
  for (int q = 0; q < kMaxQ; ++q) {
    o.w[q] = (T)c.w[q];
    for (int a = 0; a < 4; ++a) o.lam[q][a] = (T)c.lam[q][a];
    for (int m = 0; m < 10; ++m) o.psi[q][m] = (T)c.psi[q][m];
    for (int cl = 0; cl < 6; ++cl)
      for (int d = 0; d < 3; ++d) {
        o.qoff[cl][q][d] = (T)c.qoff[cl][q][d];
        for (int t = 0; t < 2; ++t) o.cs[cl][q][d][t] = (T)c.cs[cl][q][d][t];
      }
  }
  for (int d = 0; d < 3; ++d) {
    o.rot[d][0] = (T)c.rot[d][0];
    o.rot[d][1] = (T)c.rot[d][1];
    o.X0[d] = (T)c.X0[d];
    for (int a = 0; a < 3; ++a) o.H[a][d] = (T)c.H[a][d];
  }
  return o;
}

// ---------------------------------------------------------------------------
// Device: P1 constant-coefficient apply (gather; one thread per output point).
// A CTA covers 256 consecutive points of one plane k; the plane of each CTA and
// the first packed position of each plane come from small per-level tables, so
// the index arithmetic is 32-bit and free of divisions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tri(int s) { return ((s + 1) * (s + 2)) >> 1; }          // points of a plane
__device__ __forceinline__ int row32(int s, int j) { return (j * (2 * s + 3 - j)) >> 1; }  // row start in plane

// Point on a macro face that is not a Dirichlet point (Neumann, or an interface between
// macros): sum the incident micro-tets that exist (Algorithm 1 per tet).
template <typename T, bool DIRICHLET>
__device__ __noinline__ T p1_face_point(const OpConst<T>& c, const int* __restrict__ pstart, const T* __restrict__ xm,
                                        int i, int j, int k) {
  const int N = c.N;
  const uint32_t table = c.bnd_table;
  T acc = T(0);
  for (int o = 0; o < 6; ++o) {
    const int lim = N - 1 - (o == 0 ? 0 : (o == 5 ? 2 : 1));
    for (int a = 0; a < 4; ++a) {
      const int ci = i - kClassOffsetsD[o][a][0], cj = j - kClassOffsetsD[o][a][1], ck = k - kClassOffsetsD[o][a][2];
      if (ci < 0 || cj < 0 || ck < 0 || ci + cj + ck > lim) continue;
      for (int b2 = 0; b2 < 4; ++b2) {
        const int pi = ci + kClassOffsetsD[o][b2][0], pj = cj + kClassOffsetsD[o][b2][1],
                  pkk = ck + kClassOffsetsD[o][b2][2];
        if (DIRICHLET && on_dirichlet(table, N, pi, pj, pkk)) continue;
        acc += c.A[o][a][b2] * __ldg(xm + __ldg(pstart + pkk) + row32(N - pkk, pj) + pi);
      }
    }
  }
  return acc;
}

// P1 constant-coefficient apply, one thread per output point (gather).  A CTA covers 256
// consecutive points of one plane k; the plane of each CTA and the first packed position of each
// plane come from per-level tables, so the index arithmetic is 32-bit and free of divisions.
// Points off the macro faces use the 15-point stencil (Dirichlet columns dropped near Dirichlet
// faces), points inside a face the face's stencil, points on macro edges/vertices the per-tet sum.
template <typename T, bool DIRICHLET>
__global__ void __launch_bounds__(256) p1_gather_kernel(const OpConst<T>* __restrict__ cst,
                                                              const int* __restrict__ cta_plane,
                                                              const int* __restrict__ cta_start,
                                                              const int* __restrict__ pstart,
                                                              const T* __restrict__ x, T* __restrict__ y) {
  const OpConst<T>& c = cst[blockIdx.y];
  const int N = c.N;
  const int k = __ldg(cta_plane + blockIdx.x);
  const int s = N - k;
  const int q = (blockIdx.x - __ldg(cta_start + k)) * 256 + threadIdx.x;
  if (q >= tri(s)) return;
  // row j: largest j with row32(s, j) <= q
  const float b = 2.0f * s + 3.0f;
  int j = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)q, 0.0f))));
  j = max(0, min(j, s));
  if (j < s && row32(s, j + 1) <= q) ++j;
  if (j > 0 && row32(s, j) > q) --j;
  const int i = q - row32(s, j);
  const int pk = __ldg(pstart + k);
  const int p = pk + q;
  const T* __restrict__ xm = x + c.base;
  T* __restrict__ ym = y + c.base;
  const uint32_t table = c.bnd_table;
  const bool on_face = (i == 0) | (j == 0) | (k == 0) | (i + j + k == N);
  T acc = T(0);
  if (!on_face) {
    // all 24 incident micro-tets exist: 15-point stencil
    const int r00 = p - i;                                 // (j, k)
    const int rp0 = r00 + (s + 1 - j);                     // (j+1, k)
    const int rm0 = r00 - (s + 2 - j);                     // (j-1, k)
    const int pk1 = pk + tri(s);
    const int r01 = pk1 + row32(s - 1, j);                 // (j, k+1)
    const int rm1 = pk1 + row32(s - 1, j - 1);             // (j-1, k+1)
    const int pkm = pk - tri(s + 1);
    const int r0m = pkm + row32(s + 1, j);                 // (j, k-1)
    const int rpm = pkm + row32(s + 1, j + 1);             // (j+1, k-1)
    T v[15];
    v[0] = __ldg(xm + r00 + i);
    v[1] = __ldg(xm + r00 + i + 1);
    v[2] = __ldg(xm + r00 + i - 1);
    v[3] = __ldg(xm + rp0 + i);
    v[4] = __ldg(xm + rm0 + i);
    v[5] = __ldg(xm + r01 + i);
    v[6] = __ldg(xm + r0m + i);
    v[7] = __ldg(xm + rm0 + i + 1);
    v[8] = __ldg(xm + rp0 + i - 1);
    v[9] = __ldg(xm + r0m + i + 1);
    v[10] = __ldg(xm + r01 + i - 1);
    v[11] = __ldg(xm + rpm + i);
    v[12] = __ldg(xm + rm1 + i);
    v[13] = __ldg(xm + rm1 + i + 1);
    v[14] = __ldg(xm + rpm + i - 1);
    if (DIRICHLET && !(i >= 2 && j >= 2 && k >= 2 && i + j + k <= N - 2)) {
      // a neighbour may lie on a Dirichlet face: its column is dropped
#pragma unroll
      for (int d = 0; d < 15; ++d)
        if (on_dirichlet(table, N, i + kStencilD[d][0], j + kStencilD[d][1], k + kStencilD[d][2])) v[d] = T(0);
    }
#pragma unroll
    for (int d = 0; d < 15; ++d) acc += c.S[d] * v[d];
  } else {
    if (DIRICHLET && on_dirichlet(table, N, i, j, k)) {
      ym[p] = xm[p];
      return;
    }
    const int z = zero_mask(N, i, j, k);
    if (__popc(z) == 1) {
      // inside one macro face: the face's own stencil; neighbours outside the macro drop out
      const T* Sf = c.Sface[__ffs(z) - 1];
#pragma unroll
      for (int d = 0; d < 15; ++d) {
        const int pi = i + kStencilD[d][0], pj = j + kStencilD[d][1], pkk = k + kStencilD[d][2];
        if (!inside(N, pi, pj, pkk)) continue;
        if (DIRICHLET && on_dirichlet(table, N, pi, pj, pkk)) continue;
        acc += Sf[d] * __ldg(xm + __ldg(pstart + pkk) + row32(N - pkk, pj) + pi);
      }
    } else {
      // on a macro edge or vertex: sum the incident micro-tets that exist
      acc = p1_face_point<T, DIRICHLET>(c, pstart, xm, i, j, k);
    }
  }
  ym[p] = acc;
}


// Window of row (jr, kr): x at i = i0 - 1 .. i0 + V, zero outside the row and (DIRICHLET) at
// Dirichlet points.
template <typename T, int V, bool DIRICHLET>
__device__ __forceinline__ void p1_window(const T* __restrict__ xm, const int* __restrict__ pstart, int N,
                                          uint32_t table, int i0, int jr, int kr, T w[V + 2]) {
  const int len = N - jr - kr + 1;   // points of the row (none if <= 0)
  if (jr < 0 || kr < 0 || kr > N || len <= 0) {
#pragma unroll
    for (int t = 0; t < V + 2; ++t) w[t] = T(0);
    return;
  }
  const T* __restrict__ row = xm + __ldg(pstart + kr) + row32(N - kr, jr);
  const bool rowface = (jr == 0) | (kr == 0);
  if (!rowface && i0 >= 2 && i0 + V < len - 1) {
    // the window lies inside the row, away from its end points: no bounds, no Dirichlet points
#pragma unroll
    for (int t = 0; t < V + 2; ++t) w[t] = __ldg(row + i0 - 1 + t);
    return;
  }
#pragma unroll
  for (int t = 0; t < V + 2; ++t) {
    const int ii = i0 - 1 + t;
    T v = (ii >= 0 && ii < len) ? __ldg(row + ii) : T(0);
    if (DIRICHLET && (rowface || ii == 0 || ii == len - 1) && ii >= 0 && ii < len &&
        on_dirichlet(table, N, ii, jr, kr))
      v = T(0);
    w[t] = v;
  }
}

// P1 constant-coefficient apply.  A CTA of 8 warps owns 8 rows j (one per warp) of an i-chunk of
// 32*V points (V consecutive points per lane) and climbs the planes k of a k-chunk.  Each lane
// keeps the seven row windows of the 15-point stencil -- rows (j,k), (j+-1,k), (j,k+1),
// (j-1,k+1), (j,k-1), (j+1,k-1) -- in registers and rotates them when k advances, so a step
// loads three new windows.  All 24 micro-tets around a point off the macro faces exist, so its
// row of A is the 15-point stencil folded from the six hoisted class matrices; Dirichlet
// columns were zeroed when the windows were loaded.
template <typename T, int V, bool DIRICHLET>
__global__ void __launch_bounds__(256) p1_stencil_kernel(const OpConst<T>* __restrict__ cst,
                                                          const int4* __restrict__ tasks, int kch,
                                                          const int* __restrict__ pstart, const T* __restrict__ x,
                                                          T* __restrict__ y) {
  const int4 task = tasks[blockIdx.x];
  const OpConst<T>& c = cst[task.w];
  const int N = c.N;
  const uint32_t table = c.bnd_table;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = task.x * 32 * V + V * lane;
  const int j = task.y * kStencilWarps + warp;
  const int k0 = task.z * kch;
  // last plane with a point of this warp's row segment
  const int k_end = min(k0 + kch - 1, N - j - task.x * 32 * V);
  if (k_end < k0) return;
  const T* __restrict__ xm = x + c.base;
  T* __restrict__ ym = y + c.base;
  T S[15];
#pragma unroll
  for (int d = 0; d < 15; ++d) S[d] = c.S[d];
  T w00[V + 2], wp0[V + 2], wm0[V + 2], w01[V + 2], wm1[V + 2], w0m[V + 2], wpm[V + 2];
  p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j, k0, w00);
  p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j + 1, k0, wp0);
  p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j - 1, k0, wm0);
  p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j, k0 + 1, w01);
  p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j - 1, k0 + 1, wm1);
  p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j, k0 - 1, w0m);
  p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j + 1, k0 - 1, wpm);
  for (int k = k0; k <= k_end; ++k) {
    const int len = N - j - k + 1;
    if (i0 < len) {
      const int rowbase = __ldg(pstart + k) + row32(N - k, j);
      if (j >= 1 && k >= 1 && i0 >= 1 && i0 + V <= len - 2) {
        // all V points lie off the macro faces: the interior stencil
#pragma unroll
        for (int v = 0; v < V; ++v)
          ym[rowbase + i0 + v] = S[0] * w00[v + 1] + S[1] * w00[v + 2] + S[2] * w00[v] + S[3] * wp0[v + 1] +
                                 S[4] * wm0[v + 1] + S[5] * w01[v + 1] + S[6] * w0m[v + 1] + S[7] * wm0[v + 2] +
                                 S[8] * wp0[v] + S[9] * w0m[v + 2] + S[10] * w01[v] + S[11] * wpm[v + 1] +
                                 S[12] * wm1[v + 1] + S[13] * wm1[v + 2] + S[14] * wpm[v];
      } else
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int ii = i0 + v;
        if (ii >= len) break;
        T acc;
        const int z = (ii == len - 1) | ((ii == 0) << 1) | ((j == 0) << 2) | ((k == 0) << 3);
        if (DIRICHLET && z && ((table >> z) & 1u)) {
          acc = __ldg(xm + rowbase + ii);
        } else if (__popc(z) <= 1) {
          // inside the macro, or inside one macro face (its own stencil: the missing micro-tets
          // drop out; the neighbours outside the macro read as zero)
          T W[15];
          if (z == 0) {
#pragma unroll
            for (int d = 0; d < 15; ++d) W[d] = S[d];
          } else {
            const T* Sf = c.Sface[__ffs(z) - 1];
#pragma unroll
            for (int d = 0; d < 15; ++d) W[d] = Sf[d];
          }
          acc = W[0] * w00[v + 1] + W[1] * w00[v + 2] + W[2] * w00[v] + W[3] * wp0[v + 1] + W[4] * wm0[v + 1] +
                W[5] * w01[v + 1] + W[6] * w0m[v + 1] + W[7] * wm0[v + 2] + W[8] * wp0[v] + W[9] * w0m[v + 2] +
                W[10] * w01[v] + W[11] * wpm[v + 1] + W[12] * wm1[v + 1] + W[13] * wm1[v + 2] + W[14] * wpm[v];
        } else {
          // on a macro edge or vertex
          acc = p1_face_point<T, DIRICHLET>(c, pstart, xm, ii, j, k);
        }
        ym[rowbase + ii] = acc;
      }
    }
    if (k == k_end) break;
    // rotate: plane k becomes k-1, plane k+1 becomes k; load the three new windows
#pragma unroll
    for (int t = 0; t < V + 2; ++t) {
      w0m[t] = w00[t];
      wpm[t] = wp0[t];
      w00[t] = w01[t];
      wm0[t] = wm1[t];
    }
    p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j + 1, k + 1, wp0);
    p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j, k + 2, w01);
    p1_window<T, V, DIRICHLET>(xm, pstart, N, table, i0, j - 1, k + 2, wm1);
  }
}

// P1 constant-coefficient apply with shared-memory plane tiles.  A CTA owns rows j0..j0+7 and
// points i0..i0+127 of a k-chunk (task list of the stencil kernel).  For every plane it stages
// the tile plus a one-point halo (10 rows x 130 points) into a three-plane rolling buffer --
// one coalesced global load per staged value, Dirichlet points staged as zero -- and each thread
// then evaluates the 15-point stencil of four points (i = i0 + lane + 32 v) from shared memory.
constexpr int kTileI = 32 * kStencilV;           // 128 points along i
constexpr int kTileJ = kStencilWarps;            // 8 rows
constexpr int kTileW = kTileI + 4;               // staged width (130 used, padded)
constexpr int kTileH = kTileJ + 2;               // staged rows

constexpr int kTileDepth = 4;                      // planes staged ahead of the one being computed
constexpr int kTileRing = kTileDepth + 2;          // planes k-1 .. k+kTileDepth

__device__ __forceinline__ void cp_async_zfill(void* smem, const void* gmem, int bytes, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int src = valid ? bytes : 0;   // src-size 0: the destination is zero-filled, nothing is read
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NPENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(NPENDING));
}

// Issue the asynchronous staging of plane kk (tile rows j0-1 .. j0+8, points i0-1 .. i0+128);
// positions outside the macro are zero-filled.
template <typename T>
__device__ __forceinline__ void p1_issue_plane(T (*slot)[kTileW], const T* __restrict__ xm,
                                               const int* __restrict__ pstart, int N, int i0, int j0, int kk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < kTileH; r += kTileJ) {
    const int jr = j0 - 1 + r;
    const int len = N - jr - kk + 1;
    const bool rowok = jr >= 0 && kk >= 0 && kk <= N && len > 0;
    const T* __restrict__ row = rowok ? xm + __ldg(pstart + kk) + row32(N - kk, jr) : xm;
    for (int cidx = lane; cidx < kTileI + 2; cidx += 32) {
      const int ii = i0 - 1 + cidx;
      const bool ok = rowok && ii >= 0 && ii < len;
      cp_async_zfill(&slot[r][cidx], ok ? row + ii : xm, (int)sizeof(T), ok);
    }
  }
}

// After plane kk has arrived: zero the Dirichlet points this thread staged.
template <typename T>
__device__ __forceinline__ void p1_mask_plane(T (*slot)[kTileW], int N, uint32_t table, int i0, int j0, int kk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < kTileH; r += kTileJ) {
    const int jr = j0 - 1 + r;
    const int len = N - jr - kk + 1;
    if (!(jr >= 0 && kk >= 0 && kk <= N && len > 0)) continue;
    const bool rowface = (jr == 0) | (kk == 0);
    for (int cidx = lane; cidx < kTileI + 2; cidx += 32) {
      const int ii = i0 - 1 + cidx;
      if (ii < 0 || ii >= len) continue;
      if ((rowface || ii == 0 || ii == len - 1) && on_dirichlet(table, N, ii, jr, kk)) slot[r][cidx] = T(0);
    }
  }
}

template <typename T, bool DIRICHLET>
__global__ void __launch_bounds__(256) p1_tile_kernel(const OpConst<T>* __restrict__ cst,
                                                       const int4* __restrict__ tasks, int kch,
                                                       const int* __restrict__ pstart, const T* __restrict__ x,
                                                       T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char tile_smem[];
  T (*buf)[kTileH][kTileW] = reinterpret_cast<T (*)[kTileH][kTileW]>(tile_smem);
  const int4 task = tasks[blockIdx.x];
  const OpConst<T>& c = cst[task.w];
  const int N = c.N;
  const uint32_t table = c.bnd_table;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = task.x * kTileI, j0 = task.y * kTileJ, k0 = task.z * kch;
  const int k_end = min(k0 + kch - 1, N - j0 - i0);   // last plane holding a point of the tile
  if (k_end < k0) return;
  const T* __restrict__ xm = x + c.base;
  T* __restrict__ ym = y + c.base;
  T S[15];
#pragma unroll
  for (int d = 0; d < 15; ++d) S[d] = c.S[d];
  const int j = j0 + warp;
  auto slot = [&](int kk) { return buf[(kk - k0 + 1) % kTileRing]; };   // kk >= k0 - 1
  // prologue: planes k0-1 .. k0+kTileDepth-1, one commit group each
  for (int kk = k0 - 1; kk < k0 + kTileDepth; ++kk) {
    if (kk <= k_end + 1) p1_issue_plane<T>(slot(kk), xm, pstart, N, i0, j0, kk);
    cp_async_commit();
  }
  // planes k0-1 and k0 must be complete before the loop (the loop waits for k+1 only)
  cp_async_wait<kTileDepth - 1>();
  if (DIRICHLET) {
    p1_mask_plane<T>(slot(k0 - 1), N, table, i0, j0, k0 - 1);
    p1_mask_plane<T>(slot(k0), N, table, i0, j0, k0);
  }
  for (int k = k0; k <= k_end; ++k) {
    // plane k+1 has arrived once at most kTileDepth-1 later groups are pending
    cp_async_wait<kTileDepth - 2>();
    if (DIRICHLET) p1_mask_plane<T>(slot(k + 1), N, table, i0, j0, k + 1);
    __syncthreads();
    const T (*pm)[kTileW] = slot(k - 1);
    const T (*p0)[kTileW] = slot(k);
    const T (*pp)[kTileW] = slot(k + 1);
    const int len = N - j - k + 1;
    const int r = warp + 1;                     // staged row of j
    if (len > 0) {
      const int rowbase = __ldg(pstart + k) + row32(N - k, j);
#pragma unroll
      for (int v = 0; v < kStencilV; ++v) {
        const int cc = lane + 32 * v + 1;       // staged column of i
        const int ii = i0 + cc - 1;
        if (ii >= len) continue;
        const int z = (ii == len - 1) | ((ii == 0) << 1) | ((j == 0) << 2) | ((k == 0) << 3);
        T acc;
        if (z == 0) {
          acc = S[0] * p0[r][cc] + S[1] * p0[r][cc + 1] + S[2] * p0[r][cc - 1] + S[3] * p0[r + 1][cc] +
                S[4] * p0[r - 1][cc] + S[5] * pp[r][cc] + S[6] * pm[r][cc] + S[7] * p0[r - 1][cc + 1] +
                S[8] * p0[r + 1][cc - 1] + S[9] * pm[r][cc + 1] + S[10] * pp[r][cc - 1] + S[11] * pm[r + 1][cc] +
                S[12] * pp[r - 1][cc] + S[13] * pp[r - 1][cc + 1] + S[14] * pm[r + 1][cc - 1];
        } else if (DIRICHLET && ((table >> z) & 1u)) {
          acc = __ldg(xm + rowbase + ii);
        } else if (__popc(z) == 1) {
          const T* Sf = c.Sface[__ffs(z) - 1];
          acc = Sf[0] * p0[r][cc] + Sf[1] * p0[r][cc + 1] + Sf[2] * p0[r][cc - 1] + Sf[3] * p0[r + 1][cc] +
                Sf[4] * p0[r - 1][cc] + Sf[5] * pp[r][cc] + Sf[6] * pm[r][cc] + Sf[7] * p0[r - 1][cc + 1] +
                Sf[8] * p0[r + 1][cc - 1] + Sf[9] * pm[r][cc + 1] + Sf[10] * pp[r][cc - 1] +
                Sf[11] * pm[r + 1][cc] + Sf[12] * pp[r - 1][cc] + Sf[13] * pp[r - 1][cc + 1] +
                Sf[14] * pm[r + 1][cc - 1];
        } else {
          acc = p1_face_point<T, DIRICHLET>(c, pstart, xm, ii, j, k);
        }
        ym[rowbase + ii] = acc;
      }
    }
    __syncthreads();   // every thread is done with plane k-1: its slot takes plane k+kTileDepth
    const int kn = k + kTileDepth;
    if (kn <= k_end + 1) p1_issue_plane<T>(slot(kn), xm, pstart, N, i0, j0, kn);
    cp_async_commit();
  }
  cp_async_wait<0>();
}

template <typename T>
constexpr size_t p1_tile_smem() {
  return sizeof(T) * kTileRing * kTileH * kTileW;
}

// diag(A) for the constant-coefficient operators: sum of A_T[a][a] over the incident micro-tets.
template <typename T>
__global__ void const_diag_kernel(const OpConst<T>* __restrict__ cst, int degree, bool dirichlet, T* __restrict__ d) {
  const OpConst<T>& c = cst[blockIdx.y];
  const int N = c.N, n = c.n;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= dV(N)) return;
  int i, j, k;
  decode_point(p, N, i, j, k);
  if (dirichlet && on_dirichlet(c.bnd_table, N, i, j, k)) {
    d[c.base + p] = T(1);
    return;
  }
  T acc = T(0);
  const int nloc = degree == 1 ? 4 : 10;
  for (int o = 0; o < 6; ++o) {
    const int lim = n - 1 - (o == 0 ? 0 : (o == 5 ? 2 : 1));
    for (int a = 0; a < nloc; ++a) {
      // lattice point (resolution N) of local node a relative to the cube origin, in units of 1/degree cubes
      int off[3];
      if (a < 4) {
        for (int t = 0; t < 3; ++t) off[t] = degree * kClassOffsetsD[o][a][t];
      } else {
        const int e0 = kP2EdgesD[a - 4][0], e1 = kP2EdgesD[a - 4][1];
        for (int t = 0; t < 3; ++t) off[t] = kClassOffsetsD[o][e0][t] + kClassOffsetsD[o][e1][t];
      }
      const int qi = i - off[0], qj = j - off[1], qk = k - off[2];
      if (qi % degree || qj % degree || qk % degree) continue;
      const int ci = qi / degree, cj = qj / degree, ck = qk / degree;
      if (qi < 0 || qj < 0 || qk < 0 || ci + cj + ck > lim) continue;
      acc += c.A[o][a][a];
    }
  }
  d[c.base + p] = acc;
}

// ---------------------------------------------------------------------------
// Interface reconciliation between macros (on-device replacement of the
// paper's MPI communication of shared macro-primitives).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void iface_sum_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                 const uint8_t* __restrict__ bnd, int64_t ngroups, int per_point, bool dirichlet,
                                 T* __restrict__ y) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  if (dirichlet && bnd[g]) return;    // boundary rows already hold x in every copy
  const int64_t a = ptr[g], b = ptr[g + 1];
  for (int c = 0; c < per_point; ++c) {
    T s = T(0);
    for (int64_t t = a; t < b; ++t) s += y[idx[t] * per_point + c];
    for (int64_t t = a; t < b; ++t) y[idx[t] * per_point + c] = s;
  }
}

template <typename T>
__global__ void iface_copy_owner_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                        int64_t ngroups, int per_point, T* __restrict__ x) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  const int64_t a = ptr[g], b = ptr[g + 1];
  for (int c = 0; c < per_point; ++c) {
    const T v = x[idx[a] * per_point + c];
    for (int64_t t = a + 1; t < b; ++t) x[idx[t] * per_point + c] = v;
  }
}

template <typename T>
int launch_interface_sum(const Interface* itf, T* y, int per_point, bool dirichlet, cudaStream_t s) {
  if (itf->ngroups == 0) return HHG_OK;
  const int th = 128;
  iface_sum_kernel<T><<<(unsigned)((itf->ngroups + th - 1) / th), th, 0, s>>>(itf->d_ptr, itf->d_idx, itf->d_bnd,
                                                                             itf->ngroups, per_point, dirichlet, y);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

template <typename T>
int launch_make_consistent(const Interface* itf, T* x, int per_point, cudaStream_t s) {
  if (itf->ngroups == 0) return HHG_OK;
  const int th = 128;
  iface_copy_owner_kernel<T><<<(unsigned)((itf->ngroups + th - 1) / th), th, 0, s>>>(itf->d_ptr, itf->d_idx,
                                                                                    itf->ngroups, per_point, x);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

// Dot product over distinct points: the sum over all entries minus the non-owner copies.
template <typename T>
__global__ void dot_partial_kernel(const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                   const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                   int64_t ngroups, int per_point, double* __restrict__ partial) {
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    acc += (double)x[t] * (double)y[t];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride)
    for (int64_t t = ptr[g] + 1; t < ptr[g + 1]; ++t)
      for (int c = 0; c < per_point; ++c) {
        const int64_t e = idx[t] * per_point + c;
        acc -= (double)x[e] * (double)y[e];
      }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) acc += partial[t];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

template int launch_interface_sum<double>(const Interface*, double*, int, bool, cudaStream_t);
template int launch_interface_sum<float>(const Interface*, float*, int, bool, cudaStream_t);
template int launch_make_consistent<double>(const Interface*, double*, int, cudaStream_t);
template int launch_make_consistent<float>(const Interface*, float*, int, cudaStream_t);

constexpr int kDotBlocks = 304;   // 2 x 152 SMs

template <typename T>
int launch_dot(const Interface* itf, const T* x, const T* y, int64_t n, int per_point, double* d_scratch,
               cudaStream_t s) {
  dot_partial_kernel<T><<<kDotBlocks, 256, 0, s>>>(x, y, n, itf->d_ptr, itf->d_idx, itf->ngroups, per_point,
                                                   d_scratch + 1);
  sum_partials_kernel<<<1, 256, 0, s>>>(d_scratch + 1, kDotBlocks, d_scratch);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
template <typename T>
const OpConst<T>* dconst(const hhg_op* op);
template <>
const OpConst<double>* dconst<double>(const hhg_op* op) {
  return (const OpConst<double>*)op->d_const64;
}
template <>
const OpConst<float>* dconst<float>(const hhg_op* op) {
  return (const OpConst<float>*)op->d_const32;
}

template <typename T>
const T* field_ptr(const hhg_op* op) {
  return (op->coeff.type == HHG_COEFF_FIELD_P1 || op->coeff.type == HHG_COEFF_FIELD_P2) ? (const T*)op->coeff.field
                                                                                          : nullptr;
}

template <typename T>
int launch_apply(const hhg_op* op, const T* x, T* y, cudaStream_t s) {
  const int64_t V = lattice_size(op->N);
  const int nm = op->mesh->nmacro();
  if (op->kind == HHG_DIFFUSION && op->degree == 1 && op->coeff.type == HHG_COEFF_CONST) {
    (void)V;
    const Interface* I = op->itf;
    if (sizeof(T) == 8) {
      // FP64: the FP64 pipe bounds the apply; one point per thread keeps the most warps in flight
      dim3 grid((unsigned)I->ncta, nm);
      if (op->bc == HHG_DIRICHLET)
        p1_gather_kernel<T, true><<<grid, 256, 0, s>>>(dconst<T>(op), I->d_cta_plane, I->d_cta_start, I->d_pstart,
                                                        x, y);
      else
        p1_gather_kernel<T, false><<<grid, 256, 0, s>>>(dconst<T>(op), I->d_cta_plane, I->d_cta_start,
                                                         I->d_pstart, x, y);
      HHG_CUDA_TRY(cudaGetLastError());
      return HHG_OK;
    }
    const unsigned grid = (unsigned)I->n_stencil_tasks;
    const size_t smem = p1_tile_smem<T>();
    if (op->bc == HHG_DIRICHLET)
      p1_tile_kernel<T, true><<<grid, 256, smem, s>>>(dconst<T>(op), I->d_stencil_tasks, I->stencil_kchunk,
                                                      I->d_pstart, x, y);
    else
      p1_tile_kernel<T, false><<<grid, 256, smem, s>>>(dconst<T>(op), I->d_stencil_tasks, I->stencil_kchunk,
                                                       I->d_pstart, x, y);
    HHG_CUDA_TRY(cudaGetLastError());
    return HHG_OK;
  }
  if (op->kind == HHG_DIFFUSION) return launch_march<T>(op, dconst<T>(op), 0, x, nullptr, field_ptr<T>(op), y, s);
  return fail(HHG_E_UNSUPPORTED, "apply: operator kind %d degree %d coefficient %d not implemented", op->kind,
              op->degree, op->coeff.type);
}

template <typename T>
int launch_diag(const hhg_op* op, T* d, cudaStream_t s) {
  const int64_t V = lattice_size(op->N);
  if (op->kind == HHG_DIFFUSION && op->coeff.type == HHG_COEFF_CONST) {
    dim3 grid((unsigned)((V + 255) / 256), op->mesh->nmacro());
    const_diag_kernel<T><<<grid, 256, 0, s>>>(dconst<T>(op), op->degree, op->bc == HHG_DIRICHLET, d);
    HHG_CUDA_TRY(cudaGetLastError());
    return HHG_OK;
  }
  if (op->kind == HHG_DIFFUSION) return launch_march<T>(op, dconst<T>(op), 1, nullptr, nullptr, field_ptr<T>(op), d, s);
  return fail(HHG_E_UNSUPPORTED, "diagonal: operator not implemented");
}

}  // namespace hhg

using namespace hhg;

hhg_op::~hhg_op() {
  if (mg) hhg::destroy_mg(mg);
  if (work) hhg::destroy_work(work);
  cudaFree(d_const64);
  cudaFree(d_const32);
}

static int check_dtype(int dtype) {
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "dtype must be HHG_F32 or HHG_F64");
  return HHG_OK;
}

static int check_field(const hhg_op* op, int dtype) {
  if (op->coeff.type != HHG_COEFF_FIELD_P1 && op->coeff.type != HHG_COEFF_FIELD_P2) return HHG_OK;
  if (!op->coeff.field) return fail(HHG_E_ARG, "coefficient field pointer is null");
  if (op->coeff.field_dtype != dtype)
    return fail(HHG_E_ARG, "coefficient field dtype %d differs from the apply dtype %d", op->coeff.field_dtype, dtype);
  return HHG_OK;
}

extern "C" int hhg_op_create(hhg_mesh_t* mesh, int level, int kind, int degree, const hhg_coeff_t* coeff, int bc,
                             int quad_degree, hhg_op_t** out) {
  clear_error();
  if (!mesh || !coeff || !out) return fail(HHG_E_ARG, "op_create: null pointer");
  *out = nullptr;
  if (level < 0) level = mesh->level;
  if (level > mesh->level) return fail(HHG_E_ARG, "op_create: level %d above the mesh's %d", level, mesh->level);
  if (kind != HHG_DIFFUSION && kind != HHG_EPSILON) return fail(HHG_E_ARG, "op_create: unknown kind %d", kind);
  if (degree != 1 && degree != 2) return fail(HHG_E_ARG, "op_create: degree must be 1 or 2");
  if (kind == HHG_EPSILON && degree != 2) return fail(HHG_E_ARG, "op_create: EPSILON needs degree 2");
  if (bc != HHG_DIRICHLET && bc != HHG_NEUMANN) return fail(HHG_E_ARG, "op_create: unknown boundary mode %d", bc);
  if (coeff->type < HHG_COEFF_CONST || coeff->type > HHG_COEFF_FIELD_P2)
    return fail(HHG_E_ARG, "op_create: unknown coefficient type %d", coeff->type);
  if ((coeff->type == HHG_COEFF_FIELD_P1 && degree != 1) || (coeff->type == HHG_COEFF_FIELD_P2 && degree != 2))
    return fail(HHG_E_UNSUPPORTED, "op_create: the coefficient field must have the operator's degree");
  if (kind == HHG_EPSILON && coeff->type != HHG_COEFF_CONST && coeff->type != HHG_COEFF_FIELD_P2)
    return fail(HHG_E_UNSUPPORTED, "op_create: EPSILON takes a CONST or FIELD_P2 viscosity");
  if ((coeff->type == HHG_COEFF_SIN3 || coeff->type == HHG_COEFF_FIELD_P2) && quad_degree > 5)
    return fail(HHG_E_UNSUPPORTED, "op_create: quadrature degree above 5");
  std::unique_ptr<hhg_op> op(new hhg_op());
  op->mesh = mesh;
  op->level = level;
  op->kind = kind;
  op->degree = degree;
  op->bc = bc;
  op->quad_degree = quad_degree;
  op->coeff = *coeff;
  op->n = 1 << level;
  op->N = degree << level;
  op->npts = (int64_t)mesh->nmacro() * lattice_size(op->N);
  HHG_TRY(quad_rule(quad_degree, &op->rule));
  const Interface* itf = nullptr;
  HHG_TRY(mesh->interface(level, degree, &itf));
  if (coeff->type == HHG_COEFF_FIELD_P1 || coeff->type == HHG_COEFF_FIELD_P2)
    HHG_TRY(mesh->interface(level, coeff->type == HHG_COEFF_FIELD_P1 ? 1 : 2, &itf));
  build_const(op.get());
  HHG_TRY(mesh->interface(level, degree, &op->itf));
  const int nm = mesh->nmacro();
  std::vector<OpConst<float>> c32(nm);
  for (int m = 0; m < nm; ++m) c32[m] = convert_const<float>(op->h_const[m]);
  HHG_CUDA_TRY(cudaMalloc(&op->d_const64, sizeof(OpConst<double>) * nm));
  HHG_CUDA_TRY(cudaMalloc(&op->d_const32, sizeof(OpConst<float>) * nm));
  HHG_CUDA_TRY(cudaMemcpy(op->d_const64, op->h_const.data(), sizeof(OpConst<double>) * nm, cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(op->d_const32, c32.data(), sizeof(OpConst<float>) * nm, cudaMemcpyHostToDevice));
  *out = op.release();
  return HHG_OK;
}

extern "C" int hhg_op_destroy(hhg_op_t* op) {
  delete op;
  return HHG_OK;
}

extern "C" int hhg_op_set_field(hhg_op_t* op, const void* field, int field_dtype) {
  clear_error();
  if (!op) return fail(HHG_E_ARG, "op_set_field: null op");
  if (op->coeff.type != HHG_COEFF_FIELD_P1 && op->coeff.type != HHG_COEFF_FIELD_P2)
    return fail(HHG_E_ARG, "op_set_field: operator has no coefficient field");
  HHG_TRY(check_dtype(field_dtype));
  op->coeff.field = field;
  op->coeff.field_dtype = field_dtype;
  return HHG_OK;
}

extern "C" int hhg_op_apply(hhg_op_t* op, const void* x, void* y, int dtype, int nrhs, void* stream) {
  clear_error();
  if (!op || !x || !y) return fail(HHG_E_ARG, "op_apply: null pointer");
  HHG_TRY(check_dtype(dtype));
  if (nrhs < 1 || (nrhs > 1 && op->kind != HHG_EPSILON)) return fail(HHG_E_ARG, "op_apply: bad nrhs %d", nrhs);
  if (x == y) return fail(HHG_E_ARG, "op_apply: x and y must not overlap");
  HHG_TRY(check_field(op, dtype));
  cudaStream_t s = (cudaStream_t)stream;
  const Interface* itf = nullptr;
  HHG_TRY(op->mesh->interface(op->level, op->degree, &itf));
  if (op->kind == HHG_EPSILON) {
    const int pp = 3 * nrhs;
    if (dtype == HHG_F64) {
      HHG_TRY(launch_eps<double>(op, dconst<double>(op), 0, nrhs, (const double*)x, nullptr, field_ptr<double>(op),
                                 (double*)y, s));
      HHG_TRY(launch_interface_sum<double>(itf, (double*)y, pp, op->bc == HHG_DIRICHLET, s));
    } else {
      HHG_TRY(launch_eps<float>(op, dconst<float>(op), 0, nrhs, (const float*)x, nullptr, field_ptr<float>(op),
                                (float*)y, s));
      HHG_TRY(launch_interface_sum<float>(itf, (float*)y, pp, op->bc == HHG_DIRICHLET, s));
    }
    return HHG_OK;
  }
  if (dtype == HHG_F64) {
    HHG_TRY(launch_apply<double>(op, (const double*)x, (double*)y, s));
    HHG_TRY(launch_interface_sum<double>(itf, (double*)y, 1, op->bc == HHG_DIRICHLET, s));
  } else {
    HHG_TRY(launch_apply<float>(op, (const float*)x, (float*)y, s));
    HHG_TRY(launch_interface_sum<float>(itf, (float*)y, 1, op->bc == HHG_DIRICHLET, s));
  }
  return HHG_OK;
}

extern "C" int hhg_op_diagonal(hhg_op_t* op, void* d, int dtype, void* stream) {
  clear_error();
  if (!op || !d) return fail(HHG_E_ARG, "op_diagonal: null pointer");
  HHG_TRY(check_dtype(dtype));
  if (op->kind != HHG_DIFFUSION) return fail(HHG_E_UNSUPPORTED, "op_diagonal: scalar operators only");
  HHG_TRY(check_field(op, dtype));
  cudaStream_t s = (cudaStream_t)stream;
  const Interface* itf = nullptr;
  HHG_TRY(op->mesh->interface(op->level, op->degree, &itf));
  if (dtype == HHG_F64) {
    HHG_TRY(launch_diag<double>(op, (double*)d, s));
    HHG_TRY(launch_interface_sum<double>(itf, (double*)d, 1, op->bc == HHG_DIRICHLET, s));
  } else {
    HHG_TRY(launch_diag<float>(op, (float*)d, s));
    HHG_TRY(launch_interface_sum<float>(itf, (float*)d, 1, op->bc == HHG_DIRICHLET, s));
  }
  return HHG_OK;
}

namespace hhg {
// Physical position of every packed point: P0 + (i e0 + j e1 + k e2) / N.
__global__ void coordinates_kernel(const MacroGeom* __restrict__ mg, int N, const int* __restrict__ cta_plane,
                                   const int* __restrict__ cta_start, const int* __restrict__ pstart,
                                   double* __restrict__ xyz) {
  const int k = __ldg(cta_plane + blockIdx.x);
  const int s = N - k;
  const int q = (blockIdx.x - __ldg(cta_start + k)) * 256 + threadIdx.x;
  if (q >= tri(s)) return;
  const float b = 2.0f * s + 3.0f;
  int j = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)q, 0.0f))));
  j = max(0, min(j, s));
  if (j < s && row32(s, j + 1) <= q) ++j;
  if (j > 0 && row32(s, j) > q) --j;
  const int i = q - row32(s, j);
  const MacroGeom& g = mg[blockIdx.y];
  const int64_t e = (int64_t)blockIdx.y * dV(N) + __ldg(pstart + k) + q;
  for (int d = 0; d < 3; ++d)
    xyz[3 * e + d] = g.p0[d] + ((double)i * g.e[0][d] + (double)j * g.e[1][d] + (double)k * g.e[2][d]) / N;
}
}  // namespace hhg

extern "C" int hhg_vec_coordinates(const hhg_mesh_t* mesh, int level, int degree, double* xyz, void* stream) {
  clear_error();
  if (!mesh || !xyz) return fail(HHG_E_ARG, "vec_coordinates: null pointer");
  const Interface* itf = nullptr;
  HHG_TRY(const_cast<hhg_mesh_t*>(mesh)->interface(level, degree, &itf));
  dim3 grid((unsigned)itf->ncta, mesh->nmacro());
  coordinates_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(mesh->d_macros, degree << level, itf->d_cta_plane,
                                                             itf->d_cta_start, itf->d_pstart, xyz);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

extern "C" int hhg_vec_make_consistent(const hhg_mesh_t* mesh, int level, int degree, void* x, int dtype,
                                       int n_per_point, void* stream) {
  clear_error();
  if (!mesh || !x || n_per_point < 1) return fail(HHG_E_ARG, "vec_make_consistent: bad argument");
  HHG_TRY(check_dtype(dtype));
  const Interface* itf = nullptr;
  HHG_TRY(const_cast<hhg_mesh_t*>(mesh)->interface(level, degree, &itf));
  if (dtype == HHG_F64) return launch_make_consistent<double>(itf, (double*)x, n_per_point, (cudaStream_t)stream);
  return launch_make_consistent<float>(itf, (float*)x, n_per_point, (cudaStream_t)stream);
}

extern "C" int hhg_vec_dot(const hhg_mesh_t* mesh, int level, int degree, const void* x, const void* y, int dtype,
                           int n_per_point, double* result, void* stream) {
  clear_error();
  if (!mesh || !x || !y || !result || n_per_point < 1) return fail(HHG_E_ARG, "vec_dot: bad argument");
  HHG_TRY(check_dtype(dtype));
  const Interface* itf = nullptr;
  hhg_mesh_t* m = const_cast<hhg_mesh_t*>(mesh);
  HHG_TRY(m->interface(level, degree, &itf));
  HHG_TRY(m->scratch_reserve((kDotBlocks + 1) * sizeof(double)));
  const int64_t n = (int64_t)m->nmacro() * lattice_size((int64_t)degree << level) * n_per_point;
  cudaStream_t s = (cudaStream_t)stream;
  double* d = (double*)m->d_scratch;
  if (dtype == HHG_F64)
    HHG_TRY(launch_dot<double>(itf, (const double*)x, (const double*)y, n, n_per_point, d, s));
  else
    HHG_TRY(launch_dot<float>(itf, (const float*)x, (const float*)y, n, n_per_point, d, s));
  HHG_CUDA_TRY(cudaMemcpyAsync(result, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  HHG_CUDA_TRY(cudaStreamSynchronize(s));
  return HHG_OK;
}

extern "C" int hhg_op_apply_adjoint_coeff(hhg_op_t* op, const void* u, const void* g, void* dk, int dtype, int nrhs,
                                          void* stream) {
  clear_error();
  if (!op || !u || !g || !dk) return fail(HHG_E_ARG, "op_apply_adjoint_coeff: null pointer");
  HHG_TRY(check_dtype(dtype));
  if (op->coeff.type != HHG_COEFF_FIELD_P1 && op->coeff.type != HHG_COEFF_FIELD_P2)
    return fail(HHG_E_UNSUPPORTED, "op_apply_adjoint_coeff: the coefficient is not a field");
  if (nrhs < 1 || (nrhs != 1 && op->kind != HHG_EPSILON))
    return fail(HHG_E_ARG, "op_apply_adjoint_coeff: nrhs must be 1 for scalar operators");
  HHG_TRY(check_field(op, dtype));
  cudaStream_t s = (cudaStream_t)stream;
  const Interface* itf = nullptr;
  HHG_TRY(op->mesh->interface(op->level, op->degree, &itf));
  if (op->kind == HHG_EPSILON) {
    if (dtype == HHG_F64) {
      HHG_TRY(launch_eps<double>(op, dconst<double>(op), 2, nrhs, (const double*)u, (const double*)g,
                                 field_ptr<double>(op), (double*)dk, s));
      HHG_TRY(launch_interface_sum<double>(itf, (double*)dk, 1, false, s));
    } else {
      HHG_TRY(launch_eps<float>(op, dconst<float>(op), 2, nrhs, (const float*)u, (const float*)g,
                                field_ptr<float>(op), (float*)dk, s));
      HHG_TRY(launch_interface_sum<float>(itf, (float*)dk, 1, false, s));
    }
    return HHG_OK;
  }
  if (dtype == HHG_F64) {
    HHG_TRY(launch_march<double>(op, dconst<double>(op), 2, (const double*)u, (const double*)g,
                                 field_ptr<double>(op), (double*)dk, s));
    HHG_TRY(launch_interface_sum<double>(itf, (double*)dk, 1, false, s));
  } else {
    HHG_TRY(launch_march<float>(op, dconst<float>(op), 2, (const float*)u, (const float*)g, field_ptr<float>(op),
                                (float*)dk, s));
    HHG_TRY(launch_interface_sum<float>(itf, (float*)dk, 1, false, s));
  }
  return HHG_OK;
}
