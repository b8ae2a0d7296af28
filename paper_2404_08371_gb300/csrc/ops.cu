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
#include <array>
#include <tuple>
#include <type_traits>
#include <utility>
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
        c.lam4[q][a] = 4.0 * lam[a];
        c.lam4m1[q][a] = 4.0 * lam[a] - 1.0;
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
        // the first coordinate's entries carry the point's factor of the analytic coefficient:
        // P1 element mean k_T = 1 + sum_q 3 w_q prod_d sin(2 pi x_d) (sum_q w_q = 1/6), P2 point
        // weight w_q k_q = w_q + 0.5 w_q prod_d sin(2 pi x_d)
        const double fq = op->degree == 1 ? 3.0 * rq.w[q] : 0.5 * rq.w[q];
        for (int d = 0; d < 3; ++d) {
          double delta = 0;
          for (int a = 0; a < 3; ++a) delta += c.h[a][d] * ref[a];
          const double f = d == 0 ? fq : 1.0;
          c.cs[o][q][d][0] = f * std::cos(2.0 * M_PI * delta);
          c.cs[o][q][d][1] = f * std::sin(2.0 * M_PI * delta);
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
    for (int a = 0; a < 4; ++a) {
      o.lam[q][a] = (T)c.lam[q][a];
      o.lam4[q][a] = (T)c.lam4[q][a];
      o.lam4m1[q][a] = (T)c.lam4m1[q][a];
    }
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

// Row of a P1 point on a macro face: Dirichlet points keep x; a point inside one face uses that
// face's stencil (neighbours outside the macro drop out); a point on a macro edge or vertex sums its
// incident micro-tets that exist.
template <typename T, bool DIRICHLET>
__device__ __forceinline__ T p1_face_value(const OpConst<T>& c, const int* __restrict__ pstart, const T* __restrict__ xm,
                                           int i, int j, int k) {
  const int N = c.N;
  const uint32_t table = c.bnd_table;
  if (DIRICHLET && on_dirichlet(table, N, i, j, k)) return xm[__ldg(pstart + k) + row32(N - k, j) + i];
  const int z = zero_mask(N, i, j, k);
  if (__popc(z) != 1) return p1_face_point<T, DIRICHLET>(c, pstart, xm, i, j, k);
  const T* Sf = c.Sface[__ffs(z) - 1];
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < 15; ++d) {
    const int pi = i + kStencilD[d][0], pj = j + kStencilD[d][1], pkk = k + kStencilD[d][2];
    if (!inside(N, pi, pj, pkk)) continue;
    if (DIRICHLET && on_dirichlet(table, N, pi, pj, pkk)) continue;
    acc += Sf[d] * __ldg(xm + __ldg(pstart + pkk) + row32(N - pkk, pj) + pi);
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
    acc = p1_face_value<T, DIRICHLET>(c, pstart, xm, i, j, k);
  }
  ym[p] = acc;
}

// ---------------------------------------------------------------------------
// P1 constant-coefficient apply of FP64 vectors in double-float arithmetic.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the FP64 stencil above is bound by the FP64 pipe
// (15 DFMA per point).  Here every FP64 value v is carried as an unevaluated sum hi + lo of two
// FP32 numbers (hi = v rounded to FP32, lo = the rounded remainder: 48 significant bits), and the
// stencil sum_d S_d x_d is formed in FP32 arithmetic: the product of the high parts exactly by an
// FMA (Dekker's product), the cross terms by FMA, the high parts summed by Knuth's two-sum, the low
// parts summed apart.  The relative error of a row is a few units of 2^-48 (about 1e-14), far
// inside the 1e-12 of an FP64 apply; x is split once per apply by a streaming pass.
// ---------------------------------------------------------------------------
// FP64 v -> (hi, lo) from its bit fields with integer operations (the FP64 pipe, 1/64 of the FP32
// rate on GB300, would bound conversions): hi = v truncated to 24 significant bits, lo = the
// remaining 29 bits converted to FP32 and scaled.  Zero and subnormal v give (0, 0); values outside
// the exponent range that FP32 pairs represent exactly (|v| >= 2^127 or |v| < 2^-74) take the
// FP64 conversion.
__device__ __forceinline__ float2 split_double_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned uh = (unsigned)(u >> 32), ul = (unsigned)u;
  const int e = (int)((uh >> 20) & 0x7ffu);
  if (e == 0) return make_float2(0.0f, 0.0f);
  if (e < 949 || e > 1150) {
    const float hi = __double2float_rz(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
  }
  const unsigned sign = uh & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((uh & 0xfffffu) << 3) | (ul >> 29));
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);   // 2^(e - 1075)
  const float lo = __uint2float_rn(ul & 0x1fffffffu) * scale;
  return make_float2(hi, sign ? -lo : lo);
}

// FP32 -> FP64 from the bit fields (exact; subnormal FP32 values read as zero)
__device__ __forceinline__ double float_to_double_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned fe = (b >> 23) & 0xffu;
  if (fe == 0) return 0.0;
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(fe + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

__global__ void split_double_kernel(int64_t n, const double* __restrict__ x, float2* __restrict__ xs) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) xs[t] = split_double_bits(x[t]);
}

// acc += w * v for double-float w, v; acc.x the high sum, acc.y the low parts and rounding errors
// (explicitly rounded operations: a product or sum fused into an FMA by the compiler would break
// the exactness the two-sum and the product error rely on)
__device__ __forceinline__ void df_fma(float2& acc, float2 w, float2 v) {
  const float ph = __fmul_rn(w.x, v.x);
  float pl = fmaf(w.x, v.x, -ph);        // exact low part of w.hi v.hi
  pl = fmaf(w.x, v.y, pl);
  pl = fmaf(w.y, v.x, pl);
  const float sh = __fadd_rn(acc.x, ph);   // two-sum of the high parts
  const float bb = __fsub_rn(sh, acc.x);
  const float e = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(sh, bb)), __fsub_rn(ph, bb));
  acc.x = sh;
  acc.y += pl + e;
}

template <bool DIRICHLET>
__global__ void __launch_bounds__(256) p1_gather_df_kernel(const OpConst<double>* __restrict__ cst,
                                                            const float2* __restrict__ wdf,
                                                            const int* __restrict__ cta_plane,
                                                            const int* __restrict__ cta_start,
                                                            const int* __restrict__ pstart,
                                                            const double* __restrict__ x,
                                                            const float2* __restrict__ xs, double* __restrict__ y) {
  const OpConst<double>& c = cst[blockIdx.y];
  const int N = c.N;
  const int k = __ldg(cta_plane + blockIdx.x);
  const int s = N - k;
  const int q = (blockIdx.x - __ldg(cta_start + k)) * 256 + threadIdx.x;
  if (q >= tri(s)) return;
  const float bq = 2.0f * s + 3.0f;
  int j = (int)(0.5f * (bq - sqrtf(fmaxf(bq * bq - 8.0f * (float)q, 0.0f))));
  j = max(0, min(j, s));
  if (j < s && row32(s, j + 1) <= q) ++j;
  if (j > 0 && row32(s, j) > q) --j;
  const int i = q - row32(s, j);
  const int pk = __ldg(pstart + k);
  const int p = pk + q;
  const double* __restrict__ xm = x + c.base;
  const float2* __restrict__ xsm = xs + c.base;
  double* __restrict__ ym = y + c.base;
  const bool on_face = (i == 0) | (j == 0) | (k == 0) | (i + j + k == N);
  if (on_face) {
    ym[p] = p1_face_value<double, DIRICHLET>(c, pstart, xm, i, j, k);
    return;
  }
  const int r00 = p - i;                                 // (j, k)
  const int rp0 = r00 + (s + 1 - j);                     // (j+1, k)
  const int rm0 = r00 - (s + 2 - j);                     // (j-1, k)
  const int pk1 = pk + tri(s);
  const int r01 = pk1 + row32(s - 1, j);                 // (j, k+1)
  const int rm1 = pk1 + row32(s - 1, j - 1);             // (j-1, k+1)
  const int pkm = pk - tri(s + 1);
  const int r0m = pkm + row32(s + 1, j);                 // (j, k-1)
  const int rpm = pkm + row32(s + 1, j + 1);             // (j+1, k-1)
  const int at[15] = {r00 + i,     r00 + i + 1, r00 + i - 1, rp0 + i,     rm0 + i,
                      r01 + i,     r0m + i,     rm0 + i + 1, rp0 + i - 1, r0m + i + 1,
                      r01 + i - 1, rpm + i,     rm1 + i,     rm1 + i + 1, rpm + i - 1};
  const float2* __restrict__ w = wdf + 16 * blockIdx.y;
  const bool near = DIRICHLET && !(i >= 2 && j >= 2 && k >= 2 && i + j + k <= N - 2);
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int d = 0; d < 15; ++d) {
    float2 v = __ldg(xsm + at[d]);
    // a neighbour on a Dirichlet face: its column is dropped
    if (near && on_dirichlet(c.bnd_table, N, i + kStencilD[d][0], j + kStencilD[d][1], k + kStencilD[d][2]))
      v = make_float2(0.0f, 0.0f);
    df_fma(acc, __ldg(w + d), v);
  }
  ym[p] = float_to_double_bits(acc.x) + float_to_double_bits(acc.y);
}

// The register-climbing P1 FP32 kernel (p1_climb_f32_kernel) stops below the top kP1ClimbTop - 1
// planes, where rows are too short for its unchecked windows; p1_face_slice writes those points.
constexpr int kP1ClimbTop = 10;

// Point off the macro faces: the 15-point stencil with the Dirichlet columns dropped.
template <typename T, bool DIRICHLET>
__device__ __forceinline__ T p1_interior_value(const OpConst<T>& c, const int* __restrict__ pstart,
                                               const T* __restrict__ xm, int i, int j, int k) {
  const int N = c.N;
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < 15; ++d) {
    const int pi = i + kStencilD[d][0], pj = j + kStencilD[d][1], pkk = k + kStencilD[d][2];
    if (DIRICHLET && on_dirichlet(c.bnd_table, N, pi, pj, pkk)) continue;
    acc += c.S[d] * __ldg(xm + __ldg(pstart + pkk) + row32(N - pkk, pj) + pi);
  }
  return acc;
}

// Points of the P1 FP32 apply that the climbing part of p1_climb_f32_kernel does not write, one
// thread each (thread t of slice f).  Slices
// 0-3: face a of the macro, the points (a, b) with a + b <= N of its triangle (a point on several
// faces is written by the lowest).  Slices 4 and 5: the points off the faces in row j = 1 and in
// plane k = 1.  Slice 6: the points off the faces with j >= 2 on the top planes k > N - kP1ClimbTop
// (all planes k >= 2 when N < kP1ClimbTop + 2).
template <typename T, bool DIRICHLET>
__device__ __forceinline__ void p1_face_slice(const OpConst<T>& c, const int* __restrict__ pstart,
                                              const T* __restrict__ x, T* __restrict__ y, int f, int t) {
  const int N = c.N;
  int i, j, k;
  if (f <= 5) {
    if (t >= tri(N)) return;
    const float bq = 2.0f * N + 3.0f;
    int b = (int)(0.5f * (bq - sqrtf(fmaxf(bq * bq - 8.0f * (float)t, 0.0f))));
    b = max(0, min(b, N));
    if (b < N && row32(N, b + 1) <= t) ++b;
    if (b > 0 && row32(N, b) > t) --b;
    const int a = t - row32(N, b);
    if (f == 0) {
      i = 0; j = a; k = b;
    } else if (f == 1) {
      i = a; j = 0; k = b;
    } else if (f == 2) {
      i = a; j = b; k = 0;
    } else if (f == 3) {
      i = N - a - b; j = a; k = b;
    } else if (f == 4) {
      i = a; j = 1; k = b;
    } else {
      i = a; j = b; k = 1;
    }
  } else {
    // lattice of the top planes k >= kt (at most V(kP1ClimbTop - 1) points), plane by plane
    const int kt = max(2, N - kP1ClimbTop + 1);
    const int m = N - kt;
    if (m < 0 || t >= (m + 1) * (m + 2) * (m + 3) / 6) return;
    int rem = t, kk = 0;
    while (rem >= tri(m - kk)) rem -= tri(m - kk++);
    int jj = 0;
    while (rem >= m - kk - jj + 1) rem -= m - kk - jj++ + 1;
    i = rem; j = jj; k = kt + kk;
  }
  const T* __restrict__ xm = x + c.base;
  if (f <= 3) {
    if ((f >= 1 && i == 0) || (f >= 2 && j == 0) || (f == 3 && k == 0)) return;
    y[c.base + __ldg(pstart + k) + row32(N - k, j) + i] = p1_face_value<T, DIRICHLET>(c, pstart, xm, i, j, k);
    return;
  }
  const bool off_faces = i >= 1 && j >= 1 && k >= 1 && i + j + k <= N - 1;
  if (!off_faces || (f >= 5 && j < 2)) return;
  y[c.base + __ldg(pstart + k) + row32(N - k, j) + i] = p1_interior_value<T, DIRICHLET>(c, pstart, xm, i, j, k);
}


// Structural P2 stencil lists, rebuilt at compile time in the order of the host table (ascending
// packed offset = by dz, then dy, then dx), so that interior rows unroll with constant offsets.
__host__ __device__ constexpr int p2c_off(int o, int v, int d) {
  constexpr int t[6][4][3] = {
      {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {1, 1, 0}},
      {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {0, 1, 1}}, {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {0, 0, 1}},
      {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {1, 0, 0}}, {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}}};
  return t[o][v][d];
}
__host__ __device__ constexpr int p2c_node(int o, int a, int d) {
  constexpr int e[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  return a < 4 ? 2 * p2c_off(o, a, d) : p2c_off(o, e[a - 4][0], d) + p2c_off(o, e[a - 4][1], d);
}
struct P2OffList {
  int n;
  int off[65];
};
__host__ __device__ constexpr P2OffList p2_struct_list(int par) {
  P2OffList L{};
  for (int o = 0; o < 6; ++o)
    for (int a = 0; a < 10; ++a) {
      const int pa = (p2c_node(o, a, 0) & 1) | ((p2c_node(o, a, 1) & 1) << 1) | ((p2c_node(o, a, 2) & 1) << 2);
      if (pa != par) continue;
      for (int b = 0; b < 10; ++b) {
        const int v = (p2c_node(o, b, 0) - p2c_node(o, a, 0) + 2) | ((p2c_node(o, b, 1) - p2c_node(o, a, 1) + 2) << 4) |
                      ((p2c_node(o, b, 2) - p2c_node(o, a, 2) + 2) << 8);
        int pos = 0;
        while (pos < L.n && L.off[pos] < v) ++pos;
        if (pos < L.n && L.off[pos] == v) continue;
        for (int t = L.n; t > pos; --t) L.off[t] = L.off[t - 1];
        L.off[pos] = v;
        ++L.n;
      }
    }
  return L;
}
template <int PAR>
struct P2Cnt {
  static constexpr int v = p2_struct_list(PAR).n;
};
template <int PAR>
struct P2Start {
  static constexpr int v = P2Start<PAR - 1>::v + P2Cnt<PAR - 1>::v;
};
template <>
struct P2Start<0> {
  static constexpr int v = 0;
};
template <int PAR, int D>
struct P2Off {
  static constexpr int v = p2_struct_list(PAR).off[D];
};
static_assert(P2Start<7>::v + P2Cnt<7>::v == kP2StTotal, "P2 structural stencil size");

// The two points of a lane (even i of parity PA, odd i + 1 of parity PA | 1) share most staged
// cells: the union of their neighbours, as offsets from the even point, with the entry of each
// stencil that uses the cell (-1: not used), lets each cell be loaded once.
struct P2UnionList {
  int n;
  int off[65];
  int ia[65];
  int ib[65];
};
__host__ __device__ constexpr P2UnionList p2_union_list(int pa) {
  P2UnionList U{};
  const P2OffList A = p2_struct_list(pa), B = p2_struct_list(pa | 1);
  for (int s = 0; s < 2; ++s) {
    const P2OffList& L = s == 0 ? A : B;
    for (int d = 0; d < L.n; ++d) {
      const int v = L.off[d] + s;   // dx + 1 for the odd point
      int pos = 0;
      while (pos < U.n && U.off[pos] < v) ++pos;
      if (!(pos < U.n && U.off[pos] == v)) {
        for (int t = U.n; t > pos; --t) {
          U.off[t] = U.off[t - 1];
          U.ia[t] = U.ia[t - 1];
          U.ib[t] = U.ib[t - 1];
        }
        U.off[pos] = v;
        U.ia[pos] = -1;
        U.ib[pos] = -1;
        ++U.n;
      }
      (s == 0 ? U.ia[pos] : U.ib[pos]) = d;
    }
  }
  return U;
}
template <int PA>
struct P2UCnt {
  static constexpr int v = p2_union_list(PA).n;
};
template <int PA, int C>
struct P2UCell {
  static constexpr int off = p2_union_list(PA).off[C];
  static constexpr int ia = p2_union_list(PA).ia[C];
  static constexpr int ib = p2_union_list(PA).ib[C];
};

// cp.async helpers of the plane-tile kernels.
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


// P1 constant-coefficient apply in FP32 with the planes carried in registers.  A CTA takes a tile
// task (rows j0..j0+7, points i0..i0+32 PT-1 of a k-chunk); warp w owns row j = j0 + w and the
// points i = i0 + lane + 32 t (t < PT) and climbs k.  The 15-point stencil of row (j, k) reads seven
// rows: (j, k) at i-1, i, i+1; (j+1, k) and (j+1, k-1) at i-1, i; (j-1, k) and (j-1, k+1) at i,
// i+1; (j, k+1) at i-1, i; (j, k-1) at i, i+1.  A row j' = j+1 serves the warp in two consecutive
// steps, a row j' = j in three and a row j' = j-1 in two, so each step reads three new rows from
// global memory (through L1, where the warps of rows j-1 and j+1 find them again): (j+1, k+1),
// (j-1, k+2), (j, k+2), one step before they are needed.  The rows live in register rings of
// 3, 4 and 3 slots; the k loop is unrolled by 12, the least common multiple, so that every slot
// index is a compile-time constant.  No shared memory, no barriers.
//
// The kernel writes the points with 1 <= i <= N-j-k-1, j >= 2 and 2 <= k <= N - kP1ClimbTop; the
// other points off the macro faces (rows j = 1, planes k = 1 and the top planes) and the face points
// are written by p1_face_slice.  Every row it reads then exists, and a row is read without bounds
// checks: positions before its first or after its last point fall inside the macro's array (on
// these planes at least V(8) = 165 points follow every row, more than a window reaches past it) and
// feed only points that are not written.  With rows j, k >= 2 the only neighbours on a macro face are
// the points i = 0 (face i = 0, for the point i = 1) and the points on the face i + j + k = N (for
// the point i = N-j-k-1), each lying on that face alone; their four terms are summed apart and
// dropped when the face is Dirichlet.

template <int SLO, int SHI, int PT>
__device__ __forceinline__ void p1_climb_row(float (&v)[SHI - SLO + 1][PT], const float* __restrict__ at) {
#pragma unroll
  for (int s = SLO; s <= SHI; ++s)
#pragma unroll
    for (int t = 0; t < PT; ++t) v[s - SLO][t] = __ldg(at + 32 * t + s);
}

// The loads of a row are issued one step before its first use, which alone does not cover the
// DRAM latency: the three rows that step k + kClimbAhead loads are prefetched into L2 at step k
// (0 or 1: no prefetch).  The window [ib-1, ib+32 PT] spans at most PT + 2 lines of 32 floats;
// lane l <= PT + 1 touches the line at offset min(32 l, 32 PT + 1).
constexpr int kClimbAhead = 2;

__device__ __forceinline__ void p1_climb_prefetch(const float* a) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// points per lane of the climbing kernel (its tile tasks are 32 * kClimbPT points wide)
constexpr int kClimbPT = 2;

template <int PT>
struct P1Climb {
  float P[3][2][PT];   // rows j+1 at i-1, i
  float Z[4][3][PT];   // rows j at i-1, i, i+1
  float M[3][2][PT];   // rows j-1 at i, i+1
  // running offsets (from point ib + lane of the macro) of the rows loaded next, (j+1, k+1),
  // (j-1, k+2), (j, k+2), of the same rows kClimbAhead planes higher (prefetch, at the lane's line
  // offset), and of y at (j, k); a row advances by start(jr, kr + 1) = start(jr, kr) + tri(N - kr) - jr
  int ap, am, az, fp, fm, fz, ay;
  int t0;              // tri(N - k)
  int ta;              // tri(N - k - kClimbAhead)
};

// Step U (mod 12) of the climb: row (j, k).  Slots: row j+1 of plane k in P[(U+1)%3], row j of
// plane k in Z[(U+1)%4], row j-1 of plane k in M[U%3].
template <int U, int PT, bool DIRICHLET>
__device__ __forceinline__ void p1_climb_step(P1Climb<PT>& R, const float (&S)[15], const float* __restrict__ xb,
                                              float* __restrict__ yb, int N, bool dir_i0, bool dir_diag, int ib,
                                              int j, int k, int ke) {
  constexpr int pm = U % 3, p0 = (U + 1) % 3, pn = (U + 2) % 3;
  constexpr int zm = U % 4, z0 = (U + 1) % 4, zp = (U + 2) % 4, zn = (U + 3) % 4;
  constexpr int m0 = U % 3, mp = (U + 1) % 3, mn = (U + 2) % 3;
  const int lane = threadIdx.x & 31;
  if (k < ke) {
    p1_climb_row<-1, 0, PT>(R.P[pn], xb + R.ap);
    p1_climb_row<0, 1, PT>(R.M[mn], xb + R.am);
    p1_climb_row<-1, 1, PT>(R.Z[zn], xb + R.az);
  }
  if (kClimbAhead > 1 && k + kClimbAhead < ke && lane <= PT + 1) {   // rows of step k + kClimbAhead
    p1_climb_prefetch(xb + R.fp);
    p1_climb_prefetch(xb + R.fm);
    p1_climb_prefetch(xb + R.fz);
  }
  const int len = N - j - k + 1;
  float mid[PT], lft[PT], rgt[PT];
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    float a = S[0] * R.Z[z0][1][t];
    a = fmaf(S[4], R.M[m0][0][t], a);     // ( 0,-1, 0)
    a = fmaf(S[7], R.M[m0][1][t], a);     // ( 1,-1, 0)
    a = fmaf(S[6], R.Z[zm][1][t], a);     // ( 0, 0,-1)
    a = fmaf(S[9], R.Z[zm][2][t], a);     // ( 1, 0,-1)
    a = fmaf(S[11], R.P[pm][1][t], a);    // ( 0, 1,-1)
    a = fmaf(S[12], R.M[mp][0][t], a);    // ( 0,-1, 1)
    mid[t] = a;
    // neighbours with i-1 (on face i = 0 for the point i = 1)
    float l = S[2] * R.Z[z0][0][t];       // (-1, 0, 0)
    l = fmaf(S[8], R.P[p0][0][t], l);     // (-1, 1, 0)
    l = fmaf(S[10], R.Z[zp][0][t], l);    // (-1, 0, 1)
    l = fmaf(S[14], R.P[pm][0][t], l);    // (-1, 1,-1)
    lft[t] = l;
    // neighbours one step nearer the face i + j + k = N (on it for the point i = N-j-k-1)
    float r = S[1] * R.Z[z0][2][t];       // ( 1, 0, 0)
    r = fmaf(S[3], R.P[p0][1][t], r);     // ( 0, 1, 0)
    r = fmaf(S[5], R.Z[zp][1][t], r);     // ( 0, 0, 1)
    r = fmaf(S[13], R.M[mp][1][t], r);    // ( 1,-1, 1)
    rgt[t] = r;
  }
  if (DIRICHLET) {
    if (dir_i0 && ib == 0 && lane == 1) lft[0] = 0.0f;
    const int q = len - 2 - ib;           // the point i = N-j-k-1, relative to the window
    if (dir_diag && q >= 0 && q < 32 * PT) {
#pragma unroll
      for (int t = 0; t < PT; ++t)
        if (lane + 32 * t == q) rgt[t] = 0.0f;
    }
  }
  const int lo = 1 - ib - lane, hi = len - 2 - ib - lane;   // 32 t in [lo, hi]: a point to write
#pragma unroll
  for (int t = 0; t < PT; ++t)
    if (32 * t >= lo && 32 * t <= hi) yb[R.ay + 32 * t] = mid[t] + lft[t] + rgt[t];
  // next plane
  const int s = N - k;
  const int t1 = R.t0 - (s + 1), t2 = t1 - s;   // tri(s - 1), tri(s - 2)
  R.ay += R.t0 - j;
  R.ap += t1 - (j + 1);
  R.am += t2 - (j - 1);
  R.az += t2 - j;
  R.t0 = t1;
  if (kClimbAhead > 1) {
    const int sa = s - kClimbAhead;
    const int a1 = R.ta - (sa + 1), a2 = a1 - sa;
    R.fp += a1 - (j + 1);
    R.fm += a2 - (j - 1);
    R.fz += a2 - j;
    R.ta = a1;
  }
}

// One launch does both parts: blocks below ntasks climb (tile tasks, heaviest first), the blocks after
// them write the other points (p1_face_slice: per macro, slices 0-5 of nfb blocks each and one block
// for the top planes), so that those fill the SMs that the last climbing tasks leave idle.
template <int PT, bool DIRICHLET>
__global__ void __launch_bounds__(256, PT == 4 ? 2 : 3) p1_climb_f32_kernel(const OpConst<float>* __restrict__ cst,
                                                                             const int4* __restrict__ tasks,
                                                                             int ntasks, int kch, int nfb,
                                                                             const int* __restrict__ pstart,
                                                                             const float* __restrict__ x,
                                                                             float* __restrict__ y) {
  if ((int)blockIdx.x >= ntasks) {
    const int b = blockIdx.x - ntasks;
    const int per_macro = 6 * nfb + 1;
    const int macro = b / per_macro, r = b - macro * per_macro;
    const int f = min(r / nfb, 6);
    p1_face_slice<float, DIRICHLET>(cst[macro], pstart, x, y, f, (r - f * nfb) * 256 + threadIdx.x);
    return;
  }
  const int4 task = tasks[blockIdx.x];
  const OpConst<float>& c = cst[task.w];
  const int N = c.N;
  const int lane = threadIdx.x & 31;
  const int j = task.y * kStencilWarps + (threadIdx.x >> 5);
  const int ib = task.x * 32 * PT;
  const int k0 = task.z * kch;
  const int kb = max(k0, 2);
  // row (j, k) holds a point i >= max(ib, 1) off the macro faces iff ib <= N - j - k - 1
  const int ke = min(min(k0 + kch - 1, N - j - ib - 1), N - kP1ClimbTop);
  if (j < 2 || ke < kb) return;   // whole warps only; the kernel has no barrier
  // faces i = 0 and i + j + k = N: zero sets {i} and {i+j+k = N} of the boundary table
  const bool dir_i0 = DIRICHLET && ((c.bnd_table >> 2) & 1u);
  const bool dir_diag = DIRICHLET && ((c.bnd_table >> 1) & 1u);
  const float* __restrict__ xb = x + c.base + ib + lane;
  float* __restrict__ yb = y + c.base + ib + lane;
  float S[15];
#pragma unroll
  for (int d = 0; d < 15; ++d) S[d] = c.S[d];
  P1Climb<PT> R;
  auto at = [&](int jr, int kr) { return __ldg(pstart + kr) + row32(N - kr, jr); };
  // planes kb-1 .. kb+1 for step 0 (slots of U = 0)
  p1_climb_row<-1, 0, PT>(R.P[0], xb + at(j + 1, kb - 1));
  p1_climb_row<-1, 0, PT>(R.P[1], xb + at(j + 1, kb));
  p1_climb_row<-1, 1, PT>(R.Z[0], xb + at(j, kb - 1));
  p1_climb_row<-1, 1, PT>(R.Z[1], xb + at(j, kb));
  p1_climb_row<-1, 1, PT>(R.Z[2], xb + at(j, kb + 1));
  p1_climb_row<0, 1, PT>(R.M[0], xb + at(j - 1, kb));
  p1_climb_row<0, 1, PT>(R.M[1], xb + at(j - 1, kb + 1));
  R.ap = at(j + 1, kb + 1);
  R.am = at(j - 1, kb + 2);
  R.az = at(j, kb + 2);
  R.ay = at(j, kb);
  R.t0 = tri(N - kb);
  if (kClimbAhead > 1) {
    // planes up to kb + kClimbAhead + 2 <= N - kP1ClimbTop + kClimbAhead + 2 < N
    const int off = min(32 * lane, 32 * PT + 1) - 1 - lane;
    R.fp = at(j + 1, kb + kClimbAhead + 1) + off;
    R.fm = at(j - 1, kb + kClimbAhead + 2) + off;
    R.fz = at(j, kb + kClimbAhead + 2) + off;
    R.ta = tri(N - kb - kClimbAhead);
  }
  for (int k = kb; k <= ke; k += 12) {
#define HHG_CLIMB_STEP(U)                                                                                     \
  if (k + U > ke) break;                                                                                      \
  p1_climb_step<U, PT, DIRICHLET>(R, S, xb, yb, N, dir_i0, dir_diag, ib, j, k + U, ke);
    HHG_CLIMB_STEP(0) HHG_CLIMB_STEP(1) HHG_CLIMB_STEP(2) HHG_CLIMB_STEP(3) HHG_CLIMB_STEP(4) HHG_CLIMB_STEP(5)
    HHG_CLIMB_STEP(6) HHG_CLIMB_STEP(7) HHG_CLIMB_STEP(8) HHG_CLIMB_STEP(9) HHG_CLIMB_STEP(10) HHG_CLIMB_STEP(11)
#undef HHG_CLIMB_STEP
  }
}

// ---------------------------------------------------------------------------
// P2 constant-coefficient apply in FP64 from shared-memory plane tiles (FP32 and double-float:
// p2_quad_kernel below).  A CTA owns rows j0..j0+7 and points i0..i0+TI-1 of a k-chunk and climbs its planes.  Each plane of the tile plus a halo of two
// points (the reach of a P2 row) is staged with cp.async into a ring of planes, kP2Ahead planes
// beyond the k+2 that the plane k being computed needs; staged Dirichlet points are zeroed on
// arrival.  A lane evaluates the points i0 + 64 v + 2 lane + {0, 1}: both node parities of its row,
// so a warp never diverges between stencils, with offsets known at compile time.  Even and odd
// staged columns are kept apart (column c at (c & 1) W/2 + c/2), so the 32 lanes of a warp read 32
// consecutive words.  The tile writes the points off the macro faces; p2_face_point the rest (extra
// blocks of the same launch).
constexpr int kP2TileJ = 8;
constexpr int kP2TileH = kP2TileJ + 4;
constexpr int kP2Ahead = 2;
constexpr int kP2Ring = kP2Ahead + 5;   // planes k-2 .. k+2+kP2Ahead; one barrier per plane

template <typename T, int TI>
constexpr size_t p2_tile_smem() {
  return sizeof(T) * kP2Ring * (TI + 4) * kP2TileH + sizeof(T) * kP2StTotal;
}

__host__ __device__ constexpr int p2_scol(int c, int W) { return (c & 1) * (W / 2) + (c >> 1); }

template <typename T, int TI>
__device__ __forceinline__ void p2_issue_plane(T* slot, const T* __restrict__ xm, const int* __restrict__ pstart, int N,
                                               int i0, int j0, int kk) {
  constexpr int W = TI + 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = warp + 8 * h;
    if (r >= kP2TileH) break;
    const int jr = j0 - 2 + r;
    const int len = N - jr - kk + 1;
    const bool rowok = jr >= 0 && kk >= 0 && kk <= N && len > 0;
    const T* __restrict__ row = rowok ? xm + __ldg(pstart + kk) + row32(N - kk, jr) : xm;
#pragma unroll
    for (int t = 0; t < (W + 31) / 32; ++t) {
      const int col = lane + 32 * t;
      if (col >= W) break;
      const int ii = i0 - 2 + col;
      // cells outside the macro are never read by a point the tile stores: not staged
      if (rowok && ii >= 0 && ii < len) cp_async_zfill(slot + r * W + p2_scol(col, W), row + ii, (int)sizeof(T), true);
    }
  }
}

// Zero the staged Dirichlet points of plane kk; each thread clears only what it staged itself.
template <typename T, int TI>
__device__ __forceinline__ void p2_mask_plane(T* slot, int N, uint32_t table, int i0, int j0, int kk) {
  constexpr int W = TI + 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = warp + 8 * h;
    if (r >= kP2TileH) break;
    const int jr = j0 - 2 + r;
    const int len = N - jr - kk + 1;
    if (!(jr >= 0 && kk >= 0 && kk <= N && len > 0)) continue;
    if (jr == 0 || kk == 0) {
#pragma unroll
      for (int t = 0; t < (W + 31) / 32; ++t) {
        const int col = lane + 32 * t;
        if (col >= W) break;
        const int ii = i0 - 2 + col;
        if (ii >= 0 && ii < len && on_dirichlet(table, N, ii, jr, kk)) slot[r * W + p2_scol(col, W)] = T(0);
      }
    } else {
      const int cand[2] = {2 - i0, len + 1 - i0};   // columns of i = 0 and i = len - 1
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int col = cand[e];
        if (col >= 0 && col < W && (col & 31) == lane) {
          const int ii = i0 - 2 + col;
          if (on_dirichlet(table, N, ii, jr, kk)) slot[r * W + p2_scol(col, W)] = T(0);
        }
      }
    }
  }
}

// Cell C of the union list of row parity PA (even point) for the lane; ob = r W + 1 + lane.
template <typename T, int W, int NV, int PA, int C>
__device__ __forceinline__ void p2_tile_cell(const T* w, const T* const (&pl)[5], int ob, T (&a0)[NV], T (&a1)[NV]) {
  constexpr int O = P2UCell<PA, C>::off, IA = P2UCell<PA, C>::ia, IB = P2UCell<PA, C>::ib;
  constexpr int dx = (O & 15) - 2, dy = ((O >> 4) & 15) - 2, dz = ((O >> 8) & 15) - 2;
  constexpr int off = dy * W + (dx & 1) * (W / 2) + ((dx + 4) >> 1) - 2;   // staged column 2 + 2 lane + dx
  const T* p = pl[dz + 2] + ob + off;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T xv = p[32 * v];
    if constexpr (IA >= 0) a0[v] += w[P2Start<PA>::v + IA] * xv;
    if constexpr (IB >= 0) a1[v] += w[P2Start<PA | 1>::v + IB] * xv;
  }
}

template <typename T, int W, int NV, int PA, int... C>
__device__ __forceinline__ void p2_tile_cells(const T* w, const T* const (&pl)[5], int ob,
                                              T (&a0)[NV], T (&a1)[NV], std::integer_sequence<int, C...>) {
  (p2_tile_cell<T, W, NV, PA, C>(w, pl, ob, a0, a1), ...);
}

// Interior rows of parities PA (even i) and PA | 1 (odd i) over the union of their cells.
template <typename T, int W, int NV, int PA>
__device__ __forceinline__ void p2_tile_pair(const T* w, const T* const (&pl)[5], int ob,
                                             T (&a0)[NV], T (&a1)[NV]) {
  p2_tile_cells<T, W, NV, PA>(w, pl, ob, a0, a1, std::make_integer_sequence<int, P2UCnt<PA>::v>{});
}

// Interior points of one tile row (row parity PA): the second half of a 128-point tile only when
// the row reaches into it.  Points on macro faces are left to p2_face_point.
template <typename T, int W, int NV, int PA>
__device__ __forceinline__ void p2_tile_row(const T* w, const T* const (&pl)[5], int ob, int i0,
                                            int len, T* __restrict__ yrow) {
  const int lane = threadIdx.x & 31;
  if (NV == 2 && len - i0 <= 64) {
    T a0[1] = {T(0)}, a1[1] = {T(0)};
    p2_tile_pair<T, W, 1, PA>(w, pl, ob, a0, a1);
    const int ii = i0 + 2 * lane;
    if (ii > 0 && ii < len - 1) yrow[ii] = a0[0];
    if (ii + 1 < len - 1) yrow[ii + 1] = a1[0];
    return;
  }
  T a0[NV], a1[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) a0[v] = a1[v] = T(0);
  p2_tile_pair<T, W, NV, PA>(w, pl, ob, a0, a1);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int ii = i0 + 64 * v + 2 * lane;
    if (ii > 0 && ii < len - 1) yrow[ii] = a0[v];
    if (ii + 1 < len - 1) yrow[ii + 1] = a1[v];
  }
}

// Points on the faces of the macros (zero mask z != 0), one thread each (thread t of face f): face a
// of the macro has the points (a, b) with a + b <= N of its triangle; a point on several faces is
// written by the lowest.  Its row comes from the face table (zero weights outside the macro); x is
// read from global memory.  offs / starts: the stencil offsets and class starts, staged in shared
// memory by the caller.
template <typename T, bool DIRICHLET>
__device__ __forceinline__ void p2_face_point(const OpConst<T>& c, const P2Stencil<T>& stm, const int* offs,
                                              const int* starts, const int* __restrict__ pstart,
                                              const T* __restrict__ x, T* __restrict__ y, int f, int t) {
  const int N = c.N;
  if (t >= tri(N)) return;
  const float bq = 2.0f * N + 3.0f;
  int b = (int)(0.5f * (bq - sqrtf(fmaxf(bq * bq - 8.0f * (float)t, 0.0f))));
  b = max(0, min(b, N));
  if (b < N && row32(N, b + 1) <= t) ++b;
  if (b > 0 && row32(N, b) > t) --b;
  const int a = t - row32(N, b);
  int i, j, k;
  if (f == 0) {
    i = 0; j = a; k = b;
  } else if (f == 1) {
    i = a; j = 0; k = b;
  } else if (f == 2) {
    i = a; j = b; k = 0;
  } else {
    i = N - a - b; j = a; k = b;
  }
  if ((f >= 1 && i == 0) || (f >= 2 && j == 0) || (f == 3 && k == 0)) return;
  const T* __restrict__ xm = x + c.base;
  T* __restrict__ ym = y + c.base;
  const uint32_t table = c.bnd_table;
  const int p = __ldg(pstart + k) + row32(N - k, j) + i;
  if (DIRICHLET && on_dirichlet(table, N, i, j, k)) {
    ym[p] = xm[p];
    return;
  }
  const int z = zero_mask(N, i, j, k);
  const T* __restrict__ wz = stm.w[z];
  const int par = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
  T acc = T(0);
  const int d1 = starts[par + 1];
  for (int d = starts[par]; d < d1; ++d) {
    const T w = __ldg(wz + d);
    if (w == T(0)) continue;   // no micro-tet of the macro couples the two points
    const int o = offs[d];
    const int ii = i + (o & 15) - 2, jj = j + ((o >> 4) & 15) - 2, kk = k + ((o >> 8) & 15) - 2;
    if (DIRICHLET && on_dirichlet(table, N, ii, jj, kk)) continue;
    acc += w * __ldg(xm + __ldg(pstart + kk) + row32(N - kk, jj) + ii);
  }
  ym[p] = acc;
}

template <typename T, int TI, bool DIRICHLET>
__global__ void __launch_bounds__(256) p2_tile_kernel(const OpConst<T>* __restrict__ cst,
                                                      const P2Stencil<T>* __restrict__ st,
                                                      const P2StencilIndex* __restrict__ sidx,
                                                      const int4* __restrict__ tasks, int ntasks, int kch, int nfb,
                                                      const int* __restrict__ pstart, const T* __restrict__ x,
                                                      T* __restrict__ y) {
  constexpr int W = TI + 4;
  constexpr int SLOT = W * kP2TileH;
  constexpr int NV = TI / 64;
  extern __shared__ __align__(16) unsigned char p2_tile_smem_raw[];
  if ((int)blockIdx.x >= ntasks) {
    // blocks after the tile tasks write the face points (4 faces x nfb blocks per macro), filling the
    // SMs that the last tiles leave idle
    int* offs = reinterpret_cast<int*>(p2_tile_smem_raw);
    int* starts = offs + kP2StTotal;
    for (int t = threadIdx.x; t < kP2StTotal; t += blockDim.x) offs[t] = sidx->off[t];
    if (threadIdx.x < 9) starts[threadIdx.x] = sidx->start[threadIdx.x];
    __syncthreads();
    const int b = blockIdx.x - ntasks;
    const int macro = b / (4 * nfb), r = b - macro * 4 * nfb;
    const int f = r / nfb;
    p2_face_point<T, DIRICHLET>(cst[macro], st[macro], offs, starts, pstart, x, y, f, (r - f * nfb) * 256 + threadIdx.x);
    return;
  }
  static_assert(std::is_same<T, double>::value, "FP32 runs p2_quad_kernel");
  T* buf = reinterpret_cast<T*>(p2_tile_smem_raw);
  T* w0 = buf + kP2Ring * SLOT;
  const int4 task = tasks[blockIdx.x];
  const OpConst<T>& c = cst[task.w];
  const int N = c.N;
  const int i0 = task.x * TI, j0 = task.y * kP2TileJ, k0 = task.z * kch;
  const int k_end = min(k0 + kch - 1, N - j0 - i0);
  if (k_end < k0) return;   // uniform over the CTA
  for (int t = threadIdx.x; t < kP2StTotal; t += blockDim.x) w0[t] = st[task.w].w[0][t];
  const uint32_t table = c.bnd_table;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* __restrict__ xm = x + c.base;
  T* __restrict__ ym = y + c.base;
  for (int q = 0; q < kP2Ring - 1; ++q) {
    const int kk = k0 - 2 + q;
    if (kk <= k_end + 2) p2_issue_plane<T, TI>(buf + q * SLOT, xm, pstart, N, i0, j0, kk);
    cp_async_commit();
  }
  cp_async_wait<kP2Ahead>();   // planes k0-2 .. k0+1 have arrived
  // a staged plane can hold points of a macro face only if the tile touches i = 0, j = 0, k = 0 or
  // reaches i + j + k = N; only then are its Dirichlet points looked for (uniform over the CTA)
  const bool edge_tile = i0 == 0 || j0 == 0 || i0 + TI + 1 + j0 + kP2TileJ + 1 + k_end + 2 >= N;
  if (DIRICHLET && (edge_tile || k0 <= 2)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) p2_mask_plane<T, TI>(buf + q * SLOT, N, table, i0, j0, k0 - 2 + q);
  }
  const int j = j0 + warp;
  const int ob = (warp + 2) * W + 1 + lane;
  for (int k = k0; k <= k_end; ++k) {
    const int q = k - k0;   // plane kk sits in ring slot (kk - k0 + 2) mod kP2Ring
    cp_async_wait<kP2Ahead - 1>();   // plane k+2 has arrived
    if (DIRICHLET && edge_tile) p2_mask_plane<T, TI>(buf + ((q + 4) % kP2Ring) * SLOT, N, table, i0, j0, k + 2);
    __syncthreads();
    {
      const int kn = k + 2 + kP2Ahead;   // into the slot of plane k-3, read for the last time in step k-1
      if (kn <= k_end + 2) p2_issue_plane<T, TI>(buf + ((q + 4 + kP2Ahead) % kP2Ring) * SLOT, xm, pstart, N, i0, j0, kn);
      cp_async_commit();
    }
    const int len = N - j - k + 1;
    // rows j = 0 and planes k = 0 hold only points on macro faces
    if (j > 0 && k > 0 && len > 0 && i0 < len) {
      const T* pl[5];
#pragma unroll
      for (int t = 0; t < 5; ++t) pl[t] = buf + ((q + t) % kP2Ring) * SLOT;
      T* __restrict__ yrow = ym + __ldg(pstart + k) + row32(N - k, j);
      switch ((j & 1) | ((k & 1) << 1)) {
        case 0: p2_tile_row<T, W, NV, 0>(w0, pl, ob, i0, len, yrow); break;
        case 1: p2_tile_row<T, W, NV, 2>(w0, pl, ob, i0, len, yrow); break;
        case 2: p2_tile_row<T, W, NV, 4>(w0, pl, ob, i0, len, yrow); break;
        default: p2_tile_row<T, W, NV, 6>(w0, pl, ob, i0, len, yrow); break;
      }
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// P2 constant-coefficient apply with two planes per step and the weights in the parameter bank, in
// FP32 or in double-float arithmetic (FP64 vectors, FP32 pairs).  The launch covers one macro; its
// 230 interior weights come by value (P2ParamW / P2ParamWDF), so every FMA takes its weight from the
// constant bank and no load feeds it.  The tiles and the staging are those of p2_tile_kernel (8 rows
// x TI points plus a halo of two, even and odd columns apart), but a step evaluates the planes k and
// k+1 together: a lane's four points (even and odd i, planes k and k+1) share the union of their
// cells, which is loaded from shared memory once (2.8 x fewer loads per point than one plane at a
// time).  The ring holds 10 planes: at step k the planes k-2 .. k+3 are read, k+4 and k+5 (landed)
// get their Dirichlet points zeroed, k+6 and k+7 are being copied; one barrier per step.
constexpr int kP2QRing = 10;
constexpr int kP2QStreams = 8;   // streams the per-macro launches of a multi-macro apply share

// FP32: 128-point tiles, staged values and weights in FP32.
struct P2QF32 {
  using E = float;    // staged value
  using V = float;    // vector entry
  using WP = P2ParamW;
  static constexpr int TI = 128;
  __device__ __forceinline__ static void fma(float& acc, float w, float v) { acc = fmaf(w, v, acc); }
  __device__ __forceinline__ static float out(float acc) { return acc; }
};
// Double-float: FP64 vectors split into FP32 pairs by a streaming pass, weights split on the host,
// products and sums by df_fma (exact products, two-sum of the high parts); 64-point tiles (the
// staged pairs take twice the shared memory).
struct P2QDF {
  using E = float2;
  using V = double;
  using WP = P2ParamWDF;
  static constexpr int TI = 64;
  __device__ __forceinline__ static void fma(float2& acc, float2 w, float2 v) { df_fma(acc, w, v); }
  __device__ __forceinline__ static double out(float2 acc) {
    return float_to_double_bits(acc.x) + float_to_double_bits(acc.y);
  }
};
template <class A>
constexpr size_t p2q_smem() {
  return sizeof(typename A::E) * kP2QRing * (A::TI + 4) * kP2TileH;   // FP32 63,360, double-float 65,280 bytes
}

// Union of the cells of the four points of a lane in one step, as offsets from the even point of
// plane k (packed (dx+2) | (dy+2) << 4 | (dz+2) << 8, dx in -2..3, dz in -2..3), sorted; e[c][q]:
// the entry of point q's stencil that uses cell c (-1: none).  q = 0 / 1: even / odd point of
// plane k (parities PA, PA | 1), q = 2 / 3: the same on plane k+1 (parities PA ^ 4, (PA ^ 4) | 1).
struct P2QuadList {
  int n;
  int off[128];
  int e[128][4];
};
__host__ __device__ constexpr int p2q_par(int pa, int q) { return ((q & 2) ? (pa ^ 4) : pa) | (q & 1); }
__host__ __device__ constexpr P2QuadList p2_quad_list(int pa) {
  P2QuadList U{};
  for (int q = 0; q < 4; ++q) {
    const P2OffList L = p2_struct_list(p2q_par(pa, q));
    for (int d = 0; d < L.n; ++d) {
      const int v = L.off[d] + (q & 1) + ((q >> 1) << 8);   // dx + 1 for the odd point, dz + 1 for plane k+1
      int pos = 0;
      while (pos < U.n && U.off[pos] < v) ++pos;
      if (!(pos < U.n && U.off[pos] == v)) {
        for (int t = U.n; t > pos; --t) {
          U.off[t] = U.off[t - 1];
          for (int r = 0; r < 4; ++r) U.e[t][r] = U.e[t - 1][r];
        }
        U.off[pos] = v;
        for (int r = 0; r < 4; ++r) U.e[pos][r] = -1;
        ++U.n;
      }
      U.e[pos][q] = d;
    }
  }
  return U;
}
template <int PA>
struct P2QCnt {
  static constexpr int v = p2_quad_list(PA).n;
};
template <int PA, int C>
struct P2QCell {
  static constexpr P2QuadList L = p2_quad_list(PA);   // host-side constant only, read below
  static constexpr int off = L.off[C];
  static constexpr int e0 = L.e[C][0], e1 = L.e[C][1], e2 = L.e[C][2], e3 = L.e[C][3];
};
// first weight of parity p in the 230-entry list
__host__ __device__ constexpr int p2_start(int p) {
  int s = 0;
  for (int t = 0; t < p; ++t) s += p2_struct_list(t).n;
  return s;
}
template <int PA, int Q>
struct P2QStart {
  static constexpr int v = p2_start(p2q_par(PA, Q));
};

// Staging plan.  A plane of the tile is 12 rows of W = TI + 4 columns, chunks of 32 columns per row
// (5 for TI = 128, 3 for TI = 64, the last one 4 wide).  Warp w copies row w whole (h = 0) and of
// row 8 + (w & 3) (h = 1) chunks 0-2 (w < 4) and 3-4 (w >= 4).  Per row the plan keeps what does not
// change from plane to plane: the row j, the packed offset of its column 0 without the plane terms,
// and the column limit, so that plane kk costs one multiply-add per row:
// start(j, kk) = pstart[kk] + row32(N - kk, j) = pstart[kk] + j (2N + 3 - j) / 2 - j kk.
struct P2QStage {
  int jr[2];        // row j of the staged row (h = 0, 1)
  int off[2];       // j (2N + 3 - j) / 2 + i0 - 2 + lane: add pstart[kk] - j kk
  int lim[2];       // N - j + 3 - i0: staged column col < lim - kk lies inside the row (very negative
                    // for rows j < 0)
  unsigned dst[2];  // shared address of the lane's column in ring slot 0
  int r[2];
};

// chunks 0 .. kP2QLo - 1 of an h = 1 row are copied by warps 0-3, the others by warps 4-7
constexpr int kP2QLo = 3;
__device__ __forceinline__ bool p2q_mine(int h, int t, int warp) { return h == 0 || ((warp < 4) == (t < kP2QLo)); }

template <int TI, typename E>
__device__ __forceinline__ P2QStage p2q_plan(E* buf, int N, int i0, int j0) {
  constexpr int W = TI + 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s0 = (lane & 1) * (W / 2) + (lane >> 1);
  P2QStage st;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = h == 0 ? warp : 8 + (warp & 3);
    const int jr = j0 - 2 + r;
    st.r[h] = r;
    st.jr[h] = jr;
    st.off[h] = ((jr * (2 * N + 3 - jr)) >> 1) + i0 - 2 + lane;
    st.lim[h] = jr >= 0 ? N - jr + 3 - i0 : -(1 << 30);
    st.dst[h] = (unsigned)__cvta_generic_to_shared(buf + r * W + s0);
  }
  return st;
}

// Chunk T of a staged row of B-byte values: columns lane + 32 T, at byte offsets 16 B T (shared)
// and 32 B T (global).
template <int T, int B>
__device__ __forceinline__ void p2q_copy(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0+%2], [%1+%3], %4;\n" ::"r"(dst), "l"(src), "n"(16 * B * T),
               "n"(32 * B * T), "n"(B));
}

// Copy plane kk (first packed position pk) into ring slot `slot` by the plan.  Columns outside the
// row (before i = 0, after i = len - 1) feed only points the tile does not store, so a row whose
// window of W values lies inside the vector (packed offsets gmin .. gmax of its first value) is
// copied whole without tests; only rows at the two ends of the vector test each column.
template <int TI, typename E>
__device__ __forceinline__ void p2q_issue_plane(const P2QStage& st, int slot, const E* __restrict__ xm, int pk, int N,
                                                int i0, int kk, int gmin, int gmax) {
  constexpr int W = TI + 4;
  constexpr int B = (int)sizeof(E);
  constexpr unsigned SLOT_BYTES = B * W * kP2TileH;
  constexpr int NCH = (W + 31) / 32;
  static_assert(W - 32 * (NCH - 1) == 4 && NCH >= kP2QLo, "chunks of 32 columns, the last 4 wide");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (kk < 0 || kk > N) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int jr = st.jr[h];
    const int lim = st.lim[h] - kk;   // staged column col holds i = i0 - 2 + col < len
    if (lim + i0 - 2 <= 0) continue;  // no row (j < 0 or beyond the plane)
    const int g = pk - jr * kk + st.off[h] - lane;   // packed offset of column 0
    const E* __restrict__ src = xm + (g + lane);
    const unsigned dst = st.dst[h] + slot * SLOT_BYTES;
    const bool lo = h == 0 || warp < 4, hi = h == 0 || warp >= 4;   // chunks below / from kP2QLo
    if (g >= gmin && g <= gmax) {
      if (lo) {
        p2q_copy<0, B>(dst, src);
        p2q_copy<1, B>(dst, src);
        if (NCH == 5) p2q_copy<2, B>(dst, src);
        else if (lane < 4) p2q_copy<2, B>(dst, src);
      }
      if (NCH == 5 && hi) {
        p2q_copy<3, B>(dst, src);
        if (lane < 4) p2q_copy<4, B>(dst, src);
      }
    } else {
#pragma unroll 1
      for (int t = lo ? 0 : kP2QLo; t < (hi ? NCH : kP2QLo); ++t) {
        const int col = lane + 32 * t;
        if (col < W && col < lim && col + i0 >= 2) {
          const unsigned sa = dst + 16 * B * t;
          asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(src + 32 * t), "n"(B));
        }
      }
    }
  }
}

// Dirichlet points of staged planes, zeroed once the copies are visible to the whole CTA (after a
// barrier, before the barrier that precedes their first read).  A row with j, k >= 1 meets the
// macro faces only at i = 0 (zero set {i}, or {i, diagonal} for a row of one point) and i = len - 1
// ({diagonal}, or {i, diagonal}): one thread per (plane, row, end) checks and zeroes that point.
// Rows j = 0 and k = 0 lie on a face: a warp looks up each of their points (p2q_mask_face_row).
template <int TI, typename E>
__device__ __forceinline__ void p2q_mask_end(E* buf, int slot, int N, uint32_t table, int i0, int j0, int kk, int r,
                                             int end) {
  constexpr int W = TI + 4;
  const int jr = j0 - 2 + r;
  const int len = N - jr - kk + 1;
  if (jr < 1 || kk < 1 || len < 1) return;
  const bool one = len == 1;
  const int col = end == 0 ? 2 - i0 : len + 1 - i0;   // column of i = 0 / i = len - 1
  const bool dir = (table >> (one ? 3 : (end == 0 ? 2 : 1))) & 1u;
  if (dir && (unsigned)col < (unsigned)W) buf[slot * (W * kP2TileH) + r * W + p2_scol(col, W)] = E{};
}

template <int TI, typename E>
__device__ __forceinline__ void p2q_mask_face_row(E* buf, int slot, int N, uint32_t table, int i0, int j0, int kk,
                                                  int r) {
  constexpr int W = TI + 4;
  const int lane = threadIdx.x & 31;
  const int jr = j0 - 2 + r;
  const int len = N - jr - kk + 1;
  if (jr < 0 || kk < 0 || len < 1 || !(jr == 0 || kk == 0)) return;
#pragma unroll 1
  for (int col = lane; col < W; col += 32) {
    const int ii = i0 - 2 + col;
    if (ii >= 0 && ii < len && on_dirichlet(table, N, ii, jr, kk)) buf[slot * (W * kP2TileH) + r * W + p2_scol(col, W)] = E{};
  }
}

template <class A, int W, int NV, int PA, int C>
__device__ __forceinline__ void p2q_cell(const typename A::WP& wp, const typename A::E* const (&pl)[6], int ob,
                                         typename A::E (&acc)[4][NV]) {
  using Cell = P2QCell<PA, C>;
  constexpr int O = Cell::off;
  constexpr int dx = (O & 15) - 2, dy = ((O >> 4) & 15) - 2, dz = ((O >> 8) & 15) - 2;
  constexpr int off = dy * W + (dx & 1) * (W / 2) + ((dx + 4) >> 1) - 2;   // staged column 2 + 2 lane + dx
  const typename A::E* p = pl[dz + 2] + ob + off;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const typename A::E xv = p[32 * v];
    if constexpr (Cell::e0 >= 0) A::fma(acc[0][v], wp.w[P2QStart<PA, 0>::v + Cell::e0], xv);
    if constexpr (Cell::e1 >= 0) A::fma(acc[1][v], wp.w[P2QStart<PA, 1>::v + Cell::e1], xv);
    if constexpr (Cell::e2 >= 0) A::fma(acc[2][v], wp.w[P2QStart<PA, 2>::v + Cell::e2], xv);
    if constexpr (Cell::e3 >= 0) A::fma(acc[3][v], wp.w[P2QStart<PA, 3>::v + Cell::e3], xv);
  }
}

template <class A, int W, int NV, int PA, int... C>
__device__ __forceinline__ void p2q_cells(const typename A::WP& wp, const typename A::E* const (&pl)[6], int ob,
                                          typename A::E (&acc)[4][NV], std::integer_sequence<int, C...>) {
  (p2q_cell<A, W, NV, PA, C>(wp, pl, ob, acc), ...);
}

// Points of row j on planes k (length len0) and k+1 (len0 - 1; only if wk1) for row parity PA
// (of plane k): the interior points among i0 + 64 v + 2 lane + {0, 1}.
template <class A, int W, int NV, int PA>
__device__ __forceinline__ void p2q_rows(const typename A::WP& wp, const typename A::E* const (&pl)[6], int ob, int i0,
                                         int len0, bool wk0, bool wk1, typename A::V* __restrict__ y0,
                                         typename A::V* __restrict__ y1) {
  const int lane = threadIdx.x & 31;
  typename A::E acc[4][NV];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[q][v] = typename A::E{};
  p2q_cells<A, W, NV, PA>(wp, pl, ob, acc, std::make_integer_sequence<int, P2QCnt<PA>::v>{});
  if (i0 > 0 && i0 + 64 * NV + 1 < len0 && wk0 && wk1) {
    // every point of the lane on both planes is off the macro faces
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int ii = i0 + 64 * v + 2 * lane;
      y0[ii] = A::out(acc[0][v]);
      y0[ii + 1] = A::out(acc[1][v]);
      y1[ii] = A::out(acc[2][v]);
      y1[ii + 1] = A::out(acc[3][v]);
    }
    return;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int ii = i0 + 64 * v + 2 * lane;
    if (wk0) {
      if (ii > 0 && ii < len0 - 1) y0[ii] = A::out(acc[0][v]);
      if (ii + 1 < len0 - 1) y0[ii + 1] = A::out(acc[1][v]);
    }
    if (wk1) {
      if (ii > 0 && ii < len0 - 2) y1[ii] = A::out(acc[2][v]);
      if (ii + 1 < len0 - 2) y1[ii + 1] = A::out(acc[3][v]);
    }
  }
}

template <class A, int W, int PA>
__device__ __forceinline__ void p2q_step(const typename A::WP& wp, const typename A::E* const (&pl)[6], int ob, int i0,
                                         int len0, bool wk0, bool wk1, typename A::V* __restrict__ y0,
                                         typename A::V* __restrict__ y1) {
  // the second 64 points only when the longer row reaches into them
  if (A::TI == 64 || len0 - i0 <= 64)
    p2q_rows<A, W, 1, PA>(wp, pl, ob, i0, len0, wk0, wk1, y0, y1);
  else
    p2q_rows<A, W, A::TI / 64, PA>(wp, pl, ob, i0, len0, wk0, wk1, y0, y1);
}

// One macro (cm = its constants, stm = its face stencils); blocks after the tile tasks write the
// macro's face points (4 faces x nfb blocks, from x in the vector type).  xs: the staged vector
// (x itself in FP32, its split pairs in double-float).
template <class A, bool DIRICHLET>
__global__ void __launch_bounds__(256, 3) p2_quad_kernel(const __grid_constant__ typename A::WP wp,
                                                      const OpConst<typename A::V>* __restrict__ cm,
                                                      const P2Stencil<typename A::V>* __restrict__ stm,
                                                      const P2StencilIndex* __restrict__ sidx,
                                                      const int4* __restrict__ tasks, int ntasks, int kch, int nfb,
                                                      const int* __restrict__ pstart,
                                                      const typename A::E* __restrict__ xs,
                                                      const typename A::V* __restrict__ x,
                                                      typename A::V* __restrict__ y, int64_t npts) {
  using E = typename A::E;
  using V = typename A::V;
  constexpr int TI = A::TI;
  constexpr int W = TI + 4;
  constexpr int SLOT = W * kP2TileH;
  extern __shared__ __align__(16) unsigned char p2_quad_smem_raw[];
  if ((int)blockIdx.x >= ntasks) {
    int* offs = reinterpret_cast<int*>(p2_quad_smem_raw);
    int* starts = offs + kP2StTotal;
    for (int t = threadIdx.x; t < kP2StTotal; t += blockDim.x) offs[t] = sidx->off[t];
    if (threadIdx.x < 9) starts[threadIdx.x] = sidx->start[threadIdx.x];
    __syncthreads();
    const int b = blockIdx.x - ntasks;
    const int f = b / nfb;
    p2_face_point<V, DIRICHLET>(*cm, *stm, offs, starts, pstart, x, y, f, (b - f * nfb) * 256 + threadIdx.x);
    return;
  }
  E* buf = reinterpret_cast<E*>(p2_quad_smem_raw);
  const int4 task = tasks[blockIdx.x];
  const OpConst<V>& c = *cm;
  const int N = c.N;
  const int i0 = task.x * TI, j0 = task.y * kP2TileJ, k0 = task.z * kch;
  const int k_end = min(k0 + kch - 1, N - j0 - i0);
  if (k_end < k0) return;   // uniform over the CTA
  const uint32_t table = c.bnd_table;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const E* __restrict__ xm = xs + c.base;
  V* __restrict__ ym = y + c.base;
  const P2QStage st = p2q_plan<TI>(buf, N, i0, j0);
  auto plane_start = [&](int kk) { return (kk >= 0 && kk <= N) ? __ldg(pstart + kk) : 0; };
  // a staged row's W values (first at packed offset g of the macro) lie inside the vector
  const int gmin = c.base >= 2 ? -2 : -(int)c.base;
  const int gmax = (int)min(npts - c.base - W, (int64_t)INT_MAX);
  // plane kk sits in ring slot (kk - k0 + 2) mod 10; planes k0-2 .. k0+5 first, their Dirichlet points
  // zeroed before the first step
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    const int kk = k0 - 2 + q;
    if (kk <= k_end + 3) p2q_issue_plane<TI>(st, q, xm, plane_start(kk), N, i0, kk, gmin, gmax);
  }
  cp_async_commit();
  // a staged plane can hold points of a macro face only if the tile touches i = 0, j = 0, k = 0 or
  // reaches i + j + k = N; only then are its Dirichlet points looked for (uniform over the CTA)
  const bool edge_tile = i0 == 0 || j0 == 0 || i0 + TI + 1 + j0 + kP2TileJ + 1 + k_end + 3 >= N;
  if (DIRICHLET && (edge_tile || k0 <= 2)) {
    cp_async_wait<0>();
    __syncthreads();
    // 8 planes x 12 rows x 2 ends: 192 threads; the rows on a face: warp w for plane k0-2+w
    if (threadIdx.x < 192) {
      const int q = threadIdx.x / 24, rr = threadIdx.x % 24;
      p2q_mask_end<TI>(buf, q, N, table, i0, j0, k0 - 2 + q, rr >> 1, rr & 1);
    }
    if ((j0 <= 2 || k0 <= 2) && k0 - 2 + warp <= k_end + 3) {
#pragma unroll 1
      for (int r = 0; r < kP2TileH; ++r) p2q_mask_face_row<TI>(buf, warp, N, table, i0, j0, k0 - 2 + warp, r);
    }
  }
  const int j = j0 + warp;
  const int ob = (warp + 2) * W + 1 + lane;
  int sq = 0;   // ring slot of plane k - 2
  for (int k = k0; k <= k_end; k += 2) {
    const int q = k - k0;
    const int pk6 = plane_start(k + 6), pk7 = plane_start(k + 7);
    auto slot = [&](int t) { const int v = sq + t; return v >= kP2QRing ? v - kP2QRing : v; };
    cp_async_wait<0>();   // planes up to k+5 have landed
    __syncthreads();      // ... and are visible; planes up to k+3 have their Dirichlet points zeroed
    if (DIRICHLET && edge_tile && q > 0) {
      // planes k+4, k+5 (first read in step k+2)
      if (threadIdx.x < 48) {
        const int p = threadIdx.x / 24, rr = threadIdx.x % 24;
        p2q_mask_end<TI>(buf, slot(6 + p), N, table, i0, j0, k + 4 + p, rr >> 1, rr & 1);
      }
      if (j0 <= 2 && warp >= 6) p2q_mask_face_row<TI>(buf, slot(warp), N, table, i0, j0, k + warp - 2, 2 - j0);
    }
    // planes k+6, k+7 into the slots of k-4, k-3, read for the last time in step k-2
    if (k + 6 <= k_end + 3) p2q_issue_plane<TI>(st, slot(8), xm, pk6, N, i0, k + 6, gmin, gmax);
    if (k + 7 <= k_end + 3) p2q_issue_plane<TI>(st, slot(9), xm, pk7, N, i0, k + 7, gmin, gmax);
    cp_async_commit();
    const int len0 = N - j - k + 1;
    // rows j = 0 and planes k = 0 hold only points on macro faces
    const bool wk0 = k > 0 && k <= k_end, wk1 = k + 1 <= k_end;
    if (j > 0 && len0 > 0 && i0 < len0) {
      const E* pl[6];
#pragma unroll
      for (int t = 0; t < 6; ++t) pl[t] = buf + slot(t) * SLOT;
      V* __restrict__ y0 = ym + __ldg(pstart + k) + row32(N - k, j);
      V* __restrict__ y1 = ym + __ldg(pstart + k + 1) + row32(N - k - 1, j);
      switch ((j & 1) | ((k & 1) << 1)) {
        case 0: p2q_step<A, W, 0>(wp, pl, ob, i0, len0, wk0, wk1, y0, y1); break;
        case 1: p2q_step<A, W, 2>(wp, pl, ob, i0, len0, wk0, wk1, y0, y1); break;
        case 2: p2q_step<A, W, 4>(wp, pl, ob, i0, len0, wk0, wk1, y0, y1); break;
        default: p2q_step<A, W, 6>(wp, pl, ob, i0, len0, wk0, wk1, y0, y1); break;
      }
    }
    sq = slot(2);
  }
  cp_async_wait<0>();
}

// The two-plane kernel's ring exceeds the default 48 KB of dynamic shared memory.
static int p2_quad_prepare() {
  static_assert(p2q_smem<P2QF32>() >= sizeof(int) * (kP2StTotal + 9), "face blocks stage the stencil index in the tile's shared memory");
  HHG_CUDA_TRY(cudaFuncSetAttribute(p2_quad_kernel<P2QF32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)p2q_smem<P2QF32>()));
  HHG_CUDA_TRY(cudaFuncSetAttribute(p2_quad_kernel<P2QF32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)p2q_smem<P2QF32>()));
  HHG_CUDA_TRY(cudaFuncSetAttribute(p2_quad_kernel<P2QDF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)p2q_smem<P2QDF>()));
  HHG_CUDA_TRY(cudaFuncSetAttribute(p2_quad_kernel<P2QDF, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)p2q_smem<P2QDF>()));
  return HHG_OK;
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

// Edge DoFs of the Nedelec operator: copies are related by orientation signs.
template <typename T>
__global__ void iface_sum_signed_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                        const int8_t* __restrict__ sgn, const uint8_t* __restrict__ bnd,
                                        int64_t ngroups, bool dirichlet, T* __restrict__ y) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  if (dirichlet && bnd[g]) return;
  const int64_t a = ptr[g], b = ptr[g + 1];
  T s = T(0);
  for (int64_t t = a; t < b; ++t) s += T(sgn[t]) * y[idx[t]];
  for (int64_t t = a; t < b; ++t) y[idx[t]] = T(sgn[t]) * s;
}

template <typename T>
int launch_interface_sum_signed(const Interface* itf, T* y, bool dirichlet, cudaStream_t s) {
  if (itf->ngroups == 0) return HHG_OK;
  const int th = 128;
  iface_sum_signed_kernel<T><<<(unsigned)((itf->ngroups + th - 1) / th), th, 0, s>>>(
      itf->d_ptr, itf->d_idx, itf->d_sign, itf->d_bnd, itf->ngroups, dirichlet, y);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}
template <typename T>
__global__ void iface_copy_owner_signed_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ idx,
                                               const int8_t* __restrict__ sgn, int64_t ngroups, T* __restrict__ x) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  const int64_t a = ptr[g], b = ptr[g + 1];
  const T v = T(sgn[a]) * x[idx[a]];
  for (int64_t t = a + 1; t < b; ++t) x[idx[t]] = T(sgn[t]) * v;
}

template <typename T>
int launch_make_consistent_signed(const Interface* itf, T* x, cudaStream_t s) {
  if (itf->ngroups == 0) return HHG_OK;
  iface_copy_owner_signed_kernel<T><<<(unsigned)((itf->ngroups + 255) / 256), 256, 0, s>>>(itf->d_ptr, itf->d_idx,
                                                                                          itf->d_sign, itf->ngroups, x);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}
template int launch_make_consistent_signed<double>(const Interface*, double*, cudaStream_t);
template int launch_make_consistent_signed<float>(const Interface*, float*, cudaStream_t);

template int launch_interface_sum_signed<double>(const Interface*, double*, bool, cudaStream_t);
template int launch_interface_sum_signed<float>(const Interface*, float*, bool, cudaStream_t);

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

static inline int64_t tri_host(int64_t s) { return (s + 1) * (s + 2) / 2; }

// The two-plane P2 kernel over every macro of the op: one launch per macro (its weights w[m] in the
// parameter bank), on the caller's stream or, for several macros, side by side on the op's streams
// (a launch per macro alone leaves the GPU part empty while its last tiles run), forked from and
// joined back into the caller's stream.
template <class A>
static int launch_p2_quad(const hhg_op* op, const typename A::WP* w, const typename A::E* xs, const typename A::V* x,
                          typename A::V* y, cudaStream_t s) {
  using V = typename A::V;
  const Interface* I = op->itf;
  const int nm = op->mesh->nmacro();
  const OpConst<V>* cst = (const OpConst<V>*)(sizeof(V) == 8 ? op->d_const64 : op->d_const32);
  const P2Stencil<V>* st = (const P2Stencil<V>*)(sizeof(V) == 8 ? op->d_p2st64 : op->d_p2st32);
  const TileTasks& tt = I->tile[A::TI == 128 ? 0 : 2];
  const P2StencilIndex* ix = (const P2StencilIndex*)op->d_p2idx;
  const int nfb = (int)((tri_host(op->N) + 255) / 256);
  const unsigned grid = (unsigned)(tt.n + 4 * nfb);
  const int ns = (int)op->aux_streams.size();
  if (ns > 0) {
    HHG_CUDA_TRY(cudaEventRecord(op->aux_events[0], s));
    for (int i = 0; i < ns; ++i) HHG_CUDA_TRY(cudaStreamWaitEvent(op->aux_streams[i], op->aux_events[0], 0));
  }
  for (int m = 0; m < nm; ++m) {
    const cudaStream_t sm = ns > 0 ? op->aux_streams[m % ns] : s;
    if (op->bc == HHG_DIRICHLET)
      p2_quad_kernel<A, true><<<grid, 256, p2q_smem<A>(), sm>>>(w[m], cst + m, st + m, ix, tt.d, (int)tt.n, tt.kchunk,
                                                                nfb, I->d_pstart, xs, x, y, op->npts);
    else
      p2_quad_kernel<A, false><<<grid, 256, p2q_smem<A>(), sm>>>(w[m], cst + m, st + m, ix, tt.d, (int)tt.n, tt.kchunk,
                                                                 nfb, I->d_pstart, xs, x, y, op->npts);
    HHG_CUDA_TRY(cudaGetLastError());
  }
  for (int i = 0; i < ns; ++i) {
    HHG_CUDA_TRY(cudaEventRecord(op->aux_events[1 + i], op->aux_streams[i]));
    HHG_CUDA_TRY(cudaStreamWaitEvent(s, op->aux_events[1 + i], 0));
  }
  return HHG_OK;
}

template <typename T>
int launch_apply(const hhg_op* op, const T* x, T* y, cudaStream_t s) {
  const int64_t V = lattice_size(op->N);
  const int nm = op->mesh->nmacro();
  // precomputed variant: local matrices stored in this dtype
  if (op->d_elem && op->elem_dtype == (sizeof(T) == 8 ? HHG_F64 : HHG_F32)) return launch_march_stored<T>(op, x, y, s);
  if (op->kind == HHG_DIFFUSION && op->degree == 1 && op->coeff.type == HHG_COEFF_CONST) {
    (void)V;
    const Interface* I = op->itf;
    if (sizeof(T) == 8 && op->d_p1df) {
      // FP64 vectors in double-float arithmetic: split x once, then the stencil on the FP32 pipes
      const int64_t n = op->npts;
      split_double_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
          n, (const double*)x, (float2*)op->d_dfx);
      dim3 grid((unsigned)I->ncta, nm);
      if (op->bc == HHG_DIRICHLET)
        p1_gather_df_kernel<true><<<grid, 256, 0, s>>>((const OpConst<double>*)op->d_const64, (const float2*)op->d_p1df,
                                                       I->d_cta_plane, I->d_cta_start, I->d_pstart, (const double*)x,
                                                       (const float2*)op->d_dfx, (double*)y);
      else
        p1_gather_df_kernel<false><<<grid, 256, 0, s>>>((const OpConst<double>*)op->d_const64, (const float2*)op->d_p1df,
                                                        I->d_cta_plane, I->d_cta_start, I->d_pstart, (const double*)x,
                                                        (const float2*)op->d_dfx, (double*)y);
      HHG_CUDA_TRY(cudaGetLastError());
      return HHG_OK;
    }
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
    const OpConst<float>* cf = (const OpConst<float>*)op->d_const32;
    const TileTasks& tt = I->tile[kClimbPT == 4 ? 0 : 1];
    // face blocks: slices 0-5 need tri(N) threads each, the top planes at most V(kP1ClimbTop - 1) <= 256
    static_assert(kP1ClimbTop * (kP1ClimbTop + 1) * (kP1ClimbTop + 2) / 6 <= 256, "top planes exceed one block");
    const int nfb = (int)((tri_host(op->N) + 255) / 256);
    const unsigned grid = (unsigned)(tt.n + (int64_t)nm * (6 * nfb + 1));
    if (op->bc == HHG_DIRICHLET)
      p1_climb_f32_kernel<kClimbPT, true><<<grid, 256, 0, s>>>(cf, tt.d, (int)tt.n, tt.kchunk, nfb, I->d_pstart,
                                                               (const float*)x, (float*)y);
    else
      p1_climb_f32_kernel<kClimbPT, false><<<grid, 256, 0, s>>>(cf, tt.d, (int)tt.n, tt.kchunk, nfb, I->d_pstart,
                                                                (const float*)x, (float*)y);
    HHG_CUDA_TRY(cudaGetLastError());
    return HHG_OK;
  }
  // P2 constant coefficient: stencil rows (28.75 FMA per point against about 74 in element form)
  // from shared-memory plane tiles.  FP32 and double-float: two planes per step, one launch per macro
  // with its weights in the parameter bank (p2_quad_kernel); small lattices, the coarse levels of
  // multigrid, run one marching launch (FP32) or the FP64 tile kernel instead (there a launch costs
  // more than the work).  FP64: one plane per step, all macros in one launch (p2_tile_kernel; in
  // FP64 the few CTAs of a small march would leave the FP64 pipes of most SMs idle).
  if (op->kind == HHG_DIFFUSION && op->degree == 2 && op->coeff.type == HHG_COEFF_CONST && op->d_p2st64 &&
      op->N > 32) {
    if constexpr (sizeof(T) == 4) return launch_p2_quad<P2QF32>(op, op->h_p2w32.data(), x, x, y, s);
    if constexpr (sizeof(T) == 8) {
      if (!op->h_p2wdf.empty()) {
        const int64_t n = op->npts;
        split_double_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            n, (const double*)x, (float2*)op->d_dfx);
        HHG_CUDA_TRY(cudaGetLastError());
        return launch_p2_quad<P2QDF>(op, op->h_p2wdf.data(), (const float2*)op->d_dfx, x, y, s);
      }
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (op->kind == HHG_DIFFUSION && op->degree == 2 && op->coeff.type == HHG_COEFF_CONST && op->d_p2st64) {
      const Interface* I = op->itf;
      const P2Stencil<T>* st = (const P2Stencil<T>*)op->d_p2st64;
      constexpr int TI = 64;
      const TileTasks& tt = I->tile[1];
      constexpr size_t smem = p2_tile_smem<T, TI>();
      static_assert(smem <= 48 * 1024, "P2 tile exceeds the default dynamic shared memory");
      const P2StencilIndex* ix = (const P2StencilIndex*)op->d_p2idx;
      static_assert(smem >= sizeof(int) * (kP2StTotal + 9), "face blocks stage the stencil index in the tile's shared memory");
      const int nfb = (int)((tri_host(op->N) + 255) / 256);
      const unsigned grid = (unsigned)(tt.n + (int64_t)nm * 4 * nfb);
      if (op->bc == HHG_DIRICHLET)
        p2_tile_kernel<T, TI, true><<<grid, 256, smem, s>>>(dconst<T>(op), st, ix, tt.d, (int)tt.n, tt.kchunk, nfb,
                                                            I->d_pstart, x, y);
      else
        p2_tile_kernel<T, TI, false><<<grid, 256, smem, s>>>(dconst<T>(op), st, ix, tt.d, (int)tt.n, tt.kchunk, nfb,
                                                             I->d_pstart, x, y);
      HHG_CUDA_TRY(cudaGetLastError());
      return HHG_OK;
    }
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
  cudaFree(d_n1_64);
  cudaFree(d_n1_32);
  cudaFree(d_p2st64);
  cudaFree(d_p2st32);
  cudaFree(d_p2idx);
  cudaFree(d_elem);
  cudaFree(d_face);
  cudaFree(d_p1df);
  cudaFree(d_dfx);
  for (cudaStream_t t : aux_streams) cudaStreamDestroy(t);
  for (cudaEvent_t e : aux_events) cudaEventDestroy(e);
}

static int check_dtype(int dtype) {
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "dtype must be HHG_F32 or HHG_F64");
  return HHG_OK;
}

static int check_one_field(const hhg_coeff_t& c, int dtype) {
  if (c.type != HHG_COEFF_FIELD_P1 && c.type != HHG_COEFF_FIELD_P2) return HHG_OK;
  if (!c.field) return fail(HHG_E_ARG, "coefficient field pointer is null");
  if (c.field_dtype != dtype)
    return fail(HHG_E_ARG, "coefficient field dtype %d differs from the apply dtype %d", c.field_dtype, dtype);
  return HHG_OK;
}
static int check_field(const hhg_op* op, int dtype) {
  HHG_TRY(check_one_field(op->coeff, dtype));
  if (op->kind == HHG_CURLCURL) HHG_TRY(check_one_field(op->coeff2, dtype));
  return HHG_OK;
}


// Stencils of the P2 constant-coefficient operator from the hoisted class matrices A_o.  The
// structural neighbours of a parity class are the node offsets of all micro-tets that have a node
// of that parity; the weights for parity p and zero mask z are accumulated over the micro-tets
// around one representative point with that parity and mask in a virtual macro of 8 cubes per
// edge (the micro-tets around a point are fixed by its parity and the faces it lies on).
static int p2_node(int o, int a, int d) {
  return a < 4 ? 2 * kClassOffsets[o][a][d] : kClassOffsets[o][kP2Edges[a - 4][0]][d] + kClassOffsets[o][kP2Edges[a - 4][1]][d];
}

static int build_p2_stencil(const hhg_op* op, P2StencilIndex& ix, std::vector<P2Stencil<double>>& W) {
  std::vector<std::array<int, 3>> lists[8];
  for (int o = 0; o < 6; ++o)
    for (int a = 0; a < 10; ++a) {
      const int par = (p2_node(o, a, 0) & 1) | ((p2_node(o, a, 1) & 1) << 1) | ((p2_node(o, a, 2) & 1) << 2);
      for (int b = 0; b < 10; ++b) {
        const std::array<int, 3> d = {p2_node(o, b, 0) - p2_node(o, a, 0), p2_node(o, b, 1) - p2_node(o, a, 1),
                                      p2_node(o, b, 2) - p2_node(o, a, 2)};
        if (std::find(lists[par].begin(), lists[par].end(), d) == lists[par].end()) lists[par].push_back(d);
      }
    }
  int tot = 0;
  for (int par = 0; par < 8; ++par) {
    std::sort(lists[par].begin(), lists[par].end(), [](const std::array<int, 3>& u, const std::array<int, 3>& v) {
      return std::make_tuple(u[2], u[1], u[0]) < std::make_tuple(v[2], v[1], v[0]);
    });
    ix.start[par] = tot;
    for (auto& d : lists[par]) {
      if (tot >= kP2StTotal) return fail(HHG_E_UNSUPPORTED, "P2 stencil: more structural entries than expected");
      ix.off[tot++] = (d[0] + 2) | ((d[1] + 2) << 4) | ((d[2] + 2) << 8);
    }
  }
  ix.start[8] = tot;
  if (tot != kP2StTotal) return fail(HHG_E_UNSUPPORTED, "P2 stencil: %d structural entries, expected %d", tot, kP2StTotal);
  // the tile kernel unrolls the same lists at compile time: both orders must agree entry by entry
  for (int par = 0; par < 8; ++par) {
    const P2OffList L = p2_struct_list(par);
    if (L.n != ix.start[par + 1] - ix.start[par]) return fail(HHG_E_UNSUPPORTED, "P2 stencil: list size mismatch");
    for (int d = 0; d < L.n; ++d)
      if (L.off[d] != ix.off[ix.start[par] + d]) return fail(HHG_E_UNSUPPORTED, "P2 stencil: list order mismatch");
  }
  const int nv = 8, Nv = 2 * nv;
  W.assign(op->mesh->nmacro(), P2Stencil<double>{});
  for (int m = 0; m < op->mesh->nmacro(); ++m) {
    std::memset(&W[m], 0, sizeof(P2Stencil<double>));
    const OpConst<double>& c = op->h_const[m];
    for (int par = 0; par < 8; ++par)
      for (int z = 0; z < 15; ++z) {
        // representative point: coordinate d is 0 on face d+1, else 2 + parity; on face 0 the
        // last free coordinate closes i + j + k = Nv
        int P[3], last = -1;
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          const int pd = (par >> d) & 1;
          if ((z >> (d + 1)) & 1) {
            if (pd) ok = false;
            P[d] = 0;
          } else {
            P[d] = 2 + pd;
            last = d;
          }
        }
        if (!ok) continue;
        if (z & 1) {
          if (last < 0) continue;
          int rest = 0;
          for (int d = 0; d < 3; ++d)
            if (d != last) rest += P[d];
          P[last] = Nv - rest;
          if ((P[last] & 1) != ((par >> last) & 1) || P[last] < 2) continue;
        }
        for (int ck = 0; ck < nv; ++ck)
          for (int cj = 0; cj + ck < nv; ++cj)
            for (int ci = 0; ci + cj + ck < nv; ++ci)
              for (int o = 0; o < 6; ++o) {
                if (ci + cj + ck > nv - 1 - kClassShrink[o]) continue;
                const int cc[3] = {ci, cj, ck};
                for (int a = 0; a < 10; ++a) {
                  if (2 * cc[0] + p2_node(o, a, 0) != P[0] || 2 * cc[1] + p2_node(o, a, 1) != P[1] ||
                      2 * cc[2] + p2_node(o, a, 2) != P[2])
                    continue;
                  for (int b = 0; b < 10; ++b) {
                    const std::array<int, 3> d = {p2_node(o, b, 0) - p2_node(o, a, 0),
                                                  p2_node(o, b, 1) - p2_node(o, a, 1),
                                                  p2_node(o, b, 2) - p2_node(o, a, 2)};
                    const auto it = std::find(lists[par].begin(), lists[par].end(), d);
                    W[m].w[z][ix.start[par] + (int)(it - lists[par].begin())] += c.A[o][a][b];
                  }
                }
              }
      }
  }
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
  if (kind == HHG_DIFFUSION && degree == 2 && coeff->type == HHG_COEFF_CONST) {
    P2StencilIndex ix;
    std::vector<P2Stencil<double>> w64;
    HHG_TRY(build_p2_stencil(op.get(), ix, w64));
    std::vector<P2Stencil<float>> w32(nm);
    op->h_p2w32.resize(nm);
    for (int m = 0; m < nm; ++m) {
      for (int z = 0; z < 16; ++z)
        for (int t = 0; t < kP2StTotal; ++t) w32[m].w[z][t] = (float)w64[m].w[z][t];
      for (int t = 0; t < kP2StTotal; ++t) op->h_p2w32[m].w[t] = w32[m].w[0][t];
    }
    HHG_CUDA_TRY(cudaMalloc(&op->d_p2idx, sizeof(P2StencilIndex)));
    HHG_CUDA_TRY(cudaMemcpy(op->d_p2idx, &ix, sizeof(P2StencilIndex), cudaMemcpyHostToDevice));
    HHG_CUDA_TRY(cudaMalloc(&op->d_p2st64, sizeof(P2Stencil<double>) * nm));
    HHG_CUDA_TRY(cudaMalloc(&op->d_p2st32, sizeof(P2Stencil<float>) * nm));
    HHG_CUDA_TRY(cudaMemcpy(op->d_p2st64, w64.data(), sizeof(P2Stencil<double>) * nm, cudaMemcpyHostToDevice));
    HHG_CUDA_TRY(cudaMemcpy(op->d_p2st32, w32.data(), sizeof(P2Stencil<float>) * nm, cudaMemcpyHostToDevice));
    HHG_TRY(p2_quad_prepare());
    if (nm > 1) {
      const int ns = std::min(nm, kP2QStreams);
      for (int i = 0; i < ns; ++i) {
        cudaStream_t t;
        HHG_CUDA_TRY(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
        op->aux_streams.push_back(t);
      }
      for (int i = 0; i <= ns; ++i) {
        cudaEvent_t e;
        HHG_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        op->aux_events.push_back(e);
      }
    }
  }
  HHG_TRY(alloc_face_scratch(op.get()));
  HHG_TRY(noalloc_prepare());
  *out = op.release();
  return HHG_OK;
}

extern "C" int hhg_op_set_fp64_arith(hhg_op_t* op, int mode) {
  clear_error();
  if (!op) return fail(HHG_E_ARG, "set_fp64_arith: null op");
  if (mode != HHG_FP64_NATIVE && mode != HHG_FP64_DOUBLE_FLOAT) return fail(HHG_E_ARG, "set_fp64_arith: bad mode");
  const bool set = op->d_dfx != nullptr;
  if (mode == HHG_FP64_NATIVE) {
    if (set) {
      HHG_CUDA_TRY(cudaDeviceSynchronize());   // no apply in flight may still read them
      cudaFree(op->d_p1df);
      cudaFree(op->d_dfx);
    }
    op->d_p1df = op->d_dfx = nullptr;
    op->h_p2wdf.clear();
    return HHG_OK;
  }
  const bool p1 = op->kind == HHG_DIFFUSION && op->degree == 1 && op->coeff.type == HHG_COEFF_CONST;
  const bool p2 = op->kind == HHG_DIFFUSION && op->degree == 2 && op->coeff.type == HHG_COEFF_CONST && op->d_p2st64;
  if (!p1 && !p2)
    return fail(HHG_E_UNSUPPORTED, "set_fp64_arith: double-float arithmetic exists for P1 and P2 constant-coefficient "
                                   "diffusion only");
  if (set) return HHG_OK;
  // the weights split into FP32 pairs per macro (hi = the value rounded to FP32, lo = the rest), and
  // the scratch of the split input vector
  const int nm = op->mesh->nmacro();
  auto split = [](double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  };
  void *dw = nullptr, *dx = nullptr;
  std::vector<hhg::P2ParamWDF> w2;
  if (p1) {
    std::vector<float2> w(16 * (size_t)nm, make_float2(0.0f, 0.0f));
    for (int m = 0; m < nm; ++m)
      for (int d = 0; d < 15; ++d) w[16 * m + d] = split(op->h_const[m].S[d]);
    HHG_CUDA_TRY(cudaMalloc(&dw, sizeof(float2) * w.size()));
    HHG_CUDA_TRY(cudaMemcpy(dw, w.data(), sizeof(float2) * w.size(), cudaMemcpyHostToDevice));
  } else {
    std::vector<P2Stencil<double>> w64(nm);
    HHG_CUDA_TRY(cudaMemcpy(w64.data(), op->d_p2st64, sizeof(P2Stencil<double>) * nm, cudaMemcpyDeviceToHost));
    w2.resize(nm);
    for (int m = 0; m < nm; ++m)
      for (int t = 0; t < kP2StTotal; ++t) w2[m].w[t] = split(w64[m].w[0][t]);
  }
  if (cudaMalloc(&dx, sizeof(float2) * (size_t)op->npts) != cudaSuccess) {
    cudaFree(dw);
    return fail(HHG_E_OOM, "set_fp64_arith: no device memory for the split vector");
  }
  op->d_p1df = dw;
  op->d_dfx = dx;
  op->h_p2wdf = std::move(w2);
  return HHG_OK;
}

extern "C" int hhg_op_destroy(hhg_op_t* op) {
  delete op;
  return HHG_OK;
}

extern "C" int hhg_op_drop_element_matrices(hhg_op_t* op) {
  clear_error();
  if (!op) return fail(HHG_E_ARG, "drop_element_matrices: null op");
  if (op->d_elem) {
    HHG_CUDA_TRY(cudaDeviceSynchronize());   // no apply in flight may still read them
    cudaFree(op->d_elem);
  }
  op->d_elem = nullptr;
  op->elem_dtype = -1;
  return HHG_OK;
}

extern "C" int hhg_op_store_element_matrices(hhg_op_t* op, int dtype, void* stream) {
  clear_error();
  if (!op) return fail(HHG_E_ARG, "store_element_matrices: null op");
  HHG_TRY(check_dtype(dtype));
  const bool n1 = op->kind == HHG_CURLCURL;
  if (!n1 && (op->kind != HHG_DIFFUSION || !(op->coeff.type == HHG_COEFF_SIN3 ||
                                             (op->coeff.type == HHG_COEFF_FIELD_P1 && op->degree == 1) ||
                                             (op->coeff.type == HHG_COEFF_FIELD_P2 && op->degree == 2))))
    return fail(HHG_E_UNSUPPORTED, "store_element_matrices: needs a CURLCURL op or a DIFFUSION op with a SIN3 or FIELD "
                                   "coefficient");
  for (const hhg_coeff_t* cf : {&op->coeff, &op->coeff2})
    if ((cf->type == HHG_COEFF_FIELD_P1 || cf->type == HHG_COEFF_FIELD_P2) && cf->field_dtype != dtype &&
        (cf == &op->coeff || n1))
      return fail(HHG_E_ARG, "store_element_matrices: the coefficient fields must have the stored dtype");
  HHG_TRY(hhg_op_drop_element_matrices(op));
  const int64_t ncubes = (int64_t)op->n * (op->n + 1) * (op->n + 2) / 6;   // V(2^level - 1)
  const int ne = n1 ? kN1Sym : (op->degree == 1 ? 1 : 55);
  const size_t bytes = (size_t)op->mesh->nmacro() * 6 * ne * ncubes * (dtype == HHG_F64 ? 8 : 4);
  if (cudaMalloc(&op->d_elem, bytes) != cudaSuccess) {
    cudaGetLastError();
    op->d_elem = nullptr;
    return fail(HHG_E_OOM, "store_element_matrices: %zu bytes of device memory", bytes);
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int rc = n1 ? (dtype == HHG_F64 ? launch_elem_store_n1<double>(op, (double*)op->d_elem, s)
                                       : launch_elem_store_n1<float>(op, (float*)op->d_elem, s))
                    : (dtype == HHG_F64 ? launch_elem_store<double>(op, (double*)op->d_elem, s)
                                        : launch_elem_store<float>(op, (float*)op->d_elem, s));
  if (rc != HHG_OK) {
    cudaFree(op->d_elem);
    op->d_elem = nullptr;
    return rc;
  }
  op->elem_dtype = dtype;
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
  HHG_TRY(hhg_op_drop_element_matrices(op));   // they were integrated with the old field
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
  if (op->kind == HHG_CURLCURL) {
    if (nrhs != 1) return fail(HHG_E_ARG, "op_apply: the curl-curl operator takes nrhs = 1");
    if (dtype == HHG_F64) {
      HHG_TRY(launch_n1<double>(op, (const double*)x, (double*)y, s));
      HHG_TRY(launch_interface_sum_signed<double>(itf, (double*)y, op->bc == HHG_DIRICHLET, s));
    } else {
      HHG_TRY(launch_n1<float>(op, (const float*)x, (float*)y, s));
      HHG_TRY(launch_interface_sum_signed<float>(itf, (float*)y, op->bc == HHG_DIRICHLET, s));
    }
    return HHG_OK;
  }
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
  if (op->kind != HHG_DIFFUSION && op->kind != HHG_CURLCURL)
    return fail(HHG_E_UNSUPPORTED, "op_diagonal: scalar diffusion and curl-curl operators only");
  HHG_TRY(check_field(op, dtype));
  cudaStream_t s = (cudaStream_t)stream;
  const Interface* itf = nullptr;
  HHG_TRY(op->mesh->interface(op->level, op->degree, &itf));
  if (op->kind == HHG_CURLCURL) {
    // the diagonal does not depend on the orientation of an edge: the copies add without signs
    if (dtype == HHG_F64) {
      HHG_TRY(launch_n1_diag<double>(op, (double*)d, s));
      HHG_TRY(launch_interface_sum<double>(itf, (double*)d, 1, op->bc == HHG_DIRICHLET, s));
    } else {
      HHG_TRY(launch_n1_diag<float>(op, (float*)d, s));
      HHG_TRY(launch_interface_sum<float>(itf, (float*)d, 1, op->bc == HHG_DIRICHLET, s));
    }
    return HHG_OK;
  }
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

// ---------------------------------------------------------------------------
// Nedelec curl-curl + mass operator (Eq. N1): hoisted per-class edge matrices
// ---------------------------------------------------------------------------
namespace hhg {
// int_T lambda^m = |T| 3! prod(m_a!) / (|m| + 3)!, here |m| = 3: |T| 6 prod(m_a!) / 720
static double tri_int(int x, int y, int z, double vol) {
  int m[4] = {0, 0, 0, 0};
  m[x]++;
  m[y]++;
  m[z]++;
  double num = 1.0;
  for (int a = 0; a < 4; ++a)
    for (int t = 2; t <= m[a]; ++t) num *= t;
  return vol * 6.0 * num / 720.0;
}

static void build_n1(hhg_op* op, std::vector<N1Const<double>>& out) {
  const hhg_mesh* mesh = op->mesh;
  out.assign(mesh->nmacro(), N1Const<double>{});
  for (int m = 0; m < mesh->nmacro(); ++m) {
    N1Const<double>& q = out[m];
    std::memset(&q, 0, sizeof(q));
    q.vbase = (int64_t)m * lattice_size(op->n);
    const OpConst<double>& c = op->h_const[m];
    for (int o = 0; o < 6; ++o) {
      // grad lambda_a = J^{-T} grad_ref lambda_a
      const double gl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      double G[4][3];
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) {
          double s = 0;
          for (int e = 0; e < 3; ++e) s += c.Jinv[o][e * 3 + d] * gl[a][e];
          G[a][d] = s;
        }
      const double vol = c.adet[o] / 6.0;
      double cu[6][3], sg[6];
      for (int e = 0; e < 6; ++e) {
        const int a = kP2Edges[e][0], b = kP2Edges[e][1];
        cu[e][0] = 2.0 * (G[a][1] * G[b][2] - G[a][2] * G[b][1]);
        cu[e][1] = 2.0 * (G[a][2] * G[b][0] - G[a][0] * G[b][2]);
        cu[e][2] = 2.0 * (G[a][0] * G[b][1] - G[a][1] * G[b][0]);
        // orientation of local edge a -> b against the canonical lattice direction of its midpoint
        int vec[3], par[3];
        for (int d = 0; d < 3; ++d) {
          vec[d] = kClassOffsets[o][b][d] - kClassOffsets[o][a][d];
          par[d] = (kClassOffsets[o][a][d] + kClassOffsets[o][b][d]) & 1;
        }
        int can[3] = {par[0], par[1], par[2]};
        if (par[0] && par[1] && !par[2]) can[1] = -1;
        if (par[0] && !par[1] && par[2]) can[2] = -1;
        if (!par[0] && par[1] && par[2]) can[2] = -1;
        if (par[0] && par[1] && par[2]) can[1] = -1;
        sg[e] = (vec[0] == can[0] && vec[1] == can[1] && vec[2] == can[2]) ? 1.0 : -1.0;
      }
      auto dot = [](const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
      for (int e = 0; e < 6; ++e)
        for (int f = e; f < 6; ++f) {
          const double s = sg[e] * sg[f];
          q.C[o][n1_sym(e, f)] = s * vol * dot(cu[e], cu[f]);
          const int a = kP2Edges[e][0], b = kP2Edges[e][1], cc = kP2Edges[f][0], dd = kP2Edges[f][1];
          for (int v = 0; v < 4; ++v)
            q.M[o][v][n1_sym(e, f)] =
                s * (tri_int(v, a, cc, vol) * dot(G[b], G[dd]) - tri_int(v, a, dd, vol) * dot(G[b], G[cc]) -
                     tri_int(v, b, cc, vol) * dot(G[a], G[dd]) + tri_int(v, b, dd, vol) * dot(G[a], G[cc]));
        }
    }
  }
}
}  // namespace hhg

extern "C" int hhg_op_create_curlcurl(hhg_mesh_t* mesh, int level, const hhg_coeff_t* alpha, const hhg_coeff_t* beta,
                                      int bc, hhg_op_t** out) {
  clear_error();
  if (!mesh || !alpha || !beta || !out) return fail(HHG_E_ARG, "op_create_curlcurl: null pointer");
  *out = nullptr;
  if (level < 0) level = mesh->level;
  if (level > mesh->level) return fail(HHG_E_ARG, "op_create_curlcurl: level %d above the mesh's %d", level, mesh->level);
  if (bc != HHG_DIRICHLET && bc != HHG_NEUMANN) return fail(HHG_E_ARG, "op_create_curlcurl: unknown boundary mode");
  for (const hhg_coeff_t* c : {alpha, beta})
    if (c->type != HHG_COEFF_CONST && c->type != HHG_COEFF_FIELD_P1)
      return fail(HHG_E_UNSUPPORTED, "op_create_curlcurl: alpha and beta must be CONST or FIELD_P1");
  std::unique_ptr<hhg_op> op(new hhg_op());
  op->mesh = mesh;
  op->level = level;
  op->kind = HHG_CURLCURL;
  op->degree = 2;   // edge DoFs live in the doubled lattice
  op->bc = bc;
  op->quad_degree = 2;
  op->coeff = *alpha;
  op->coeff2 = *beta;
  op->n = 1 << level;
  op->N = 2 << level;
  op->npts = (int64_t)mesh->nmacro() * lattice_size(op->N);
  HHG_TRY(quad_rule(2, &op->rule));
  const Interface* itf1 = nullptr;
  HHG_TRY(mesh->interface(level, 1, &itf1));
  HHG_TRY(mesh->interface(level, 2, &op->itf));
  hhg_coeff_t cc{HHG_COEFF_CONST, 1.0, nullptr, HHG_F64};
  op->coeff = cc;   // geometry tables only
  build_const(op.get());
  op->coeff = *alpha;
  std::vector<N1Const<double>> n64;
  build_n1(op.get(), n64);
  const int nm = mesh->nmacro();
  std::vector<N1Const<float>> n32(nm);
  for (int m = 0; m < nm; ++m) {
    std::memset(&n32[m], 0, sizeof(N1Const<float>));
    n32[m].vbase = n64[m].vbase;
    for (int o = 0; o < 6; ++o)
      for (int t = 0; t < kN1Sym; ++t) {
        n32[m].C[o][t] = (float)n64[m].C[o][t];
        for (int v = 0; v < 4; ++v) n32[m].M[o][v][t] = (float)n64[m].M[o][v][t];
      }
  }
  std::vector<OpConst<float>> c32(nm);
  for (int m = 0; m < nm; ++m) c32[m] = convert_const<float>(op->h_const[m]);
  HHG_CUDA_TRY(cudaMalloc(&op->d_const64, sizeof(OpConst<double>) * nm));
  HHG_CUDA_TRY(cudaMalloc(&op->d_const32, sizeof(OpConst<float>) * nm));
  HHG_CUDA_TRY(cudaMalloc(&op->d_n1_64, sizeof(N1Const<double>) * nm));
  HHG_CUDA_TRY(cudaMalloc(&op->d_n1_32, sizeof(N1Const<float>) * nm));
  HHG_CUDA_TRY(cudaMemcpy(op->d_const64, op->h_const.data(), sizeof(OpConst<double>) * nm, cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(op->d_const32, c32.data(), sizeof(OpConst<float>) * nm, cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(op->d_n1_64, n64.data(), sizeof(N1Const<double>) * nm, cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(op->d_n1_32, n32.data(), sizeof(N1Const<float>) * nm, cudaMemcpyHostToDevice));
  HHG_TRY(alloc_face_scratch(op.get()));
  HHG_TRY(noalloc_prepare());
  *out = op.release();
  return HHG_OK;
}
