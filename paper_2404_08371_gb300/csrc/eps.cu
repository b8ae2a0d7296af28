// P2 vector "epsilon" operator a(u, v) = int 2 mu eps(u) : eps(v), eps(u) = (grad u + grad u^T)/2,
// applied to a batch of right-hand sides, and its adjoint in a P2 viscosity field mu.
//
// The paper names this form as the Taylor-Hood Stokes counterpart of its variable-coefficient
// diffusion (Section 7.4) and lists vector spaces as future work; the element computation follows
// Algorithm 1 with the fused local quadrature of Remark 4.1: per quadrature point the gradient of
// each velocity component is formed from its 10 nodal values (through barycentric coordinates),
// mapped with the hoisted per-class J^{-1} (Section 6.1), turned into the stress
// 2 mu eps(u) w |det J|, and tested against the basis gradients.
//
// Work per micro-tet and right-hand side is large (about 2.5e3 FP64 operations at 14 points), so
// the traversal favours simplicity over traffic: eight passes over the cubes of one index parity
// each (cubes of equal parity share no point, so plain read-modify-write accumulation is race
// free), one thread per (cube, right-hand side) with the right-hand side fastest so that loads of
// the [point][component][rhs] layout coalesce.
#include <algorithm>
#include <vector>

#include "hhg_internal.h"
#include "lattice.cuh"

namespace hhg {

__host__ __device__ constexpr int eedge(int e, int s) {
  constexpr int t[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  return t[e][s];
}

// Doubled-lattice offset of P2 node `a` of class o from 2 * (cube origin); in kernels, where o is a
// run-time value uniform over the warp, from the constant-memory class table.
__device__ __forceinline__ int enode_d(int o, int a, int d) {
  return a < 4 ? 2 * kClassOffsetsD[o][a][d]
               : kClassOffsetsD[o][eedge(a - 4, 0)][d] + kClassOffsetsD[o][eedge(a - 4, 1)][d];
}

// The reference gradient of a P2 component is affine in the barycentric coordinates:
// grad_ref u(lambda) = W0 + lambda_1 W1 + lambda_2 W2 + lambda_3 W3, formed once per micro-tet from
// W'_c = 4 u_c g_c + 4 sum_{edges (c, b)} u_(c,b) g_b - sum_a u_a g_a (g_a = grad_ref lambda_a),
// W0 = W'_0, Wc = W'_c - W'_0.
template <int B, typename T>
__device__ __forceinline__ void eps_add_g(T v[3], T f) {
  if (B == 0) {
    v[0] -= f;
    v[1] -= f;
    v[2] -= f;
  } else {
    v[B - 1] += f;
  }
}

template <typename T>
__device__ __forceinline__ void eps_grad_affine(const T* u, T W[4][3]) {
  const T U[3] = {u[1] - u[0], u[2] - u[0], u[3] - u[0]};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) W[a][d] = -U[d];
  eps_add_g<0>(W[0], T(4) * u[0]);
  eps_add_g<1>(W[1], T(4) * u[1]);
  eps_add_g<2>(W[2], T(4) * u[2]);
  eps_add_g<3>(W[3], T(4) * u[3]);
  // edges (0,1) (0,2) (0,3) (1,2) (1,3) (2,3): W'_a += 4 u_e g_b, W'_b += 4 u_e g_a
  eps_add_g<1>(W[0], T(4) * u[4]);
  eps_add_g<0>(W[1], T(4) * u[4]);
  eps_add_g<2>(W[0], T(4) * u[5]);
  eps_add_g<0>(W[2], T(4) * u[5]);
  eps_add_g<3>(W[0], T(4) * u[6]);
  eps_add_g<0>(W[3], T(4) * u[6]);
  eps_add_g<2>(W[1], T(4) * u[7]);
  eps_add_g<1>(W[2], T(4) * u[7]);
  eps_add_g<3>(W[1], T(4) * u[8]);
  eps_add_g<1>(W[3], T(4) * u[8]);
  eps_add_g<3>(W[2], T(4) * u[9]);
  eps_add_g<2>(W[3], T(4) * u[9]);
#pragma unroll
  for (int c = 1; c < 4; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) W[c][d] -= W[0][d];
}

// Testing over all quadrature points through the moments S_ab = sum_q lambda_b rho_a and
// R_a = sum_q rho_a (a, b = 1..3 given): y_a += 4 S_aa - R_a, y_(a,b) += 4 (S_ab + S_ba).
template <typename T>
__device__ __forceinline__ void eps_test_moments(const T S3[3][3], const T R3[3], T* y) {
  T S[4][4], R[4];
#pragma unroll
  for (int a = 1; a < 4; ++a) {
    R[a] = R3[a - 1];
#pragma unroll
    for (int b = 1; b < 4; ++b) S[a][b] = S3[a - 1][b - 1];
    S[a][0] = R[a] - S[a][1] - S[a][2] - S[a][3];
  }
  R[0] = -(R[1] + R[2] + R[3]);
#pragma unroll
  for (int b = 0; b < 4; ++b) S[0][b] = -(S[1][b] + S[2][b] + S[3][b]);
#pragma unroll
  for (int a = 0; a < 4; ++a) y[a] += T(4) * S[a][a] - R[a];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = eedge(e, 0), b = eedge(e, 1);
    y[4 + e] += T(4) * (S[a][b] + S[b][a]);
  }
}

// Index of the entry (c, d) of a symmetric 3 x 3 tensor stored as (0,0) (1,1) (2,2) (0,1) (0,2) (1,2).
__device__ __forceinline__ int eps_sym(int c, int d) { return c == d ? c : c + d + 2; }

// grad of component fields: G[c][d] = d u_c / d x_d = sum_e Jinv[e][d] ghat_c[e]
template <typename T>
__device__ __forceinline__ void phys_grad(const T* Ji, const T gh[3], T G[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) G[d] = Ji[0 * 3 + d] * gh[0] + Ji[1 * 3 + d] * gh[1] + Ji[2 * 3 + d] * gh[2];
}

// MODE 0: out += A u (all right-hand sides); MODE 2: out_m += sum_r g_r^T (dA/dmu_m) u_r.
// One CTA per task of its colour: up to cpb consecutive cubes of one row (cj, ck) of one macro,
// times the right-hand sides.  MODE 0 keeps each thread's affine gradient terms P (36 values) and
// nodal mu (10) in shared memory, column threadIdx.x of a [value][thread] array: the quadrature
// loop then holds only the 36 stress moments and one gradient in registers, which lets two CTAs
// (16 warps) share an SM to keep the FP64 pipes fed; reading P costs 36 shared loads per point
// against about 90 FP64 operations.
constexpr int kEpsThreads = 256;
template <typename T, bool FIELD>
constexpr size_t eps_apply_smem() { return (sizeof(T) * (36 + (FIELD ? kMaxQ : 0)) + sizeof(int) * 10) * kEpsThreads; }

template <typename T, int MODE, bool FIELD, bool DIR>
__global__ void __launch_bounds__(kEpsThreads, MODE == 0 ? 2 : 1) eps_color_kernel(const OpConst<T>* __restrict__ cst,
                                                         const int4* __restrict__ tasks, int color, int cpb,
                                                         int nrhs, T mu_const, const T* __restrict__ x,
                                                         const T* __restrict__ g, const T* __restrict__ mu,
                                                         T* __restrict__ out) {
  const int4 task = tasks[blockIdx.x];
  const int macro = task.w;
  const OpConst<T>& c = cst[macro];
  const int n = c.n, N = c.N;
  const int t = threadIdx.x;
  const int r = t % nrhs;
  const int ci = 2 * (task.x + t / nrhs) + (color & 1);
  const int cj = 2 * task.y + ((color >> 1) & 1);
  const int ck = 2 * task.z + ((color >> 2) & 1);
  const bool live = t / nrhs < cpb && ci + cj + ck <= n - 1;
  if (MODE == 0 && !live) return;
  if (MODE == 2 && __all_sync(0xffffffffu, !live)) return;
  const int64_t base = c.base;
  const int stride = 3 * nrhs;
  extern __shared__ __align__(16) unsigned char eps_smem_raw[];
  T* __restrict__ Ps = reinterpret_cast<T*>(eps_smem_raw) + threadIdx.x;   // MODE 0: P[v] at Ps[v * kEpsThreads]
  T* __restrict__ Ms = Ps + 36 * kEpsThreads;   // MODE 0, field: mu(x_q) w_q |det J| at the points
  int* __restrict__ Is = reinterpret_cast<int*>(reinterpret_cast<T*>(eps_smem_raw) + (FIELD ? 36 + kMaxQ : 36) * kEpsThreads) +
                         threadIdx.x;           // MODE 0: node indices
#pragma unroll 1
  for (int o = 0; o < 6; ++o) {
    const bool tet_ok = live && ci + cj + ck <= n - 1 - (o == 0 ? 0 : (o == 5 ? 2 : 1));
    if (MODE == 0 && !tet_ok) continue;
    int idx[10], masked = 0;   // bit a: node a reads as zero (Dirichlet point or no micro-tet)
    T m[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int pi = 2 * ci + enode_d(o, a, 0), pj = 2 * cj + enode_d(o, a, 1), pk = 2 * ck + enode_d(o, a, 2);
      idx[a] = tet_ok ? (int)packed_index(N, pi, pj, pk) : 0;
      if (MODE == 0) Is[a * kEpsThreads] = idx[a];
      if (!tet_ok || (DIR && on_dirichlet(c.bnd_table, N, pi, pj, pk))) masked |= 1 << a;
      if (MODE == 0 && FIELD) m[a] = __ldg(mu + base + idx[a]);
    }
    const T* Ji = c.Jinv[o];
    const T wdet = c.adet[o];
    if (MODE == 0 && FIELD) {
      // mu at the quadrature points, times the weight and |det J|, once per micro-tet
#pragma unroll 1
      for (int q = 0; q < c.nq; ++q) {
        T muq = T(0);
#pragma unroll
        for (int a = 0; a < 10; ++a) muq += c.psi[q][a] * m[a];
        Ms[q * kEpsThreads] = muq * c.w[q] * wdet;
      }
    }
    T dmu[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) dmu[a] = T(0);
    // physical gradients of the components, affine in lambda: G_c = P[c][0] + sum_b lambda_b P[c][b]
    // (MODE 0: one component at a time into shared memory, P[c][t][d] at Ps[(12 c + 3 t + d) kEpsThreads])
    T P[3][4][3], gv[3][10];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      T u[10], W[4][3];
#pragma unroll
      for (int a = 0; a < 10; ++a) {
        const int64_t e = (base + idx[a]) * stride + cc * nrhs + r;
        u[a] = (masked >> a) & 1 ? T(0) : __ldg(x + e);
        if (MODE == 2) gv[cc][a] = (masked >> a) & 1 ? T(0) : __ldg(g + e);
      }
      eps_grad_affine<T>(u, W);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        phys_grad<T>(Ji, W[t], P[cc][t]);
        if (MODE == 0)
#pragma unroll
          for (int d = 0; d < 3; ++d) Ps[(12 * cc + 3 * t + d) * kEpsThreads] = P[cc][t][d];
      }
    }
    if (MODE == 0) {
      // physical moments of the stress: Q[t][v] = sum_q lambda_t S_v (lambda_0 = 1), S = s (G + G^T)
      // = 2 mu eps(u) w |det J| symmetric, so only its six entries v = (0,0) (1,1) (2,2) (0,1) (0,2)
      // (1,2) are accumulated (the entry of (c, d) is eps_sym(c, d))
      T Q[4][6];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int v = 0; v < 6; ++v) Q[t][v] = T(0);
#pragma unroll 1
      for (int q = 0; q < c.nq; ++q) {
        const T l1 = c.lam[q][1], l2 = c.lam[q][2], l3 = c.lam[q][3];
        T G[3][3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const T* pc = Ps + (12 * cc + d) * kEpsThreads;
            G[cc][d] = fma(l3, pc[9 * kEpsThreads], fma(l2, pc[6 * kEpsThreads], fma(l1, pc[3 * kEpsThreads], pc[0])));
          }
        const T s = FIELD ? Ms[q * kEpsThreads] : mu_const * c.w[q] * wdet;
        const T s2 = s + s;
        T Sv[6];
        Sv[0] = s2 * G[0][0];
        Sv[1] = s2 * G[1][1];
        Sv[2] = s2 * G[2][2];
        Sv[3] = s * (G[0][1] + G[1][0]);
        Sv[4] = s * (G[0][2] + G[2][0]);
        Sv[5] = s * (G[1][2] + G[2][1]);
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          Q[0][v] += Sv[v];
          Q[1][v] = fma(l1, Sv[v], Q[1][v]);
          Q[2][v] = fma(l2, Sv[v], Q[2][v]);
          Q[3][v] = fma(l3, Sv[v], Q[3][v]);
        }
      }
      // y_c += sum_q (J^{-1} S_c) . grad_ref phi: map the moments back once, then test; the moments
      // go to shared memory (over P, no longer needed) so that one component at a time is in
      // registers, and each component is added to out as soon as it is formed
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int v = 0; v < 6; ++v) Ps[(6 * t + v) * kEpsThreads] = Q[t][v];
#pragma unroll 1
      for (int cc = 0; cc < 3; ++cc) {
        T R3[3], S3[3][3], yc[10], Qc[4][3];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int d = 0; d < 3; ++d) Qc[t][d] = Ps[(6 * t + eps_sym(cc, d)) * kEpsThreads];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          R3[e] = Ji[e * 3 + 0] * Qc[0][0] + Ji[e * 3 + 1] * Qc[0][1] + Ji[e * 3 + 2] * Qc[0][2];
#pragma unroll
          for (int b = 0; b < 3; ++b)
            S3[e][b] = Ji[e * 3 + 0] * Qc[b + 1][0] + Ji[e * 3 + 1] * Qc[b + 1][1] + Ji[e * 3 + 2] * Qc[b + 1][2];
        }
#pragma unroll
        for (int a = 0; a < 10; ++a) yc[a] = T(0);
        eps_test_moments<T>(S3, R3, yc);
#pragma unroll
        for (int a = 0; a < 10; ++a) out[(base + Is[a * kEpsThreads]) * stride + cc * nrhs + r] += yc[a];
      }
    } else {
      T Pg[3][4][3];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        T W[4][3];
        eps_grad_affine<T>(gv[cc], W);
#pragma unroll
        for (int t = 0; t < 4; ++t) phys_grad<T>(Ji, W[t], Pg[cc][t]);
      }
      for (int q = 0; q < c.nq; ++q) {
        const T l1 = c.lam[q][1], l2 = c.lam[q][2], l3 = c.lam[q][3];
        T G[3][3], Gg[3][3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            G[cc][d] = fma(l3, P[cc][3][d], fma(l2, P[cc][2][d], fma(l1, P[cc][1][d], P[cc][0][d])));
            Gg[cc][d] = fma(l3, Pg[cc][3][d], fma(l2, Pg[cc][2][d], fma(l1, Pg[cc][1][d], Pg[cc][0][d])));
          }
        T tq = T(0);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int d = 0; d < 3; ++d) tq += Gg[cc][d] * (G[cc][d] + G[d][cc]);
        tq *= c.w[q] * wdet;
#pragma unroll
        for (int a = 0; a < 10; ++a) dmu[a] += c.psi[q][a] * tq;
      }
    }
    if (MODE == 2) {
      // sum over the right-hand sides of this cube (consecutive lanes of one warp), one writer
#pragma unroll
      for (int a = 0; a < 10; ++a)
        for (int off = 1; off < nrhs; off <<= 1) dmu[a] += __shfl_xor_sync(0xffffffffu, dmu[a], off);
      if (tet_ok && r == 0) {
#pragma unroll
        for (int a = 0; a < 10; ++a) out[base + idx[a]] += dmu[a];
      }
    }
  }
}

// Dirichlet rows of the vector operator: y = x at every component and right-hand side.
template <typename T>
__global__ void eps_dirichlet_kernel(const OpConst<T>* __restrict__ cst, int per_point, const T* __restrict__ x,
                                     T* __restrict__ y) {
  const OpConst<T>& c = cst[blockIdx.y];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= dV(c.N)) return;
  int i, j, k;
  decode_point(p, c.N, i, j, k);
  if (!on_dirichlet(c.bnd_table, c.N, i, j, k)) return;
  for (int e = 0; e < per_point; ++e) y[(c.base + p) * per_point + e] = x[(c.base + p) * per_point + e];
}

template <typename T>
int launch_eps(const hhg_op* op, const OpConst<T>* cst, int mode, int nrhs, const T* x, const T* g, const T* mu,
               T* out, cudaStream_t s) {
  const int n = op->n;
  const int nm = op->mesh->nmacro();
  const int nh = (n + 1) / 2;   // cubes per parity class along an axis (upper bound)
  const int nz = nh;
  const bool field = op->coeff.type == HHG_COEFF_FIELD_P2;
  const T muc = (T)(op->coeff.type == HHG_COEFF_CONST ? op->coeff.value : 1.0);
  if (mode == 2 && (nrhs > 32 || (32 % nrhs) != 0))
    return fail(HHG_E_UNSUPPORTED, "epsilon adjoint: nrhs must divide 32");
  if (nrhs > 256) return fail(HHG_E_UNSUPPORTED, "epsilon: at most 256 right-hand sides per call");
  // tasks of live cubes per colour (cached in the operator for this number of cubes per CTA)
  const int cpb = kEpsThreads / nrhs;
  if (op->eps_cpb != cpb) {
    std::vector<int4> tv;
    int64_t off[9];
    for (int color = 0; color < 8; ++color) {
      off[color] = (int64_t)tv.size();
      const int px = color & 1, py = (color >> 1) & 1, pz = (color >> 2) & 1;
      for (int m = 0; m < nm; ++m)
        for (int kz = 0; kz < nz; ++kz)
          for (int jy = 0; jy < nh; ++jy) {
            const int rem = n - 1 - (2 * jy + py) - (2 * kz + pz) - px;   // room left for 2 ci'
            if (rem < 0) continue;
            const int len = rem / 2 + 1;                                   // live cubes of the row
            for (int st = 0; st < len; st += cpb) tv.push_back(int4{st, jy, kz, m});
          }
    }
    off[8] = (int64_t)tv.size();
    cudaFree(op->d_eps_tasks);
    op->d_eps_tasks = nullptr;
    op->eps_cpb = 0;
    HHG_CUDA_TRY(cudaMalloc(&op->d_eps_tasks, sizeof(int4) * std::max<size_t>(tv.size(), 1)));
    if (!tv.empty())
      HHG_CUDA_TRY(cudaMemcpy(op->d_eps_tasks, tv.data(), sizeof(int4) * tv.size(), cudaMemcpyHostToDevice));
    for (int c = 0; c < 9; ++c) op->eps_off[c] = off[c];
    op->eps_cpb = cpb;
  }
  const size_t bytes = sizeof(T) * (size_t)op->npts * (mode == 0 ? 3 * nrhs : 1);
  HHG_CUDA_TRY(cudaMemsetAsync(out, 0, bytes, s));
  for (int color = 0; color < 8; ++color) {
    const unsigned grid = (unsigned)(op->eps_off[color + 1] - op->eps_off[color]);
    if (grid == 0) continue;
    const int4* tk = op->d_eps_tasks + op->eps_off[color];
#define HHG_EPS(M, F, D)                                                                                       \
  do {                                                                                                       \
    const size_t sm = M == 0 ? eps_apply_smem<T, F>() : 0;                                                   \
    if (sm > 48 * 1024)                                                                                      \
      HHG_CUDA_TRY(cudaFuncSetAttribute(eps_color_kernel<T, M, F, D>,                                      \
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));              \
    eps_color_kernel<T, M, F, D><<<grid, kEpsThreads, sm, s>>>(cst, tk, color, cpb, nrhs, muc, x, g, mu, out); \
  } while (0)
    const bool dir = op->bc == HHG_DIRICHLET;
    if (mode == 0) {
      if (field) {
        if (dir) HHG_EPS(0, true, true); else HHG_EPS(0, true, false);
      } else {
        if (dir) HHG_EPS(0, false, true); else HHG_EPS(0, false, false);
      }
    } else {
      if (dir) HHG_EPS(2, true, true); else HHG_EPS(2, true, false);
    }
#undef HHG_EPS
    HHG_CUDA_TRY(cudaGetLastError());
  }
  if (mode == 0 && op->bc == HHG_DIRICHLET) {
    dim3 g2((unsigned)((lattice_size(op->N) + 255) / 256), nm);
    eps_dirichlet_kernel<T><<<g2, 256, 0, s>>>(cst, 3 * nrhs, x, out);
    HHG_CUDA_TRY(cudaGetLastError());
  }
  return HHG_OK;
}

template int launch_eps<double>(const hhg_op*, const OpConst<double>*, int, int, const double*, const double*,
                                const double*, double*, cudaStream_t);
template int launch_eps<float>(const hhg_op*, const OpConst<float>*, int, int, const float*, const float*,
                               const float*, float*, cudaStream_t);

}  // namespace hhg
