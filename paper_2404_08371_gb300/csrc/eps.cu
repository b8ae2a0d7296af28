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
#include "hhg_internal.h"
#include "lattice.cuh"

namespace hhg {

__host__ __device__ constexpr int eoff(int o, int v, int d) {
  constexpr int t[6][4][3] = {
      {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {1, 1, 0}},
      {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {0, 1, 1}}, {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {0, 0, 1}},
      {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {1, 0, 0}}, {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}}};
  return t[o][v][d];
}
__host__ __device__ constexpr int eedge(int e, int s) {
  constexpr int t[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  return t[e][s];
}
// Doubled-lattice offset of P2 node `a` of class o from 2 * (cube origin).
__host__ __device__ constexpr int enode(int o, int a, int d) {
  return a < 4 ? 2 * eoff(o, a, d) : eoff(o, eedge(a - 4, 0), d) + eoff(o, eedge(a - 4, 1), d);
}

// grad_ref u of one component at a quadrature point from its 10 nodal values, and the test
// y_i += r . grad_ref phi_i, with 4 lambda and 4 lambda - 1 tabulated per point.
template <typename T>
__device__ __forceinline__ void ref_grad10_q(const T* u, const T* L4, const T* L4m1, T g[3]) {
  T s[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) s[a] = u[a] * L4m1[a];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = eedge(e, 0), b = eedge(e, 1);
    s[a] = fma(u[4 + e], L4[b], s[a]);
    s[b] = fma(u[4 + e], L4[a], s[b]);
  }
  g[0] = s[1] - s[0];
  g[1] = s[2] - s[0];
  g[2] = s[3] - s[0];
}

template <typename T>
__device__ __forceinline__ void ref_test10_q(const T r[3], const T* L4, const T* L4m1, T* y) {
  const T rho[4] = {-(r[0] + r[1] + r[2]), r[0], r[1], r[2]};
#pragma unroll
  for (int a = 0; a < 4; ++a) y[a] = fma(L4m1[a], rho[a], y[a]);
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = eedge(e, 0), b = eedge(e, 1);
    y[4 + e] = fma(L4[a], rho[b], fma(L4[b], rho[a], y[4 + e]));
  }
}

// grad of component fields: G[c][d] = d u_c / d x_d = sum_e Jinv[e][d] ghat_c[e]
template <typename T>
__device__ __forceinline__ void phys_grad(const T* Ji, const T gh[3], T G[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) G[d] = Ji[0 * 3 + d] * gh[0] + Ji[1 * 3 + d] * gh[1] + Ji[2 * 3 + d] * gh[2];
}

// MODE 0: out += A u (all right-hand sides); MODE 2: out_m += sum_r g_r^T (dA/dmu_m) u_r.
template <typename T, int MODE, bool FIELD, bool DIR>
__global__ void __launch_bounds__(256) eps_color_kernel(const OpConst<T>* __restrict__ cst, int color, int nz,
                                                         int nrhs, T mu_const, const T* __restrict__ x,
                                                         const T* __restrict__ g, const T* __restrict__ mu,
                                                         T* __restrict__ out) {
  const int macro = blockIdx.z / nz;
  const OpConst<T>& c = cst[macro];
  const int n = c.n, N = c.N;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = t % nrhs;
  const int ci = 2 * (t / nrhs) + (color & 1);
  const int cj = 2 * blockIdx.y + ((color >> 1) & 1);
  const int ck = 2 * (blockIdx.z - macro * nz) + ((color >> 2) & 1);
  const bool live = ci + cj + ck <= n - 1;
  if (MODE == 0 && !live) return;
  if (MODE == 2 && __all_sync(0xffffffffu, !live)) return;
  const int64_t base = c.base;
  const int stride = 3 * nrhs;
  for (int o = 0; o < 6; ++o) {
    const bool tet_ok = live && ci + cj + ck <= n - 1 - (o == 0 ? 0 : (o == 5 ? 2 : 1));
    if (MODE == 0 && !tet_ok) continue;
    int64_t idx[10];
    T u[3][10], gv[3][10], m[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int pi = 2 * ci + enode(o, a, 0), pj = 2 * cj + enode(o, a, 1), pk = 2 * ck + enode(o, a, 2);
      idx[a] = tet_ok ? packed_index(N, pi, pj, pk) : 0;
      const bool masked = !tet_ok || (DIR && on_dirichlet(c.bnd_table, N, pi, pj, pk));
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        const int64_t e = (base + idx[a]) * stride + cc * nrhs + r;
        u[cc][a] = masked ? T(0) : __ldg(x + e);
        if (MODE == 2) gv[cc][a] = masked ? T(0) : __ldg(g + e);
      }
      m[a] = FIELD ? (tet_ok ? __ldg(mu + base + idx[a]) : T(0)) : mu_const;
    }
    const T* Ji = c.Jinv[o];
    const T wdet = c.adet[o];
    T y[3][10];
    T dmu[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      y[0][a] = y[1][a] = y[2][a] = T(0);
      dmu[a] = T(0);
    }
    for (int q = 0; q < c.nq; ++q) {
      const T* L4 = c.lam4[q];
      const T* L4m1 = c.lam4m1[q];
      T G[3][3];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        T gh[3];
        ref_grad10_q<T>(u[cc], L4, L4m1, gh);
        phys_grad<T>(Ji, gh, G[cc]);
      }
      if (MODE == 0) {
        T muq = T(0);
#pragma unroll
        for (int a = 0; a < 10; ++a) muq += c.psi[q][a] * m[a];
        const T s = muq * c.w[q] * wdet;
        // S = s (G + G^T) = 2 mu eps(u) w |det J|;  y_c += (J^{-1} S_c) . grad_ref phi
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          T Sc[3], rr[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) Sc[d] = s * (G[cc][d] + G[d][cc]);
#pragma unroll
          for (int e = 0; e < 3; ++e) rr[e] = Ji[e * 3 + 0] * Sc[0] + Ji[e * 3 + 1] * Sc[1] + Ji[e * 3 + 2] * Sc[2];
          ref_test10_q<T>(rr, L4, L4m1, y[cc]);
        }
      } else {
        T Gg[3][3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          T gh[3];
          ref_grad10_q<T>(gv[cc], L4, L4m1, gh);
          phys_grad<T>(Ji, gh, Gg[cc]);
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
    if (MODE == 0) {
#pragma unroll
      for (int a = 0; a < 10; ++a)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          const int64_t e = (base + idx[a]) * stride + cc * nrhs + r;
          out[e] += y[cc][a];
        }
    } else {
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
  const size_t bytes = sizeof(T) * (size_t)op->npts * (mode == 0 ? 3 * nrhs : 1);
  HHG_CUDA_TRY(cudaMemsetAsync(out, 0, bytes, s));
  dim3 grid((unsigned)((nh * nrhs + 255) / 256), (unsigned)nh, (unsigned)(nz * nm));
  for (int color = 0; color < 8; ++color) {
#define HHG_EPS(M, F, D) eps_color_kernel<T, M, F, D><<<grid, 256, 0, s>>>(cst, color, nz, nrhs, muc, x, g, mu, out)
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
