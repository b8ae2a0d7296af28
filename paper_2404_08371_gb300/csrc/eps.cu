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

// The operator needs only the symmetric gradient E = grad u + grad u^T (six entries, order of
// eps_sym), and E is affine in lambda like grad u: E(q) = H0 + sum_b lambda_b Hb, with Hb[v] =
// P[c][b][d] + P[d][b][c] for v = (c, d) from the affine gradient terms P of the components.
// H (24 values) is summed into the thread's shared-memory column one component at a time.
template <typename T, int TH>
__device__ __forceinline__ void eps_sym_affine(const OpConst<T>& c, int o, const int* idx, int masked, const T* __restrict__ x,
                                               int64_t base, int stride, int comp_stride, T* __restrict__ Hs) {
  const T* Ji = c.Jinv[o];
#pragma unroll
  for (int v = 0; v < 24; ++v) Hs[v * TH] = T(0);
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    T u[10], W[4][3];
#pragma unroll
    for (int a = 0; a < 10; ++a)
      u[a] = (masked >> a) & 1 ? T(0) : __ldg(x + (base + idx[a]) * stride + cc * comp_stride);
    eps_grad_affine<T>(u, W);
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) {
      T p3[3];
      phys_grad<T>(Ji, W[tt], p3);
#pragma unroll
      for (int d = 0; d < 3; ++d) Hs[(6 * tt + eps_sym(cc, d)) * TH] += (cc == d ? T(2) : T(1)) * p3[d];
    }
  }
}

template <int TH, typename T>
__device__ __forceinline__ void eps_sym_at(const T* __restrict__ Hs, T l1, T l2, T l3, T E[6]) {
#pragma unroll
  for (int v = 0; v < 6; ++v)
    E[v] = fma(l3, Hs[(18 + v) * TH], fma(l2, Hs[(12 + v) * TH], fma(l1, Hs[(6 + v) * TH], Hs[v * TH])));
}

// Apply, out += A u for all right-hand sides.  One CTA per task of its colour: up to cpb
// consecutive cubes of one row (cj, ck) of one macro, times the right-hand sides.  Each thread
// keeps its affine symmetric-gradient terms H (24 values), mu(x_q) w_q |det J| at the points and
// its node indices in its own column threadIdx.x of a [value][thread] shared-memory array: the
// quadrature loop then holds only the stress moments and one symmetric gradient in registers,
// which lets two CTAs (16 warps) share an SM to keep the FP64 pipes fed; reading H costs 24
// shared loads per point against about 50 FP64 operations.
constexpr int kEpsThreads = 256;
template <typename T, bool FIELD>
constexpr size_t eps_apply_smem() { return (sizeof(T) * (24 + (FIELD ? kMaxQ : 0)) + sizeof(int) * 10) * kEpsThreads; }

template <typename T, bool FIELD, bool DIR>
__global__ void __launch_bounds__(kEpsThreads, 2) eps_color_kernel(const OpConst<T>* __restrict__ cst,
                                                                    const int4* __restrict__ tasks, int color, int cpb,
                                                                    int nrhs, T mu_const, const T* __restrict__ x,
                                                                    const T* __restrict__ mu, T* __restrict__ out) {
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
  if (!live) return;
  const int64_t base = c.base;
  const int stride = 3 * nrhs;
  extern __shared__ __align__(16) unsigned char eps_smem_raw[];
  T* __restrict__ Ps = reinterpret_cast<T*>(eps_smem_raw) + threadIdx.x;   // H[v] at Ps[v * kEpsThreads]
  T* __restrict__ Ms = Ps + 24 * kEpsThreads;   // field: mu(x_q) w_q |det J| at the points
  int* __restrict__ Is = reinterpret_cast<int*>(reinterpret_cast<T*>(eps_smem_raw) + (FIELD ? 24 + kMaxQ : 24) * kEpsThreads) +
                         threadIdx.x;           // node indices
#pragma unroll 1
  for (int o = 0; o < 6; ++o) {
    if (ci + cj + ck > n - 1 - (o == 0 ? 0 : (o == 5 ? 2 : 1))) continue;
    int idx[10], masked = 0;   // bit a: node a reads as zero (Dirichlet point)
    T m[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int pi = 2 * ci + enode_d(o, a, 0), pj = 2 * cj + enode_d(o, a, 1), pk = 2 * ck + enode_d(o, a, 2);
      idx[a] = (int)packed_index(N, pi, pj, pk);
      Is[a * kEpsThreads] = idx[a];
      if (DIR && on_dirichlet(c.bnd_table, N, pi, pj, pk)) masked |= 1 << a;
      if (FIELD) m[a] = __ldg(mu + base + idx[a]);
    }
    const T* Ji = c.Jinv[o];
    const T wdet = c.adet[o];
    if (FIELD) {
      // mu at the quadrature points, times the weight and |det J|, once per micro-tet
#pragma unroll 1
      for (int q = 0; q < c.nq; ++q) {
        T muq = T(0);
#pragma unroll
        for (int a = 0; a < 10; ++a) muq += c.psi[q][a] * m[a];
        Ms[q * kEpsThreads] = muq * c.w[q] * wdet;
      }
    }
    // affine symmetric gradient of u into shared memory
    eps_sym_affine<T, kEpsThreads>(c, o, idx, masked, x + r, base, stride, nrhs, Ps);
    // physical moments of the stress: Q[t][v] = sum_q lambda_t S_v (lambda_0 = 1), S = s (G + G^T)
    // = 2 mu eps(u) w |det J| symmetric, so only its six entries v = (0,0) (1,1) (2,2) (0,1) (0,2)
    // (1,2) are accumulated (the entry of (c, d) is eps_sym(c, d))
    T Q[4][6];
#pragma unroll
    for (int tt = 0; tt < 4; ++tt)
#pragma unroll
      for (int v = 0; v < 6; ++v) Q[tt][v] = T(0);
#pragma unroll 1
    for (int q = 0; q < c.nq; ++q) {
      const T l1 = c.lam[q][1], l2 = c.lam[q][2], l3 = c.lam[q][3];
      T E[6];
      eps_sym_at<kEpsThreads>(Ps, l1, l2, l3, E);
      const T s = FIELD ? Ms[q * kEpsThreads] : mu_const * c.w[q] * wdet;
      T Sv[6];
#pragma unroll
      for (int v = 0; v < 6; ++v) Sv[v] = s * E[v];
#pragma unroll
      for (int v = 0; v < 6; ++v) {
        Q[0][v] += Sv[v];
        Q[1][v] = fma(l1, Sv[v], Q[1][v]);
        Q[2][v] = fma(l2, Sv[v], Q[2][v]);
        Q[3][v] = fma(l3, Sv[v], Q[3][v]);
      }
    }
    // y_c += sum_q (J^{-1} S_c) . grad_ref phi: map the moments back once, then test; the moments
    // go to shared memory (over H, no longer needed) so that one component at a time is in
    // registers, and each component is added to out as soon as it is formed
#pragma unroll
    for (int tt = 0; tt < 4; ++tt)
#pragma unroll
      for (int v = 0; v < 6; ++v) Ps[(6 * tt + v) * kEpsThreads] = Q[tt][v];
#pragma unroll 1
    for (int cc = 0; cc < 3; ++cc) {
      T R3[3], S3[3][3], yc[10], Qc[4][3];
#pragma unroll
      for (int tt = 0; tt < 4; ++tt)
#pragma unroll
        for (int d = 0; d < 3; ++d) Qc[tt][d] = Ps[(6 * tt + eps_sym(cc, d)) * kEpsThreads];
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
  }
}

// mu-adjoint, out_m += sum_r g_r^T (dA/dmu_m) u_r with mu a P2 field: per quadrature point
// t_q = w_q |det J| grad g : (grad u + grad u^T) = w_q |det J| E(g) : E(u) / 2 summed over the
// right-hand sides of a cube (consecutive lanes of one warp, nrhs divides 32) and tested against
// the ten basis values.  The tasks are the apply's (up to cpb cubes of a row); a CTA of
// kEpsAdjThreads threads takes them in two halves.  Each thread keeps the affine symmetric-gradient
// terms of u and of g (24 + 24 values) in its own column of shared memory, so that three CTAs
// (12 warps) share an SM.
constexpr int kEpsAdjThreads = kEpsThreads / 2;
template <typename T>
constexpr size_t eps_adjoint_smem() { return sizeof(T) * 48 * kEpsAdjThreads; }

template <typename T, bool DIR>
__global__ void __launch_bounds__(kEpsAdjThreads, 3) eps_adjoint_kernel(const OpConst<T>* __restrict__ cst,
                                                                         const int4* __restrict__ tasks, int color,
                                                                         int cpb, int nrhs, const T* __restrict__ x,
                                                                         const T* __restrict__ g, T* __restrict__ out) {
  const int4 task = tasks[blockIdx.x];
  const OpConst<T>& c = cst[task.w];
  const int n = c.n, N = c.N;
  const int r = threadIdx.x % nrhs;
  const int cj = 2 * task.y + ((color >> 1) & 1);
  const int ck = 2 * task.z + ((color >> 2) & 1);
  const int64_t base = c.base;
  const int stride = 3 * nrhs;
  extern __shared__ __align__(16) unsigned char eps_smem_raw[];
  T* __restrict__ Hu = reinterpret_cast<T*>(eps_smem_raw) + threadIdx.x;   // H of u at Hu[v * kEpsAdjThreads]
  T* __restrict__ Hg = Hu + 24 * kEpsAdjThreads;                            // H of g
  for (int half = 0; half < 2; ++half) {
    const int slot = (threadIdx.x + half * kEpsAdjThreads) / nrhs;
    const int ci = 2 * (task.x + slot) + (color & 1);
    const bool live = slot < cpb && ci + cj + ck <= n - 1;
    if (__all_sync(0xffffffffu, !live)) continue;   // whole warp (the shuffles below need all lanes)
#pragma unroll 1
    for (int o = 0; o < 6; ++o) {
      const bool tet_ok = live && ci + cj + ck <= n - 1 - (o == 0 ? 0 : (o == 5 ? 2 : 1));
      int idx[10], masked = 0;   // bit a: node a reads as zero (Dirichlet point or no micro-tet)
#pragma unroll
      for (int a = 0; a < 10; ++a) {
        const int pi = 2 * ci + enode_d(o, a, 0), pj = 2 * cj + enode_d(o, a, 1), pk = 2 * ck + enode_d(o, a, 2);
        idx[a] = tet_ok ? (int)packed_index(N, pi, pj, pk) : 0;
        if (!tet_ok || (DIR && on_dirichlet(c.bnd_table, N, pi, pj, pk))) masked |= 1 << a;
      }
      const T wdet = c.adet[o];
      eps_sym_affine<T, kEpsAdjThreads>(c, o, idx, masked, x + r, base, stride, nrhs, Hu);
      eps_sym_affine<T, kEpsAdjThreads>(c, o, idx, masked, g + r, base, stride, nrhs, Hg);
      T dmu[10];
#pragma unroll
      for (int a = 0; a < 10; ++a) dmu[a] = T(0);
#pragma unroll 1
      for (int q = 0; q < c.nq; ++q) {
        const T l1 = c.lam[q][1], l2 = c.lam[q][2], l3 = c.lam[q][3];
        T Eu[6], Eg[6];
        eps_sym_at<kEpsAdjThreads>(Hu, l1, l2, l3, Eu);
        eps_sym_at<kEpsAdjThreads>(Hg, l1, l2, l3, Eg);
        // E(g) : E(u) / 2 = the diagonal products halved plus the off-diagonal products
        T tq = T(0.5) * (Eg[0] * Eu[0] + Eg[1] * Eu[1] + Eg[2] * Eu[2]);
        tq = fma(Eg[3], Eu[3], fma(Eg[4], Eu[4], fma(Eg[5], Eu[5], tq)));
        tq *= c.w[q] * wdet;
#pragma unroll
        for (int a = 0; a < 10; ++a) dmu[a] += c.psi[q][a] * tq;
      }
      // sum over the right-hand sides of this cube, one writer (cubes of one colour share no point)
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
  // tasks of live cubes per colour, cached in the operator per number of cubes per CTA: built and
  // uploaded (asynchronously, on the caller's stream) at the first call with this batch size
  const int cpb = kEpsThreads / nrhs;
  EpsTasks* et = nullptr;
  {
    auto it = op->eps_tasks.find(cpb);
    if (it != op->eps_tasks.end()) et = it->second.get();
  }
  if (!et) {
    std::unique_ptr<EpsTasks> nt(new EpsTasks());
    std::vector<int4>& tv = nt->host;
    for (int color = 0; color < 8; ++color) {
      nt->off[color] = (int64_t)tv.size();
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
    nt->off[8] = (int64_t)tv.size();
    HHG_CUDA_TRY(cudaMalloc(&nt->d, sizeof(int4) * std::max<size_t>(tv.size(), 1)));
    if (!tv.empty())
      HHG_CUDA_TRY(cudaMemcpyAsync(nt->d, tv.data(), sizeof(int4) * tv.size(), cudaMemcpyHostToDevice, s));
    et = nt.get();
    op->eps_tasks[cpb] = std::move(nt);
  }
  const size_t bytes = sizeof(T) * (size_t)op->npts * (mode == 0 ? 3 * nrhs : 1);
  HHG_CUDA_TRY(cudaMemsetAsync(out, 0, bytes, s));
  for (int color = 0; color < 8; ++color) {
    const unsigned grid = (unsigned)(et->off[color + 1] - et->off[color]);
    if (grid == 0) continue;
    const int4* tk = et->d + et->off[color];
#define HHG_EPS(F, D)                                                                                          \
  do {                                                                                                       \
    const size_t sm = eps_apply_smem<T, F>();                                                                \
    if (sm > 48 * 1024)                                                                                      \
      HHG_CUDA_TRY(cudaFuncSetAttribute(eps_color_kernel<T, F, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        (int)sm));                                                           \
    eps_color_kernel<T, F, D><<<grid, kEpsThreads, sm, s>>>(cst, tk, color, cpb, nrhs, muc, x, mu, out);     \
  } while (0)
#define HHG_EPS_ADJ(D)                                                                                         \
  do {                                                                                                       \
    const size_t sm = eps_adjoint_smem<T>();                                                                 \
    if (sm > 48 * 1024)                                                                                      \
      HHG_CUDA_TRY(cudaFuncSetAttribute(eps_adjoint_kernel<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                        (int)sm));                                                           \
    eps_adjoint_kernel<T, D><<<grid, kEpsAdjThreads, sm, s>>>(cst, tk, color, cpb, nrhs, x, g, out);         \
  } while (0)
    const bool dir = op->bc == HHG_DIRICHLET;
    if (mode == 0) {
      if (field) {
        if (dir) HHG_EPS(true, true); else HHG_EPS(true, false);
      } else {
        if (dir) HHG_EPS(false, true); else HHG_EPS(false, false);
      }
    } else {
      if (dir) HHG_EPS_ADJ(true); else HHG_EPS_ADJ(false);
    }
#undef HHG_EPS
#undef HHG_EPS_ADJ
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
