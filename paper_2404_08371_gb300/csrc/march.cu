// Element-centric "marching" kernels: dispatch on (degree, coefficient, mode), the precomputed
// variant's local matrices, the L2 error of the manufactured solution and the Nedelec apply.  The
// kernel itself is in march_kernel.cuh; its launchers are instantiated in march_inst_<n>.cu.
#include "march_kernel.cuh"

HHG_MARCH_SHARD_0(HHG_MARCH_EXTERN)
HHG_MARCH_SHARD_1(HHG_MARCH_EXTERN)
HHG_MARCH_SHARD_2(HHG_MARCH_EXTERN)
HHG_MARCH_SHARD_3(HHG_MARCH_EXTERN)
HHG_MARCH_SHARD_4(HHG_MARCH_EXTERN)
HHG_MARCH_SHARD_5(HHG_MARCH_EXTERN)
HHG_MARCH_SHARD_6(HHG_MARCH_EXTERN)
HHG_MARCH_SHARD_7(HHG_MARCH_EXTERN)

namespace hhg {

// Local matrices of all micro-tets by quadrature, for the precomputed variant: one thread per
// (cube, class).  P2: A_T[a][b] = sum_q w_q k(x_q) gref_a(xi_q)^T M_o gref_b(xi_q), a <= b, summed per
// quadrature point into the thread's row of shared memory; P1: the element mean of k.  Classes that
// do not exist at the cube are skipped (never read).
constexpr int kElemThreads = 64;

template <typename T, int R, int COEF>
__global__ void __launch_bounds__(kElemThreads) elem_store_kernel(const OpConst<T>* __restrict__ cst,
                                                                  const T* __restrict__ kf, T* __restrict__ elem) {
  constexpr int NE = R == 1 ? 1 : 55;
  __shared__ T acc[kElemThreads][R == 1 ? 1 : 56];
  const int macro = blockIdx.y;
  const OpConst<T>& c = cst[macro];
  const int n = c.n, N = c.N;
  const int64_t ncubes = dV(n - 1);
  const int64_t t = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
  if (t >= 6 * ncubes) return;
  const int o = (int)(t % 6);
  const int64_t p = t / 6;
  int ci, cj, ck;
  decode_point(p, n - 1, ci, cj, ck);
  if (ci + cj + ck > n - 1 - class_shrink(o)) return;
  T* __restrict__ out = elem + ((int64_t)macro * 6 + o) * NE * ncubes + p;
  T so[3] = {T(0), T(0), T(0)}, co[3] = {T(0), T(0), T(0)};
  if (COEF == HHG_COEFF_SIN3) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T xd = c.X0[d] + T(ci) * c.H[0][d] + T(cj) * c.H[1][d] + T(ck) * c.H[2][d];
      sincos2pi<T>(xd, &so[d], &co[d]);
    }
  }
  constexpr int NL = R == 1 ? 4 : 10;
  T kb[NL];
  if (COEF == HHG_COEFF_FIELD_P1 || COEF == HHG_COEFF_FIELD_P2) {
#pragma unroll
    for (int a = 0; a < NL; ++a) {
      const int s = node_slot<R>(o, a), cx = s % (R + 1), cy = (s / (R + 1)) % (R + 1), cz = s / ((R + 1) * (R + 1));
      kb[a] = __ldg(kf + c.kbase + packed_index(N, R * ci + cx, R * cj + cy, R * ck + cz));
    }
  }
  if constexpr (R == 1) {
    T kbar = T(1);
    if (COEF == HHG_COEFF_SIN3) {
      for (int q = 0; q < c.nq; ++q) {
        T sv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) sv[d] = so[d] * c.cs[o][q][d][0] + co[d] * c.cs[o][q][d][1];
        kbar = fma(sv[0] * sv[1], sv[2], kbar);   // factor 3 w_q in the x table
      }
    } else {
      kbar = T(0.25) * (kb[0] + kb[1] + kb[2] + kb[3]);
    }
    out[0] = kbar;
  } else {
    T* a_row = acc[threadIdx.x];
    for (int e = 0; e < NE; ++e) a_row[e] = T(0);
    const T* M = c.M[o];
    const T g0[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};   // grad_ref lambda_a
    for (int q = 0; q < c.nq; ++q) {
      T sq;
      if (COEF == HHG_COEFF_SIN3) {
        T sv[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) sv[d] = so[d] * c.cs[o][q][d][0] + co[d] * c.cs[o][q][d][1];
        sq = fma(sv[0] * sv[1], sv[2], c.w[q]);   // factor 0.5 w_q in the x table
      } else {
        T kq = T(0);
#pragma unroll
        for (int m = 0; m < 10; ++m) kq += c.psi[q][m] * kb[m];
        sq = kq * c.w[q];
      }
      // reference gradients of the 10 basis functions at the point
      T G[10][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) G[a][d] = c.lam4m1[q][a] * g0[a][d];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int a = edge_end(e, 0), b = edge_end(e, 1);
#pragma unroll
        for (int d = 0; d < 3; ++d) G[4 + e][d] = c.lam4[q][a] * g0[b][d] + c.lam4[q][b] * g0[a][d];
      }
#pragma unroll
      for (int b = 0; b < 10; ++b) {
        T mg[3];
        metric<T>(M, G[b], mg);
        mg[0] *= sq;
        mg[1] *= sq;
        mg[2] *= sq;
#pragma unroll
        for (int a = 0; a <= b; ++a) a_row[p2_sym(a, b)] += G[a][0] * mg[0] + G[a][1] * mg[1] + G[a][2] * mg[2];
      }
    }
    for (int e = 0; e < NE; ++e) out[(int64_t)e * ncubes] = a_row[e];
  }
}

template <typename T>
int launch_elem_store(const hhg_op* op, T* elem, cudaStream_t s) {
  const int nm = op->mesh->nmacro();
  const int64_t ncubes = (int64_t)op->n * (op->n + 1) * (op->n + 2) / 6;   // V(n - 1)
  const dim3 grid((unsigned)((6 * ncubes + kElemThreads - 1) / kElemThreads), nm);
  const OpConst<T>* cst = (const OpConst<T>*)(sizeof(T) == 8 ? op->d_const64 : op->d_const32);
  const T* kf = (op->coeff.type == HHG_COEFF_FIELD_P1 || op->coeff.type == HHG_COEFF_FIELD_P2)
                    ? (const T*)op->coeff.field : nullptr;
#define HHG_ELEM(RR, CC) elem_store_kernel<T, RR, CC><<<grid, kElemThreads, 0, s>>>(cst, kf, elem)
  if (op->degree == 1 && op->coeff.type == HHG_COEFF_SIN3) HHG_ELEM(1, HHG_COEFF_SIN3);
  else if (op->degree == 1 && op->coeff.type == HHG_COEFF_FIELD_P1) HHG_ELEM(1, HHG_COEFF_FIELD_P1);
  else if (op->degree == 2 && op->coeff.type == HHG_COEFF_SIN3) HHG_ELEM(2, HHG_COEFF_SIN3);
  else if (op->degree == 2 && op->coeff.type == HHG_COEFF_FIELD_P2) HHG_ELEM(2, HHG_COEFF_FIELD_P2);
  else return fail(HHG_E_UNSUPPORTED, "store_element_matrices: needs a SIN3 or FIELD coefficient of the op's degree");
#undef HHG_ELEM
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}
template int launch_elem_store<double>(const hhg_op*, double*, cudaStream_t);
template int launch_elem_store<float>(const hhg_op*, float*, cudaStream_t);

// Apply with the stored local matrices.
template <typename T>
int launch_march_stored(const hhg_op* op, const T* x, T* y, cudaStream_t s) {
  const OpConst<T>* cst = (const OpConst<T>*)(sizeof(T) == 8 ? op->d_const64 : op->d_const32);
  if (op->degree == 1) return launch_march_t<T, 1, kCoefStored, MODE_APPLY>(op, cst, x, nullptr, (const T*)op->d_elem, y, s);
  return launch_march_t<T, 2, kCoefStored, MODE_APPLY>(op, cst, x, nullptr, (const T*)op->d_elem, y, s);
}
template int launch_march_stored<double>(const hhg_op*, const double*, double*, cudaStream_t);
template int launch_march_stored<float>(const hhg_op*, const float*, float*, cudaStream_t);

// Dispatch on (degree, coefficient, mode).  Returns HHG_E_UNSUPPORTED for other combinations.
template <typename T>
int launch_march(const hhg_op* op, const OpConst<T>* cst, int mode, const T* x, const T* g, const T* kf, T* out,
                 cudaStream_t s) {
  const int ct = op->coeff.type;
#define HHG_MARCH_CASE(RR, CC, MM) \
  if (op->degree == RR && ct == CC && mode == MM) return launch_march_t<T, RR, CC, MM>(op, cst, x, g, kf, out, s);
  HHG_MARCH_CASE(1, HHG_COEFF_SIN3, MODE_APPLY)
  HHG_MARCH_CASE(1, HHG_COEFF_FIELD_P1, MODE_APPLY)
  HHG_MARCH_CASE(1, HHG_COEFF_SIN3, MODE_DIAG)
  HHG_MARCH_CASE(1, HHG_COEFF_FIELD_P1, MODE_DIAG)
  HHG_MARCH_CASE(1, HHG_COEFF_FIELD_P1, MODE_ADJ)
  HHG_MARCH_CASE(2, HHG_COEFF_CONST, MODE_APPLY)
  // P2 variable coefficient: the affine form pays from about 7 quadrature points on
  if (op->degree == 2 && mode == MODE_APPLY && (ct == HHG_COEFF_SIN3 || ct == HHG_COEFF_FIELD_P2)) {
    const bool aff = op->rule.nq() > 6;
    if (ct == HHG_COEFF_SIN3)
      return aff ? launch_march_t<T, 2, HHG_COEFF_SIN3, MODE_APPLY, true>(op, cst, x, g, kf, out, s)
                 : launch_march_t<T, 2, HHG_COEFF_SIN3, MODE_APPLY, false>(op, cst, x, g, kf, out, s);
    return aff ? launch_march_t<T, 2, HHG_COEFF_FIELD_P2, MODE_APPLY, true>(op, cst, x, g, kf, out, s)
               : launch_march_t<T, 2, HHG_COEFF_FIELD_P2, MODE_APPLY, false>(op, cst, x, g, kf, out, s);
  }
  HHG_MARCH_CASE(2, HHG_COEFF_SIN3, MODE_DIAG)
  HHG_MARCH_CASE(2, HHG_COEFF_FIELD_P2, MODE_DIAG)
  HHG_MARCH_CASE(2, HHG_COEFF_FIELD_P2, MODE_ADJ)
  if (sizeof(T) == 8) {
    HHG_MARCH_CASE(1, HHG_COEFF_CONST, MODE_RHS)
    HHG_MARCH_CASE(2, HHG_COEFF_CONST, MODE_RHS)
  }
#undef HHG_MARCH_CASE
  return fail(HHG_E_UNSUPPORTED, "no kernel for degree %d, coefficient %d, mode %d", op->degree, ct, mode);
}

int alloc_face_scratch(hhg_op* op) {
  if (op->n < kMarchJAtomicN || op->kind == HHG_EPSILON) return HHG_OK;
  const int64_t R = op->degree, N = op->N;
  const int64_t Fi = 32 * R, Fj = kWarps * R;
  op->face_Ti = (int)(N / Fi);
  op->face_Tj = (int)(N / Fj);
  op->face_Si = face_tri_sum(Fi, op->face_Ti, N);
  op->face_Sj = face_tri_sum(Fj, op->face_Tj, N);
  op->face_S = op->face_Si + op->face_Sj + (int64_t)op->face_Ti * op->face_Tj * (N + 1);
  HHG_CUDA_TRY(cudaMalloc(&op->d_face, sizeof(double) * (size_t)op->face_S * op->mesh->nmacro()));
  return HHG_OK;
}

// Squared L2 error of u_h against u = sin(pi x) sin(pi y) sin(pi z): one thread per cube,
// the six micro-tets with the op's quadrature rule; per-CTA partial sums (no atomics).
template <int R>
__global__ void __launch_bounds__(256) l2_error_kernel(const OpConst<double>* __restrict__ cst,
                                                        const double* __restrict__ uh, double* __restrict__ partial) {
  constexpr int NL = R == 1 ? 4 : 10;
  const OpConst<double>& c = cst[blockIdx.y];
  const int n = c.n, N = c.N;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (p < dV(n - 1)) {
    int ci, cj, ck;
    decode_point(p, n - 1, ci, cj, ck);   // cube origins: i + j + k <= n - 1
    for (int o = 0; o < 6; ++o) {
      if (ci + cj + ck > n - 1 - class_shrink(o)) continue;
      double ul[NL];
      for (int a = 0; a < NL; ++a) {
        int q[3];
        for (int d = 0; d < 3; ++d) {
          if (R == 1 || a < 4)
            q[d] = R * kClassOffsetsD[o][a][d];
          else
            q[d] = kClassOffsetsD[o][kP2EdgesD[a - 4][0]][d] + kClassOffsetsD[o][kP2EdgesD[a - 4][1]][d];
        }
        ul[a] = uh[c.base + packed_index(N, R * ci + q[0], R * cj + q[1], R * ck + q[2])];
      }
      for (int q = 0; q < c.nq; ++q) {
        double xq[3];
        for (int d = 0; d < 3; ++d)
          xq[d] = c.X0[d] + ci * c.H[0][d] + cj * c.H[1][d] + ck * c.H[2][d] + c.qoff[o][q][d];
        double uhq = 0.0;
        for (int a = 0; a < NL; ++a) uhq += ul[a] * (R == 1 ? c.lam[q][a] : c.psi[q][a]);
        const double e = uhq - sinpi(xq[0]) * sinpi(xq[1]) * sinpi(xq[2]);
        acc += c.w[q] * c.adet[o] * e * e;
      }
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = red[0];
}

int64_t launch_l2_blocks(const hhg_op* op) {
  return ((lattice_size(op->n - 1) + 255) / 256) * op->mesh->nmacro();
}

int launch_l2_error(const hhg_op* op, const double* uh, double* partial, cudaStream_t s) {
  const unsigned gx = (unsigned)((lattice_size(op->n - 1) + 255) / 256);
  dim3 grid(gx, op->mesh->nmacro());
  if (op->degree == 1)
    l2_error_kernel<1><<<grid, 256, 0, s>>>((const OpConst<double>*)op->d_const64, uh, partial);
  else
    l2_error_kernel<2><<<grid, 256, 0, s>>>((const OpConst<double>*)op->d_const64, uh, partial);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

// Local matrices of the Nedelec operator for the precomputed variant: one thread per (cube, class),
// A_T = mean(alpha) C_o + sum_v beta_v M_o^v (21 entries, canonical orientation).
template <typename T>
__global__ void __launch_bounds__(kElemThreads) elem_store_n1_kernel(const N1Const<T>* __restrict__ n1, N1Args<T> a,
                                                                     T* __restrict__ elem) {
  const int macro = blockIdx.y;
  const int n = a.n;
  const int64_t ncubes = dV(n - 1);
  const int64_t t = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
  if (t >= 6 * ncubes) return;
  const int o = (int)(t % 6);
  const int64_t p = t / 6;
  int ci, cj, ck;
  decode_point(p, n - 1, ci, cj, ck);
  if (ci + cj + ck > n - 1 - class_shrink(o)) return;
  const N1Const<T>& q = n1[macro];
  T av[4], bv[4];
  for (int v = 0; v < 4; ++v) {
    const int64_t vidx = q.vbase + packed_index(n, ci + coff(o, v, 0), cj + coff(o, v, 1), ck + coff(o, v, 2));
    av[v] = a.alpha ? __ldg(a.alpha + vidx) : a.alpha_c;
    bv[v] = a.beta ? __ldg(a.beta + vidx) : a.beta_c;
  }
  const T abar = T(0.25) * (av[0] + av[1] + av[2] + av[3]);
  T* __restrict__ out = elem + ((int64_t)macro * 6 + o) * kN1Sym * ncubes + p;
  for (int e = 0; e < kN1Sym; ++e)
    out[(int64_t)e * ncubes] = abar * q.C[o][e] + bv[0] * q.M[o][0][e] + bv[1] * q.M[o][1][e] +
                               bv[2] * q.M[o][2][e] + bv[3] * q.M[o][3][e];
}

template <typename T>
static N1Args<T> n1_args(const hhg_op* op) {
  N1Args<T> a;
  a.n1 = (const N1Const<T>*)(sizeof(T) == 8 ? op->d_n1_64 : op->d_n1_32);
  a.alpha = op->coeff.type == HHG_COEFF_FIELD_P1 ? (const T*)op->coeff.field : nullptr;
  a.beta = op->coeff2.type == HHG_COEFF_FIELD_P1 ? (const T*)op->coeff2.field : nullptr;
  a.alpha_c = (T)op->coeff.value;
  a.beta_c = (T)op->coeff2.value;
  a.n = op->n;
  return a;
}

template <typename T>
int launch_elem_store_n1(const hhg_op* op, T* elem, cudaStream_t s) {
  const int64_t ncubes = (int64_t)op->n * (op->n + 1) * (op->n + 2) / 6;
  const dim3 grid((unsigned)((6 * ncubes + kElemThreads - 1) / kElemThreads), op->mesh->nmacro());
  const N1Args<T> a = n1_args<T>(op);
  elem_store_n1_kernel<T><<<grid, kElemThreads, 0, s>>>(a.n1, a, elem);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}
template int launch_elem_store_n1<double>(const hhg_op*, double*, cudaStream_t);
template int launch_elem_store_n1<float>(const hhg_op*, float*, cudaStream_t);

template <typename T>
int launch_n1(const hhg_op* op, const T* x, T* y, cudaStream_t s) {
  if (op->d_elem && op->elem_dtype == (sizeof(T) == 8 ? HHG_F64 : HHG_F32)) {
    const OpConst<T>* cst = (const OpConst<T>*)(sizeof(T) == 8 ? op->d_const64 : op->d_const32);
    return launch_march_t<T, 2, kCoefStored, MODE_N1>(op, cst, x, nullptr, (const T*)op->d_elem, y, s, n1_args<T>(op));
  }
  N1Args<T> a;
  a.n1 = (const N1Const<T>*)(sizeof(T) == 8 ? op->d_n1_64 : op->d_n1_32);
  a.alpha = op->coeff.type == HHG_COEFF_FIELD_P1 ? (const T*)op->coeff.field : nullptr;
  a.beta = op->coeff2.type == HHG_COEFF_FIELD_P1 ? (const T*)op->coeff2.field : nullptr;
  a.alpha_c = (T)op->coeff.value;
  a.beta_c = (T)op->coeff2.value;
  a.n = op->n;
  const OpConst<T>* cst = (const OpConst<T>*)(sizeof(T) == 8 ? op->d_const64 : op->d_const32);
  return launch_march_t<T, 2, HHG_COEFF_CONST, MODE_N1>(op, cst, x, nullptr, nullptr, y, s, a);
}
// Diagonal of the Nedelec operator (vertex points of the doubled lattice, which carry no DoF, get 0).
template <typename T>
int launch_n1_diag(const hhg_op* op, T* d, cudaStream_t s) {
  const OpConst<T>* cst = (const OpConst<T>*)(sizeof(T) == 8 ? op->d_const64 : op->d_const32);
  return launch_march_t<T, 2, HHG_COEFF_CONST, MODE_N1D>(op, cst, nullptr, nullptr, nullptr, d, s, n1_args<T>(op));
}
template int launch_n1_diag<double>(const hhg_op*, double*, cudaStream_t);
template int launch_n1_diag<float>(const hhg_op*, float*, cudaStream_t);

template int launch_n1<double>(const hhg_op*, const double*, double*, cudaStream_t);
template int launch_n1<float>(const hhg_op*, const float*, float*, cudaStream_t);

template int launch_march<double>(const hhg_op*, const OpConst<double>*, int, const double*, const double*,
                                  const double*, double*, cudaStream_t);
template int launch_march<float>(const hhg_op*, const OpConst<float>*, int, const float*, const float*, const float*,
                                 float*, cudaStream_t);

}  // namespace hhg
