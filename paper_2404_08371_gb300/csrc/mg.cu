// Geometric multigrid on the refinement hierarchy (Section 8): grid transfers,
// Chebyshev smoother, power iteration, load vector / L2 error of the manufactured
// Poisson problem, exact FP64 coarse solve, and the FMG + iterative-refinement driver.
//
// Uniform refinement makes the FE spaces nested, so prolongation evaluates the
// coarse FE function at the fine nodes and restriction is its transpose.  Both
// are translation invariant inside a macro: a fine node's position inside its
// coarse cube fixes the coarse micro-tet that contains it and the basis weights,
// tabulated once per degree.  Restriction sums over distinct fine points: a copy
// of a shared point only counts in the macro that owns it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "hhg_internal.h"
#include "lattice.cuh"

namespace hhg {

// Coarse-cube block position (0..R per axis) of local node `node` of class o.
static void node_pos(int R, int o, int node, int p[3]) {
  for (int d = 0; d < 3; ++d) {
    if (R == 1 || node < 4)
      p[d] = R * kClassOffsets[o][node][d];
    else
      p[d] = kClassOffsets[o][kP2Edges[node - 4][0]][d] + kClassOffsets[o][kP2Edges[node - 4][1]][d];
  }
}

// Transfer tables of one degree R (device):
//   pos table over fine positions a in [0, 2R]^3 inside a coarse cube: class and nloc weights;
//   restriction stencils per coarse node type: (dx, dy, dz, w) lists.
struct TransferTables {
  int R = 0;
  int npos = 0;
  int* d_pos_cls = nullptr;        // npos
  int* d_pos_off = nullptr;        // npos x 10: node position in the coarse cube block, q0 | q1 << 4 | q2 << 8
  double* d_pos_w64 = nullptr;     // npos x 10
  float* d_pos_w32 = nullptr;
  int ntypes = 0;
  int* d_st_ptr = nullptr;         // ntypes + 1
  int* d_st_off = nullptr;         // per entry (dx + 8) | (dy + 8) << 5 | (dz + 8) << 10
  double* d_st_w64 = nullptr;
  float* d_st_w32 = nullptr;
  ~TransferTables() {
    cudaFree(d_pos_cls);
    cudaFree(d_pos_off);
    cudaFree(d_pos_w64);
    cudaFree(d_pos_w32);
    cudaFree(d_st_ptr);
    cudaFree(d_st_off);
    cudaFree(d_st_w64);
    cudaFree(d_st_w32);
  }
};

static void basis_at(int R, const double lam[4], double* w) {
  if (R == 1) {
    for (int a = 0; a < 4; ++a) w[a] = lam[a];
    return;
  }
  for (int a = 0; a < 4; ++a) w[a] = lam[a] * (2.0 * lam[a] - 1.0);
  for (int e = 0; e < 6; ++e) w[4 + e] = 4.0 * lam[kP2Edges[e][0]] * lam[kP2Edges[e][1]];
}

// Containing class (first of white up, octahedron tets, white down) and basis weights of the
// point with cube coordinates xi (each in [0, 1]).
static int locate(int R, const double xi[3], double* w) {
  for (int o = 0; o < 6; ++o) {
    double D[3][3], rhs[3];
    for (int r = 0; r < 3; ++r) {
      for (int b = 0; b < 3; ++b) D[r][b] = kClassOffsets[o][b + 1][r] - kClassOffsets[o][0][r];
      rhs[r] = xi[r] - kClassOffsets[o][0][r];
    }
    // solve D l = rhs by Cramer's rule (D is unimodular)
    auto det3 = [](double A[3][3]) {
      return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
             A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    };
    const double dd = det3(D);
    double l[3];
    for (int b = 0; b < 3; ++b) {
      double Db[3][3];
      std::memcpy(Db, D, sizeof(D));
      for (int r = 0; r < 3; ++r) Db[r][b] = rhs[r];
      l[b] = det3(Db) / dd;
    }
    const double lam[4] = {1.0 - l[0] - l[1] - l[2], l[0], l[1], l[2]};
    if (lam[0] >= -1e-12 && lam[1] >= -1e-12 && lam[2] >= -1e-12 && lam[3] >= -1e-12) {
      basis_at(R, lam, w);
      return o;
    }
  }
  return -1;
}

static int upload_transfer_tables(int R, TransferTables* T, const std::vector<int>& cls, const std::vector<double>& w64);

static int build_transfer_tables(int R, TransferTables* T) {
  const int W = 2 * R + 1;
  const int npos = W * W * W;
  std::vector<int> cls(npos);
  std::vector<double> w64(npos * 10, 0.0);
  for (int az = 0; az < W; ++az)
    for (int ay = 0; ay < W; ++ay)
      for (int ax = 0; ax < W; ++ax) {
        const int t = ax + W * (ay + W * az);
        const double xi[3] = {ax / (2.0 * R), ay / (2.0 * R), az / (2.0 * R)};
        cls[t] = locate(R, xi, &w64[10 * t]);
        if (cls[t] < 0) return fail(HHG_E_CUDA, "transfer table: point not located");
      }
  return upload_transfer_tables(R, T, cls, w64);
}

// Canonical lattice direction of the edge whose doubled-lattice midpoint has parity (pi, pj, pk): the
// parity vector with its second nonzero component negated ((1,1,0) -> (1,-1,0), (1,1,1) -> (1,-1,1)).
static void edge_canonical_dir(int pi, int pj, int pk, int d[3]) {
  d[0] = pi;
  d[1] = pj;
  d[2] = pk;
  if (pi && pj) d[1] = -1;
  else if ((pi || pj) && pk) d[2] = -1;
}

// Nedelec prolongation (Section 8; the tangential integrals of the coarse Whitney field along the
// fine edges).  Fine edge midpoints in the doubled fine lattice sit at positions a in [0, 4]^3 of a
// coarse cube; a position with an odd coordinate is an edge of canonical direction d, the fine edge
// vector is d/2 and its midpoint a/4 in coarse cube coordinates.  The coarse Whitney functions
// phi_AB = lambda_A grad lambda_B - lambda_B grad lambda_A of the containing coarse micro-tet are
// linear, so the tangential integral is phi_AB(a/4) . d/2; the coarse DoF of edge (A, B) is the
// integral along its own canonical direction, so the weight carries the sign of V_B - V_A against
// it.  Index space is enough: tangential integrals are invariant under the affine map of a macro.
// Vertex positions (all coordinates even) carry no DoF and get zero weights.
static int build_n1_transfer_tables(TransferTables* T) {
  const int R = 2, W = 5, npos = W * W * W;
  std::vector<int> cls(npos, 0);
  std::vector<double> w64(npos * 10, 0.0);
  for (int az = 0; az < W; ++az)
    for (int ay = 0; ay < W; ++ay)
      for (int ax = 0; ax < W; ++ax) {
        const int t = ax + W * (ay + W * az);
        if (!((ax | ay | az) & 1)) continue;
        const double xi[3] = {ax / 4.0, ay / 4.0, az / 4.0};
        double wp2[10];
        const int o = locate(R, xi, wp2);
        if (o < 0) return fail(HHG_E_CUDA, "edge transfer table: point not located");
        cls[t] = o;
        // barycentric coordinates and index-space gradients of the coarse micro-tet of class o
        double D[3][3];
        for (int r = 0; r < 3; ++r)
          for (int b = 0; b < 3; ++b) D[r][b] = kClassOffsets[o][b + 1][r] - kClassOffsets[o][0][r];
        const double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                           D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                           D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
        double Di[3][3];   // inverse: row b-1 is grad lambda_b
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) {
            const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
            Di[r][c] = (D[r1][c1] * D[r2][c2] - D[r1][c2] * D[r2][c1]) / det;
          }
        double g[4][3], lam[4];
        for (int d = 0; d < 3; ++d) {
          g[1][d] = Di[0][d];
          g[2][d] = Di[1][d];
          g[3][d] = Di[2][d];
          g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
        }
        double l3[3];
        for (int b = 0; b < 3; ++b) {
          l3[b] = 0.0;
          for (int d = 0; d < 3; ++d) l3[b] += Di[b][d] * (xi[d] - kClassOffsets[o][0][d]);
        }
        lam[1] = l3[0];
        lam[2] = l3[1];
        lam[3] = l3[2];
        lam[0] = 1.0 - l3[0] - l3[1] - l3[2];
        int dv[3];
        edge_canonical_dir(ax & 1, ay & 1, az & 1, dv);
        const double tv[3] = {dv[0] / 2.0, dv[1] / 2.0, dv[2] / 2.0};
        for (int e = 0; e < 6; ++e) {
          const int A = kP2Edges[e][0], B = kP2Edges[e][1];
          double val = 0.0;
          for (int d = 0; d < 3; ++d) val += (lam[A] * g[B][d] - lam[B] * g[A][d]) * tv[d];
          int vec[3], dc[3];
          for (int d = 0; d < 3; ++d) vec[d] = kClassOffsets[o][B][d] - kClassOffsets[o][A][d];
          edge_canonical_dir((kClassOffsets[o][A][0] + kClassOffsets[o][B][0]) & 1,
                             (kClassOffsets[o][A][1] + kClassOffsets[o][B][1]) & 1,
                             (kClassOffsets[o][A][2] + kClassOffsets[o][B][2]) & 1, dc);
          const double sg = (vec[0] == dc[0] && vec[1] == dc[1] && vec[2] == dc[2]) ? 1.0 : -1.0;
          w64[10 * t + 4 + e] = sg * val;
        }
      }
  return upload_transfer_tables(R, T, cls, w64);
}

// Restriction stencils (columns of P per coarse node type on an unbounded lattice) and upload.
static int upload_transfer_tables(int R, TransferTables* T, const std::vector<int>& cls, const std::vector<double>& w64) {
  T->R = R;
  const int W = 2 * R + 1;
  T->npos = W * W * W;
  const int nloc = R == 1 ? 4 : 10;
  // restriction stencils: column C of P for a coarse node of each type, on an unbounded lattice
  const int ntypes = R == 1 ? 1 : 8;
  std::vector<int> st_ptr{0}, st_off;
  std::vector<double> st_w;
  for (int type = 0; type < ntypes; ++type) {
    const int C[3] = {R * 8 + (type & 1), R * 8 + ((type >> 1) & 1), R * 8 + ((type >> 2) & 1)};
    for (int dz = -2 * R; dz <= 2 * R; ++dz)
      for (int dy = -2 * R; dy <= 2 * R; ++dy)
        for (int dx = -2 * R; dx <= 2 * R; ++dx) {
          const int f[3] = {2 * C[0] + dx, 2 * C[1] + dy, 2 * C[2] + dz};
          int c[3], a[3];
          for (int d = 0; d < 3; ++d) {
            c[d] = f[d] / (2 * R);
            a[d] = f[d] - 2 * R * c[d];
          }
          const int t = a[0] + W * (a[1] + W * a[2]);
          double wsum = 0.0;
          for (int node = 0; node < nloc; ++node) {
            int p[3];
            node_pos(R, cls[t], node, p);
            if (R * c[0] + p[0] == C[0] && R * c[1] + p[1] == C[1] && R * c[2] + p[2] == C[2]) wsum += w64[10 * t + node];
          }
          if (std::fabs(wsum) > 1e-14) {
            st_off.push_back((dx + 8) | ((dy + 8) << 5) | ((dz + 8) << 10));
            st_w.push_back(wsum);
          }
        }
    st_ptr.push_back((int)st_w.size());
  }
  T->ntypes = ntypes;
  std::vector<int> poff(T->npos * 10, 0);
  for (int t = 0; t < T->npos; ++t)
    for (int node = 0; node < nloc; ++node) {
      int p[3];
      node_pos(R, cls[t], node, p);
      poff[10 * t + node] = p[0] | (p[1] << 4) | (p[2] << 8);
    }
  HHG_CUDA_TRY(cudaMalloc(&T->d_pos_off, sizeof(int) * poff.size()));
  HHG_CUDA_TRY(cudaMemcpy(T->d_pos_off, poff.data(), sizeof(int) * poff.size(), cudaMemcpyHostToDevice));
  std::vector<float> w32(w64.begin(), w64.end()), sw32(st_w.begin(), st_w.end());
  HHG_CUDA_TRY(cudaMalloc(&T->d_pos_cls, sizeof(int) * cls.size()));
  HHG_CUDA_TRY(cudaMalloc(&T->d_pos_w64, sizeof(double) * w64.size()));
  HHG_CUDA_TRY(cudaMalloc(&T->d_pos_w32, sizeof(float) * w32.size()));
  HHG_CUDA_TRY(cudaMalloc(&T->d_st_ptr, sizeof(int) * st_ptr.size()));
  HHG_CUDA_TRY(cudaMalloc(&T->d_st_off, sizeof(int) * st_off.size()));
  HHG_CUDA_TRY(cudaMalloc(&T->d_st_w64, sizeof(double) * st_w.size()));
  HHG_CUDA_TRY(cudaMalloc(&T->d_st_w32, sizeof(float) * sw32.size()));
  HHG_CUDA_TRY(cudaMemcpy(T->d_pos_cls, cls.data(), sizeof(int) * cls.size(), cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(T->d_pos_w64, w64.data(), sizeof(double) * w64.size(), cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(T->d_pos_w32, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(T->d_st_ptr, st_ptr.data(), sizeof(int) * st_ptr.size(), cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(T->d_st_off, st_off.data(), sizeof(int) * st_off.size(), cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(T->d_st_w64, st_w.data(), sizeof(double) * st_w.size(), cudaMemcpyHostToDevice));
  HHG_CUDA_TRY(cudaMemcpy(T->d_st_w32, sw32.data(), sizeof(float) * sw32.size(), cudaMemcpyHostToDevice));
  return HHG_OK;
}

// ---------------------------------------------------------------------------
// Per-point kernels over a level's packed layout (plane launch tables)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tri32(int s) { return ((s + 1) * (s + 2)) >> 1; }
__device__ __forceinline__ int rowst32(int s, int j) { return (j * (2 * s + 3 - j)) >> 1; }

// Decode the point of this thread from the plane tables; false if past the plane's end.
__device__ __forceinline__ bool plane_point(int N, const int* cta_plane, const int* cta_start, const int* pstart,
                                            int& i, int& j, int& k, int& p) {
  k = __ldg(cta_plane + blockIdx.x);
  const int s = N - k;
  const int q = (blockIdx.x - __ldg(cta_start + k)) * 256 + threadIdx.x;
  if (q >= tri32(s)) return false;
  const float b = 2.0f * s + 3.0f;
  int jj = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)q, 0.0f))));
  jj = max(0, min(jj, s));
  if (jj < s && rowst32(s, jj + 1) <= q) ++jj;
  if (jj > 0 && rowst32(s, jj) > q) --jj;
  j = jj;
  i = q - rowst32(s, jj);
  p = __ldg(pstart + k) + q;
  return true;
}

struct LevelArgs {
  int N;                 // resolution of the space
  int64_t V;             // points per macro
  const int* cta_plane;
  const int* cta_start;
  const int* pstart;
};

template <typename T, int R>
__global__ void __launch_bounds__(256) prolongate_kernel(LevelArgs fine, LevelArgs coarse, const int* __restrict__ pos_off,
                                                          const T* __restrict__ pos_w, const T* __restrict__ xc,
                                                          T* __restrict__ xf) {
  constexpr int W = 2 * R + 1;
  constexpr int NL = R == 1 ? 4 : 10;
  int i, j, k, p;
  if (!plane_point(fine.N, fine.cta_plane, fine.cta_start, fine.pstart, i, j, k, p)) return;
  const int m = blockIdx.y;
  const int nc = coarse.N / R;            // coarse cubes per edge
  int c0 = i / (2 * R), c1 = j / (2 * R), c2 = k / (2 * R);
  int a0 = i - 2 * R * c0, a1 = j - 2 * R * c1, a2 = k - 2 * R * c2;
  if (c0 + c1 + c2 > nc - 1) {
    // a coarse vertex on the top face of the macro: take it from the cube below it
    if (c0 > 0) {
      c0 -= 1;
      a0 += 2 * R;
    } else if (c1 > 0) {
      c1 -= 1;
      a1 += 2 * R;
    } else {
      c2 -= 1;
      a2 += 2 * R;
    }
  }
  const int t = a0 + W * (a1 + W * a2);
  const T* __restrict__ xm = xc + (int64_t)m * coarse.V;
  // the nodes of the containing coarse micro-tet lie in the planes R c2 .. R c2 + R
  int ps[R + 1];
#pragma unroll
  for (int dz = 0; dz <= R; ++dz) ps[dz] = __ldg(coarse.pstart + R * c2 + dz);
  T acc = T(0);
#pragma unroll
  for (int node = 0; node < NL; ++node) {
    const int q = __ldg(pos_off + 10 * t + node);
    const T wv = __ldg(pos_w + 10 * t + node);
    const int dz = q >> 8;
    const int ci = R * c0 + (q & 15), cj = R * c1 + ((q >> 4) & 15), ck = R * c2 + dz;
    const int pk = (R == 2 && dz == 2) ? ps[R] : (dz >= 1 ? ps[1] : ps[0]);
    acc += wv * __ldg(xm + pk + rowst32(coarse.N - ck, cj) + ci);
  }
  xf[(int64_t)m * fine.V + p] = acc;
}

template <typename T, int R>
__global__ void __launch_bounds__(256) restrict_kernel(LevelArgs fine, LevelArgs coarse, const MacroGeom* __restrict__ mg,
                                                        const int* __restrict__ st_ptr, const int* __restrict__ st_off,
                                                        const T* __restrict__ st_w, const T* __restrict__ rf,
                                                        T* __restrict__ rc) {
  int i, j, k, p;
  if (!plane_point(coarse.N, coarse.cta_plane, coarse.cta_start, coarse.pstart, i, j, k, p)) return;
  const int m = blockIdx.y;
  const uint32_t bnd = mg[m].bnd_table, own = mg[m].own_table;
  T* out = rc + (int64_t)m * coarse.V + p;
  if (on_dirichlet(bnd, coarse.N, i, j, k)) {
    *out = T(0);
    return;
  }
  const int type = R == 1 ? 0 : ((i & 1) | ((j & 1) << 1) | ((k & 1) << 2));
  const int Nf = fine.N;
  const T* __restrict__ rm = rf + (int64_t)m * fine.V;
  T acc = T(0);
  for (int e = __ldg(st_ptr + type); e < __ldg(st_ptr + type + 1); ++e) {
    const int o = __ldg(st_off + e);
    const int fi = 2 * i + (o & 31) - 8, fj = 2 * j + ((o >> 5) & 31) - 8, fk = 2 * k + ((o >> 10) & 31) - 8;
    if (fi < 0 || fj < 0 || fk < 0 || fi + fj + fk > Nf) continue;
    if (!((own >> zero_mask(Nf, fi, fj, fk)) & 1u)) continue;   // a copy owned by another macro
    acc += __ldg(st_w + e) * __ldg(rm + __ldg(fine.pstart + fk) + rowst32(Nf - fk, fj) + fi);
  }
  *out = acc;
}

// d = alpha d + beta dinv (b - y);  x += d
template <typename T>
__global__ void cheb_update_kernel(int64_t n, const T* __restrict__ b, const T* __restrict__ y,
                                   const T* __restrict__ dinv, T* __restrict__ x, T* __restrict__ d, T alpha, T beta) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    // the first step of a smoothing call (alpha = 0) must not read d: it holds the previous call's values
    const T dv = (alpha == T(0) ? T(0) : alpha * d[t]) + beta * dinv[t] * (b[t] - y[t]);
    d[t] = dv;
    x[t] += dv;
  }
}

// r = b - y
template <typename T>
__global__ void residual_kernel(int64_t n, const T* __restrict__ b, const T* __restrict__ y, T* __restrict__ r) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) r[t] = b[t] - y[t];
}

// x += a y (mixed types allowed: the update of an FP64 x by an FP32 correction)
template <typename TX, typename TY>
__global__ void axpy_kernel(int64_t n, TX* __restrict__ x, const TY* __restrict__ y, TX a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) x[t] += a * (TX)y[t];
}

template <typename TO, typename TI>
__global__ void convert_kernel(int64_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) out[t] = (TO)in[t];
}

// w = dinv * y
template <typename T>
__global__ void scale_kernel(int64_t n, const T* __restrict__ dinv, const T* __restrict__ y, T* __restrict__ w) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) w[t] = dinv[t] * y[t];
}

template <typename T>
__global__ void mul_scalar_kernel(int64_t n, T* __restrict__ x, T a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) x[t] *= a;
}

template <typename T>
__global__ void invert_kernel(int64_t n, T* __restrict__ d) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) d[t] = T(1) / d[t];
}

// 1/d, and 0 where d is 0 (the vertex points of a Nedelec vector, which carry no DoF)
template <typename T>
__global__ void invert_or_zero_kernel(int64_t n, T* __restrict__ d) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    d[t] = d[t] != T(0) ? T(1) / d[t] : T(0);
}

// Counter-based start vector of the power iteration: splitmix64 of (seed, position), uniform on [-1, 1),
// zero on Dirichlet points.
__global__ void start_vector_kernel(LevelArgs L, const MacroGeom* __restrict__ mg, uint64_t seed, double* __restrict__ v) {
  int i, j, k, p;
  if (!plane_point(L.N, L.cta_plane, L.cta_start, L.pstart, i, j, k, p)) return;
  const int m = blockIdx.y;
  const int64_t e = (int64_t)m * L.V + p;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  if (on_dirichlet(mg[m].bnd_table, L.N, i, j, k)) u = 0.0;
  v[e] = u;
}

// Dense coarse solve: x_int = Ainv b_int at the owner copies of the interior distinct points.
template <typename T>
__global__ void coarse_solve_kernel(int n0, const double* __restrict__ Ainv, const int64_t* __restrict__ pos,
                                    const T* __restrict__ b, T* __restrict__ x, int64_t nall) {
  // zero everything first (boundary and non-owner copies), then the interior owner copies
  for (int64_t t = threadIdx.x; t < nall; t += blockDim.x) x[t] = T(0);
  __syncthreads();
  for (int r = threadIdx.x; r < n0; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n0; ++c) s += Ainv[(int64_t)r * n0 + c] * (double)b[pos[c]];
    x[pos[r]] = (T)s;
  }
}

template <typename F>
static unsigned nblocks(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

}  // namespace hhg

using namespace hhg;

namespace hhg {
// Work buffers owned by the library for the standalone smoother / power iteration calls.
struct OpWork {
  void* y = nullptr;
  void* d = nullptr;
  size_t bytes = 0;
  ~OpWork() {
    cudaFree(y);
    cudaFree(d);
  }
  int reserve(size_t b) {
    if (b <= bytes) return HHG_OK;
    cudaFree(y);
    cudaFree(d);
    y = d = nullptr;
    bytes = 0;
    HHG_CUDA_TRY(cudaMalloc(&y, b));
    HHG_CUDA_TRY(cudaMalloc(&d, b));
    bytes = b;
    return HHG_OK;
  }
};

}  // namespace hhg

// ---------------------------------------------------------------------------
// Transfer entry points
// ---------------------------------------------------------------------------
// R = 1, 2: the scalar P1 / P2 tables; R = 3: the Nedelec edge tables (on the P2 position grid).
static TransferTables* transfer_tables(int R, int* status) {
  // per device, built on first use (device index up to 64)
  static TransferTables* cache[64][4] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) {
    *status = fail(HHG_E_CUDA, "device index out of range");
    return nullptr;
  }
  if (!cache[dev][R]) {
    TransferTables* T = new TransferTables();
    int st = R == 3 ? build_n1_transfer_tables(T) : build_transfer_tables(R, T);
    if (st != HHG_OK) {
      delete T;
      *status = st;
      return nullptr;
    }
    cache[dev][R] = T;
  }
  *status = HHG_OK;
  return cache[dev][R];
}

static LevelArgs level_args(const Interface* I, int N) {
  LevelArgs L;
  L.N = N;
  L.V = lattice_size(N);
  L.cta_plane = I->d_cta_plane;
  L.cta_start = I->d_cta_start;
  L.pstart = I->d_pstart;
  return L;
}

template <typename T>
static const T* pos_w(const TransferTables* TT);
template <>
const double* pos_w<double>(const TransferTables* TT) { return TT->d_pos_w64; }
template <>
const float* pos_w<float>(const TransferTables* TT) { return TT->d_pos_w32; }
template <typename T>
static const T* st_w(const TransferTables* TT);
template <>
const double* st_w<double>(const TransferTables* TT) { return TT->d_st_w64; }
template <>
const float* st_w<float>(const TransferTables* TT) { return TT->d_st_w32; }

template <typename T>
static int do_prolongate(hhg_mesh* mesh, int lf, int degree, const T* xc, T* xf, cudaStream_t s) {
  const Interface *If = nullptr, *Ic = nullptr;
  HHG_TRY(mesh->interface(lf, degree, &If));
  HHG_TRY(mesh->interface(lf - 1, degree, &Ic));
  int st = 0;
  TransferTables* TT = transfer_tables(degree, &st);
  if (!TT) return st;
  LevelArgs F = level_args(If, degree << lf), C = level_args(Ic, degree << (lf - 1));
  dim3 grid((unsigned)If->ncta, mesh->nmacro());
  if (degree == 1)
    prolongate_kernel<T, 1><<<grid, 256, 0, s>>>(F, C, TT->d_pos_off, pos_w<T>(TT), xc, xf);
  else
    prolongate_kernel<T, 2><<<grid, 256, 0, s>>>(F, C, TT->d_pos_off, pos_w<T>(TT), xc, xf);
  HHG_CUDA_TRY(cudaGetLastError());
  return launch_make_consistent<T>(If, xf, 1, s);
}

template <typename T>
static int do_restrict(hhg_mesh* mesh, int lf, int degree, const T* rf, T* rc, cudaStream_t s) {
  const Interface *If = nullptr, *Ic = nullptr;
  HHG_TRY(mesh->interface(lf, degree, &If));
  HHG_TRY(mesh->interface(lf - 1, degree, &Ic));
  int st = 0;
  TransferTables* TT = transfer_tables(degree, &st);
  if (!TT) return st;
  LevelArgs F = level_args(If, degree << lf), C = level_args(Ic, degree << (lf - 1));
  dim3 grid((unsigned)Ic->ncta, mesh->nmacro());
  if (degree == 1)
    restrict_kernel<T, 1><<<grid, 256, 0, s>>>(F, C, mesh->d_macros, TT->d_st_ptr, TT->d_st_off, st_w<T>(TT), rf, rc);
  else
    restrict_kernel<T, 2><<<grid, 256, 0, s>>>(F, C, mesh->d_macros, TT->d_st_ptr, TT->d_st_off, st_w<T>(TT), rf, rc);
  HHG_CUDA_TRY(cudaGetLastError());
  return launch_interface_sum<T>(Ic, rc, 1, true, s);
}

// Nedelec transfers: the same kernels on the doubled lattice with the edge tables; the copies of a
// shared edge carry their macro's orientation, so restriction sums them with signs, and the
// prolongation of a consistent coarse vector is consistent up to those signs.
template <typename T>
static int do_prolongate_n1(hhg_mesh* mesh, int lf, const T* xc, T* xf, cudaStream_t s) {
  const Interface *If = nullptr, *Ic = nullptr;
  HHG_TRY(mesh->interface(lf, 2, &If));
  HHG_TRY(mesh->interface(lf - 1, 2, &Ic));
  int st = 0;
  TransferTables* TT = transfer_tables(3, &st);
  if (!TT) return st;
  LevelArgs F = level_args(If, 2 << lf), C = level_args(Ic, 2 << (lf - 1));
  prolongate_kernel<T, 2><<<dim3((unsigned)If->ncta, mesh->nmacro()), 256, 0, s>>>(F, C, TT->d_pos_off, pos_w<T>(TT),
                                                                                    xc, xf);
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

template <typename T>
static int do_restrict_n1(hhg_mesh* mesh, int lf, const T* rf, T* rc, cudaStream_t s) {
  const Interface *If = nullptr, *Ic = nullptr;
  HHG_TRY(mesh->interface(lf, 2, &If));
  HHG_TRY(mesh->interface(lf - 1, 2, &Ic));
  int st = 0;
  TransferTables* TT = transfer_tables(3, &st);
  if (!TT) return st;
  LevelArgs F = level_args(If, 2 << lf), C = level_args(Ic, 2 << (lf - 1));
  restrict_kernel<T, 2><<<dim3((unsigned)Ic->ncta, mesh->nmacro()), 256, 0, s>>>(
      F, C, mesh->d_macros, TT->d_st_ptr, TT->d_st_off, st_w<T>(TT), rf, rc);
  HHG_CUDA_TRY(cudaGetLastError());
  return launch_interface_sum_signed<T>(Ic, rc, true, s);
}

// Discrete gradient G: P1 vertex values p (level l) -> edge values of level l, the tangential
// integral of grad p along the canonical direction d of the edge, p(m + d) - p(m - d) in doubled
// coordinates m; vertex points of the doubled lattice get 0.
template <typename T>
__global__ void __launch_bounds__(256) n1_gradient_kernel(LevelArgs E, LevelArgs P1, const T* __restrict__ p,
                                                           T* __restrict__ out) {
  int i, j, k, q;
  if (!plane_point(E.N, E.cta_plane, E.cta_start, E.pstart, i, j, k, q)) return;
  const int m = blockIdx.y;
  T v = T(0);
  if ((i | j | k) & 1) {
    int d[3];
    const int pi = i & 1, pj = j & 1, pk = k & 1;
    d[0] = pi;
    d[1] = pj;
    d[2] = pk;
    if (pi && pj) d[1] = -1;
    else if ((pi || pj) && pk) d[2] = -1;
    const int ai = (i - d[0]) >> 1, aj = (j - d[1]) >> 1, ak = (k - d[2]) >> 1;
    const int bi = (i + d[0]) >> 1, bj = (j + d[1]) >> 1, bk = (k + d[2]) >> 1;
    const T* __restrict__ pm = p + (int64_t)m * P1.V;
    v = __ldg(pm + __ldg(P1.pstart + bk) + rowst32(P1.N - bk, bj) + bi) -
        __ldg(pm + __ldg(P1.pstart + ak) + rowst32(P1.N - ak, aj) + ai);
  }
  out[(int64_t)m * E.V + q] = v;
}

// Its transpose G^T: edge values r (level l) -> P1 vertex values, sum over the 14 incident edges of
// r_e (the edge ends at the vertex) or -r_e (starts there), over the edge copies this macro owns;
// Dirichlet vertices get 0.  The caller adds the macro copies of shared vertices.
template <typename T>
__global__ void __launch_bounds__(256) n1_gradient_t_kernel(LevelArgs P1, LevelArgs E, const MacroGeom* __restrict__ mg,
                                                             const T* __restrict__ r, T* __restrict__ out) {
  int i, j, k, q;
  if (!plane_point(P1.N, P1.cta_plane, P1.cta_start, P1.pstart, i, j, k, q)) return;
  const int m = blockIdx.y;
  const uint32_t bnd = mg[m].bnd_table, own = mg[m].own_table;
  T* o = out + (int64_t)m * P1.V + q;
  if (on_dirichlet(bnd, P1.N, i, j, k)) {
    *o = T(0);
    return;
  }
  const T* __restrict__ rm = r + (int64_t)m * E.V;
  const int NE = E.N;
  T acc = T(0);
  constexpr int kDir[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, -1, 0}, {1, 0, -1}, {0, 1, -1}, {1, -1, 1}};
#pragma unroll
  for (int t = 0; t < 7; ++t) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      // side 0: the edge starting at the vertex (midpoint 2v + d); side 1: ending there (2v - d)
      const int sgn = side == 0 ? 1 : -1;
      const int ei = 2 * i + sgn * kDir[t][0], ej = 2 * j + sgn * kDir[t][1], ek = 2 * k + sgn * kDir[t][2];
      if (ei < 0 || ej < 0 || ek < 0 || ei + ej + ek > NE) continue;
      if (!((own >> zero_mask(NE, ei, ej, ek)) & 1u)) continue;   // a copy owned by another macro
      const T v = __ldg(rm + __ldg(E.pstart + ek) + rowst32(NE - ek, ej) + ei);
      acc += side == 0 ? -v : v;
    }
  }
  *o = acc;
}

static int check_transfer_args(const hhg_mesh_t* mesh, int lf, int degree, const void* a, const void* b, int dtype) {
  if (!mesh || !a || !b) return fail(HHG_E_ARG, "transfer: null pointer");
  if (lf < 1 || lf > mesh->level) return fail(HHG_E_ARG, "transfer: fine level %d outside 1..%d", lf, mesh->level);
  if (degree != 1 && degree != 2) return fail(HHG_E_ARG, "transfer: degree must be 1 or 2");
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "transfer: bad dtype");
  return HHG_OK;
}

extern "C" int hhg_prolongate(const hhg_mesh_t* mesh, int level_fine, int degree, const void* xc, void* xf, int dtype,
                              void* stream) {
  clear_error();
  HHG_TRY(check_transfer_args(mesh, level_fine, degree, xc, xf, dtype));
  hhg_mesh* m = const_cast<hhg_mesh*>(mesh);
  if (dtype == HHG_F64)
    return do_prolongate<double>(m, level_fine, degree, (const double*)xc, (double*)xf, (cudaStream_t)stream);
  return do_prolongate<float>(m, level_fine, degree, (const float*)xc, (float*)xf, (cudaStream_t)stream);
}

extern "C" int hhg_restrict(const hhg_mesh_t* mesh, int level_fine, int degree, const void* rf, void* rc, int dtype,
                            void* stream) {
  clear_error();
  HHG_TRY(check_transfer_args(mesh, level_fine, degree, rf, rc, dtype));
  hhg_mesh* m = const_cast<hhg_mesh*>(mesh);
  if (dtype == HHG_F64)
    return do_restrict<double>(m, level_fine, degree, (const double*)rf, (double*)rc, (cudaStream_t)stream);
  return do_restrict<float>(m, level_fine, degree, (const float*)rf, (float*)rc, (cudaStream_t)stream);
}

template <typename T>
static int do_gradient(hhg_mesh* mesh, int level, const T* p, T* e, bool transpose, cudaStream_t s) {
  const Interface *I1 = nullptr, *I2 = nullptr;
  HHG_TRY(mesh->interface(level, 1, &I1));
  HHG_TRY(mesh->interface(level, 2, &I2));
  const LevelArgs P1 = level_args(I1, 1 << level), E = level_args(I2, 2 << level);
  if (!transpose) {
    n1_gradient_kernel<T><<<dim3((unsigned)I2->ncta, mesh->nmacro()), 256, 0, s>>>(E, P1, p, e);
    HHG_CUDA_TRY(cudaGetLastError());
    return HHG_OK;
  }
  n1_gradient_t_kernel<T><<<dim3((unsigned)I1->ncta, mesh->nmacro()), 256, 0, s>>>(P1, E, mesh->d_macros, e,
                                                                                   const_cast<T*>(p));
  HHG_CUDA_TRY(cudaGetLastError());
  return launch_interface_sum<T>(I1, const_cast<T*>(p), 1, true, s);
}

extern "C" int hhg_prolongate_edges(const hhg_mesh_t* mesh, int level_fine, const void* xc, void* xf, int dtype,
                                    void* stream) {
  clear_error();
  HHG_TRY(check_transfer_args(mesh, level_fine, 2, xc, xf, dtype));
  hhg_mesh* m = const_cast<hhg_mesh*>(mesh);
  const Interface* If = nullptr;
  HHG_TRY(m->interface(level_fine, 2, &If));
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == HHG_F64) {
    HHG_TRY(do_prolongate_n1<double>(m, level_fine, (const double*)xc, (double*)xf, s));
    return launch_make_consistent_signed<double>(If, (double*)xf, s);
  }
  HHG_TRY(do_prolongate_n1<float>(m, level_fine, (const float*)xc, (float*)xf, s));
  return launch_make_consistent_signed<float>(If, (float*)xf, s);
}

extern "C" int hhg_restrict_edges(const hhg_mesh_t* mesh, int level_fine, const void* rf, void* rc, int dtype,
                                  void* stream) {
  clear_error();
  HHG_TRY(check_transfer_args(mesh, level_fine, 2, rf, rc, dtype));
  hhg_mesh* m = const_cast<hhg_mesh*>(mesh);
  if (dtype == HHG_F64)
    return do_restrict_n1<double>(m, level_fine, (const double*)rf, (double*)rc, (cudaStream_t)stream);
  return do_restrict_n1<float>(m, level_fine, (const float*)rf, (float*)rc, (cudaStream_t)stream);
}

extern "C" int hhg_gradient(const hhg_mesh_t* mesh, int level, const void* p, void* e, int dtype, void* stream) {
  clear_error();
  if (!mesh || !p || !e) return fail(HHG_E_ARG, "gradient: null pointer");
  if (level < 0 || level > mesh->level) return fail(HHG_E_ARG, "gradient: level %d outside 0..%d", level, mesh->level);
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "gradient: bad dtype");
  hhg_mesh* m = const_cast<hhg_mesh*>(mesh);
  if (dtype == HHG_F64) return do_gradient<double>(m, level, (const double*)p, (double*)e, false, (cudaStream_t)stream);
  return do_gradient<float>(m, level, (const float*)p, (float*)e, false, (cudaStream_t)stream);
}

extern "C" int hhg_gradient_transpose(const hhg_mesh_t* mesh, int level, const void* e, void* p, int dtype,
                                      void* stream) {
  clear_error();
  if (!mesh || !p || !e) return fail(HHG_E_ARG, "gradient_transpose: null pointer");
  if (level < 0 || level > mesh->level)
    return fail(HHG_E_ARG, "gradient_transpose: level %d outside 0..%d", level, mesh->level);
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "gradient_transpose: bad dtype");
  hhg_mesh* m = const_cast<hhg_mesh*>(mesh);
  if (dtype == HHG_F64) return do_gradient<double>(m, level, (double*)p, (double*)e, true, (cudaStream_t)stream);
  return do_gradient<float>(m, level, (float*)p, (float*)e, true, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Smoother and power iteration
// ---------------------------------------------------------------------------
template <typename T>
static int cheb_smooth_t(hhg_op* op, const T* b, T* x, const T* dinv, double lam, double lo, double hi, int order,
                         T* y, T* d, cudaStream_t s) {
  const double a = lo * lam, bb = hi * lam;
  const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int64_t n = op->npts;
  for (int it = 0; it < order; ++it) {
    HHG_TRY(hhg_op_apply(op, x, y, sizeof(T) == 8 ? HHG_F64 : HHG_F32, 1, s));
    double alpha, beta;
    if (it == 0) {
      alpha = 0.0;
      beta = 1.0 / theta;
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      alpha = rho_new * rho;
      beta = 2.0 * rho_new / delta;
      rho = rho_new;
    }
    cheb_update_kernel<T><<<nblocks<T>(n), 256, 0, s>>>(n, b, y, dinv, x, d, (T)alpha, (T)beta);
    HHG_CUDA_TRY(cudaGetLastError());
  }
  return HHG_OK;
}

extern "C" int hhg_cheb_smooth(hhg_op_t* op, const void* b, void* x, const void* dinv, double lam, double lo,
                               double hi, int order, int dtype, void* stream) {
  clear_error();
  if (!op || !b || !x || !dinv) return fail(HHG_E_ARG, "cheb_smooth: null pointer");
  if (order < 1 || !(lam > 0) || !(hi > lo) || !(lo > 0)) return fail(HHG_E_ARG, "cheb_smooth: bad parameters");
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "cheb_smooth: bad dtype");
  if (op->kind != HHG_DIFFUSION) return fail(HHG_E_UNSUPPORTED, "cheb_smooth: scalar operators only");
  if (!op->work) op->work = new OpWork();
  const size_t es = dtype == HHG_F64 ? 8 : 4;
  HHG_TRY(op->work->reserve(es * op->npts));
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == HHG_F64)
    return cheb_smooth_t<double>(op, (const double*)b, (double*)x, (const double*)dinv, lam, lo, hi, order,
                                 (double*)op->work->y, (double*)op->work->d, s);
  return cheb_smooth_t<float>(op, (const float*)b, (float*)x, (const float*)dinv, lam, lo, hi, order,
                              (float*)op->work->y, (float*)op->work->d, s);
}

// ---------------------------------------------------------------------------
// Chebyshev smoothing without device allocation.
//
// hhg_cheb_smooth allocates its two work vectors (A x and the Chebyshev direction)
// with cudaMalloc the first time it runs on an operator.  Some callers must not
// allocate device memory once they are running: processes whose device memory is
// entirely handed to another allocator (a framework's caching pool), so that a
// cudaMalloc would fail or fragment it, and latency-critical loops where the
// device-wide synchronisation of cudaMalloc is not acceptable.  The variant below
// takes its work vectors from a fixed array in the library's device image instead.
// ---------------------------------------------------------------------------
// Capacity: two work vectors of at most kNoAllocPoints entries each (FP64 or FP32),
// 8 MiB in all; every GPU that loads the library holds the array until the process exits.
constexpr int64_t kNoAllocPoints = (int64_t)1 << 19;
static __device__ __align__(256) double g_smooth_scratch[2 * kNoAllocPoints];

// Device address of g_smooth_scratch on the current device, looked up once per device.
// (In host code the name g_smooth_scratch is only a host-side stand-in for the array.)
static int noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  HHG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(HHG_E_CUDA, "cheb_smooth_noalloc: device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_smooth_scratch);
    if (e != cudaSuccess || !p)
      return fail(HHG_E_CUDA, "cheb_smooth_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    addr[dev] = p;
  }
  *out = addr[dev];
  return HHG_OK;
}

// Looks the scratch array up on the current device ahead of the first hhg_cheb_smooth_noalloc call:
// called by operator creation, which allocates anyway, so that the lookup (which can load the
// library's device image) never happens inside the allocation-free entry point.
int hhg::noalloc_prepare() {
  void* p = nullptr;
  return noalloc_scratch(&p);
}

template <typename T>
static int power_t(hhg_op* op, const T* dinv, T* v, int iters, double* lam, T* y, cudaStream_t s) {
  const int dt = sizeof(T) == 8 ? HHG_F64 : HHG_F32;
  const int64_t n = op->npts;
  double nv = 0.0;
  HHG_TRY(hhg_vec_dot(op->mesh, op->level, op->degree, v, v, dt, 1, &nv, s));
  if (!(nv > 0)) return fail(HHG_E_ARG, "power_iteration: zero start vector");
  mul_scalar_kernel<T><<<nblocks<T>(n), 256, 0, s>>>(n, v, (T)(1.0 / std::sqrt(nv)));
  double l = 0.0;
  for (int it = 0; it < iters; ++it) {
    HHG_TRY(hhg_op_apply(op, v, y, dt, 1, s));
    scale_kernel<T><<<nblocks<T>(n), 256, 0, s>>>(n, dinv, y, v);
    HHG_TRY(hhg_vec_dot(op->mesh, op->level, op->degree, v, v, dt, 1, &nv, s));
    l = std::sqrt(nv);
    if (!(l > 0) || !std::isfinite(l)) return fail(HHG_E_NAN, "power_iteration: norm %g", l);
    mul_scalar_kernel<T><<<nblocks<T>(n), 256, 0, s>>>(n, v, (T)(1.0 / l));
  }
  HHG_CUDA_TRY(cudaGetLastError());
  *lam = l;
  return HHG_OK;
}

extern "C" int hhg_cheb_smooth_noalloc(hhg_op_t* op, const void* b, void* x, const void* dinv, double lam,
                                       double lo, double hi, int order, int dtype, void* stream) {
  clear_error();
  if (!op || !b || !x || !dinv) return fail(HHG_E_ARG, "cheb_smooth_noalloc: null pointer");
  if (order < 1 || !(lam > 0) || !(hi > lo) || !(lo > 0)) return fail(HHG_E_ARG, "cheb_smooth_noalloc: bad parameters");
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "cheb_smooth_noalloc: bad dtype");
  if (op->kind != HHG_DIFFUSION) return fail(HHG_E_UNSUPPORTED, "cheb_smooth_noalloc: scalar operators only");
  if (op->npts > kNoAllocPoints)
    return fail(HHG_E_ARG,
                "cheb_smooth_noalloc: the operator's vectors have %lld entries; the fixed scratch holds at most %lld "
                "per vector (use hhg_cheb_smooth)",
                (long long)op->npts, (long long)kNoAllocPoints);
  void* scratch = nullptr;
  HHG_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  // y = A x occupies the first kNoAllocPoints entries, the direction d the next ones.  Neither
  // needs clearing: the apply writes y before it is read, and the first update writes d
  // without reading it.
  if (dtype == HHG_F64) {
    double* y = (double*)scratch;
    return cheb_smooth_t<double>(op, (const double*)b, (double*)x, (const double*)dinv, lam, lo, hi, order, y,
                                 y + kNoAllocPoints, s);
  }
  float* y = (float*)scratch;
  return cheb_smooth_t<float>(op, (const float*)b, (float*)x, (const float*)dinv, lam, lo, hi, order, y,
                              y + kNoAllocPoints, s);
}

extern "C" int hhg_power_iteration(hhg_op_t* op, const void* dinv, void* v, int iters, int dtype, double* lam,
                                   void* stream) {
  clear_error();
  if (!op || !dinv || !v || !lam || iters < 1) return fail(HHG_E_ARG, "power_iteration: bad argument");
  if (dtype != HHG_F32 && dtype != HHG_F64) return fail(HHG_E_ARG, "power_iteration: bad dtype");
  if (!op->work) op->work = new OpWork();
  HHG_TRY(op->work->reserve((dtype == HHG_F64 ? 8 : 4) * op->npts));
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == HHG_F64)
    return power_t<double>(op, (const double*)dinv, (double*)v, iters, lam, (double*)op->work->y, s);
  return power_t<float>(op, (const float*)dinv, (float*)v, iters, lam, (float*)op->work->y, s);
}

// ---------------------------------------------------------------------------
// Load vector and L2 error of the manufactured solution u = sin(pi x) sin(pi y) sin(pi z)
// ---------------------------------------------------------------------------
extern "C" int hhg_rhs_sin3_poisson(const hhg_mesh_t* mesh, int level, int degree, double* b, void* stream) {
  clear_error();
  if (!mesh || !b) return fail(HHG_E_ARG, "rhs: null pointer");
  hhg_coeff_t c{HHG_COEFF_CONST, 1.0, nullptr, HHG_F64};
  hhg_op_t* op = nullptr;
  HHG_TRY(hhg_op_create(const_cast<hhg_mesh_t*>(mesh), level, HHG_DIFFUSION, degree, &c, HHG_DIRICHLET, 5, &op));
  std::unique_ptr<hhg_op> hold(op);
  cudaStream_t s = (cudaStream_t)stream;
  HHG_TRY(launch_march<double>(op, (const OpConst<double>*)op->d_const64, 3, nullptr, nullptr, nullptr, b, s));
  HHG_TRY(launch_interface_sum<double>(op->itf, b, 1, true, s));
  HHG_CUDA_TRY(cudaStreamSynchronize(s));   // the temporary operator is freed on return
  return HHG_OK;
}

extern "C" int hhg_l2_error_sin3(const hhg_mesh_t* mesh, int level, int degree, const double* uh, double* err,
                                 void* stream) {
  clear_error();
  if (!mesh || !uh || !err) return fail(HHG_E_ARG, "l2_error: null pointer");
  hhg_coeff_t c{HHG_COEFF_CONST, 1.0, nullptr, HHG_F64};
  hhg_op_t* op = nullptr;
  HHG_TRY(hhg_op_create(const_cast<hhg_mesh_t*>(mesh), level, HHG_DIFFUSION, degree, &c, HHG_DIRICHLET, 5, &op));
  std::unique_ptr<hhg_op> hold(op);
  hhg_mesh* m = const_cast<hhg_mesh*>(mesh);
  const int64_t nblk = launch_l2_blocks(op);
  HHG_TRY(m->scratch_reserve(sizeof(double) * (nblk + 1)));
  cudaStream_t s = (cudaStream_t)stream;
  HHG_TRY(launch_l2_error(op, uh, (double*)m->d_scratch, s));
  std::vector<double> part(nblk);
  HHG_CUDA_TRY(cudaMemcpyAsync(part.data(), m->d_scratch, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s));
  HHG_CUDA_TRY(cudaStreamSynchronize(s));
  double sum = 0.0;
  for (double v : part) sum += v;
  *err = std::sqrt(sum);
  return HHG_OK;
}

// ---------------------------------------------------------------------------
// Multigrid hierarchy and solver
// ---------------------------------------------------------------------------
namespace hhg {
struct MGLevel {
  hhg_op* op = nullptr;      // the level's operator (finest: the caller's op)
  bool owned = false;
  int64_t n = 0;
  double lam = 1.0;
  double *dinv64 = nullptr, *x64 = nullptr, *b64 = nullptr, *r64 = nullptr, *y64 = nullptr, *d64 = nullptr;
  float *dinv32 = nullptr, *x32 = nullptr, *b32 = nullptr, *r32 = nullptr, *y32 = nullptr, *d32 = nullptr;
  // Nedelec hierarchies: the nodal operator G^T A G of the hybrid smoother (the P1 diffusion operator
  // with coefficient beta, Dirichlet) and its vectors over the level's P1 lattice
  hhg_op* pop = nullptr;
  int64_t np = 0;
  double lam_p = 1.0;
  double *pdinv64 = nullptr, *px64 = nullptr, *pb64 = nullptr, *py64 = nullptr, *pd64 = nullptr;
  float *pdinv32 = nullptr, *px32 = nullptr, *pb32 = nullptr, *py32 = nullptr, *pd32 = nullptr;
};

struct MGHierarchy {
  bool n1 = false;           // Nedelec (curl-curl + mass) hierarchy with Hiptmair's hybrid smoother
  int L = 0, coarse = 0;
  std::vector<MGLevel> lv;
  int n0 = 0;
  double* Ainv = nullptr;
  int64_t* pos = nullptr;
  double* xf64 = nullptr;     // finest-level FP64 work (residual, apply)
  double* rf64 = nullptr;
  double setup_ms = 0.0;
  ~MGHierarchy() {
    for (auto& l : lv) {
      for (void* p : {(void*)l.dinv64, (void*)l.x64, (void*)l.b64, (void*)l.r64, (void*)l.y64, (void*)l.d64,
                      (void*)l.dinv32, (void*)l.x32, (void*)l.b32, (void*)l.r32, (void*)l.y32, (void*)l.d32,
                      (void*)l.pdinv64, (void*)l.px64, (void*)l.pb64, (void*)l.py64, (void*)l.pd64,
                      (void*)l.pdinv32, (void*)l.px32, (void*)l.pb32, (void*)l.py32, (void*)l.pd32})
        cudaFree(p);
      if (l.owned) delete l.op;
      delete l.pop;
    }
    cudaFree(Ainv);
    cudaFree(pos);
    cudaFree(xf64);
    cudaFree(rf64);
  }
};

void destroy_mg(MGHierarchy* h) { delete h; }
void destroy_work(OpWork* w) { delete w; }

}  // namespace hhg

template <typename T>
static int vcycle(MGHierarchy* H, int l, const T* b, T* x, const hhg_mg_opts_t* o, cudaStream_t s);

template <typename T>
struct Buf;
template <>
struct Buf<double> {
  static double* x(MGLevel& l) { return l.x64; }
  static double* b(MGLevel& l) { return l.b64; }
  static double* r(MGLevel& l) { return l.r64; }
  static double* y(MGLevel& l) { return l.y64; }
  static double* d(MGLevel& l) { return l.d64; }
  static double* dinv(MGLevel& l) { return l.dinv64; }
};
template <>
struct Buf<float> {
  static float* x(MGLevel& l) { return l.x32; }
  static float* b(MGLevel& l) { return l.b32; }
  static float* r(MGLevel& l) { return l.r32; }
  static float* y(MGLevel& l) { return l.y32; }
  static float* d(MGLevel& l) { return l.d32; }
  static float* dinv(MGLevel& l) { return l.dinv32; }
};
// the nodal vectors of a Nedelec level
template <typename T>
struct PBuf;
template <>
struct PBuf<double> {
  static double* x(MGLevel& l) { return l.px64; }
  static double* b(MGLevel& l) { return l.pb64; }
  static double* y(MGLevel& l) { return l.py64; }
  static double* d(MGLevel& l) { return l.pd64; }
  static double* dinv(MGLevel& l) { return l.pdinv64; }
};
template <>
struct PBuf<float> {
  static float* x(MGLevel& l) { return l.px32; }
  static float* b(MGLevel& l) { return l.pb32; }
  static float* y(MGLevel& l) { return l.py32; }
  static float* d(MGLevel& l) { return l.pd32; }
  static float* dinv(MGLevel& l) { return l.pdinv32; }
};

// Transfers of the hierarchy's space.
template <typename T>
static int mg_restrict(MGHierarchy* H, int l, const T* rf, T* rc, cudaStream_t s) {
  hhg_op* op = H->lv[l].op;
  return H->n1 ? do_restrict_n1<T>(op->mesh, l, rf, rc, s) : do_restrict<T>(op->mesh, l, op->degree, rf, rc, s);
}
template <typename T>
static int mg_prolongate(MGHierarchy* H, int l, const T* xc, T* xf, cudaStream_t s) {
  hhg_op* op = H->lv[l].op;
  if (!H->n1) return do_prolongate<T>(op->mesh, l, op->degree, xc, xf, s);
  HHG_TRY(do_prolongate_n1<T>(op->mesh, l, xc, xf, s));
  return launch_make_consistent_signed<T>(op->itf, xf, s);
}

// Hiptmair's hybrid smoothing step on a Nedelec level (Section 8): a Chebyshev step on the edges,
// then one on the gradients of the interior vertices, r_p = G^T (b - A x), p = Chebyshev(A_p, r_p,
// 0) with A_p = G^T A G (the P1 diffusion operator with coefficient beta), and x += G p.
template <typename T>
static int hybrid_smooth(MGLevel& L, const T* b, T* x, const hhg_mg_opts_t* o, cudaStream_t s) {
  const int dt = sizeof(T) == 8 ? HHG_F64 : HHG_F32;
  HHG_TRY(cheb_smooth_t<T>(L.op, b, x, Buf<T>::dinv(L), L.lam, o->cheb_lo, o->cheb_hi, o->cheb_order, Buf<T>::y(L),
                           Buf<T>::d(L), s));
  HHG_TRY(hhg_op_apply(L.op, x, Buf<T>::y(L), dt, 1, s));
  residual_kernel<T><<<nblocks<T>(L.n), 256, 0, s>>>(L.n, b, Buf<T>::y(L), Buf<T>::r(L));
  const Interface* I1 = L.pop->itf;
  const LevelArgs P1 = level_args(I1, L.pop->N), E = level_args(L.op->itf, L.op->N);
  const int nm = L.op->mesh->nmacro();
  n1_gradient_t_kernel<T><<<dim3((unsigned)I1->ncta, nm), 256, 0, s>>>(P1, E, L.op->mesh->d_macros, Buf<T>::r(L),
                                                                       PBuf<T>::b(L));
  HHG_CUDA_TRY(cudaGetLastError());
  HHG_TRY(launch_interface_sum<T>(I1, PBuf<T>::b(L), 1, true, s));
  HHG_CUDA_TRY(cudaMemsetAsync(PBuf<T>::x(L), 0, sizeof(T) * L.np, s));
  HHG_TRY(cheb_smooth_t<T>(L.pop, PBuf<T>::b(L), PBuf<T>::x(L), PBuf<T>::dinv(L), L.lam_p, o->cheb_lo, o->cheb_hi,
                           o->cheb_order, PBuf<T>::y(L), PBuf<T>::d(L), s));
  n1_gradient_kernel<T><<<dim3((unsigned)L.op->itf->ncta, nm), 256, 0, s>>>(E, P1, PBuf<T>::x(L), Buf<T>::y(L));
  axpy_kernel<T, T><<<nblocks<T>(L.n), 256, 0, s>>>(L.n, x, Buf<T>::y(L), T(1));
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

template <typename T>
static int mg_smooth(MGHierarchy* H, MGLevel& L, const T* b, T* x, const hhg_mg_opts_t* o, cudaStream_t s) {
  if (H->n1) return hybrid_smooth<T>(L, b, x, o, s);
  return cheb_smooth_t<T>(L.op, b, x, Buf<T>::dinv(L), L.lam, o->cheb_lo, o->cheb_hi, o->cheb_order, Buf<T>::y(L),
                          Buf<T>::d(L), s);
}

template <typename T>
static int coarse_solve(MGHierarchy* H, const T* b, T* x, cudaStream_t s) {
  MGLevel& l = H->lv[H->coarse];
  coarse_solve_kernel<T><<<1, 256, 0, s>>>(H->n0, H->Ainv, H->pos, b, x, l.n);
  HHG_CUDA_TRY(cudaGetLastError());
  return H->n1 ? launch_make_consistent_signed<T>(l.op->itf, x, s) : launch_make_consistent<T>(l.op->itf, x, 1, s);
}

template <typename T>
static int vcycle(MGHierarchy* H, int l, const T* b, T* x, const hhg_mg_opts_t* o, cudaStream_t s) {
  if (l == H->coarse) return coarse_solve<T>(H, b, x, s);
  MGLevel& L = H->lv[l];
  MGLevel& C = H->lv[l - 1];
  const int dt = sizeof(T) == 8 ? HHG_F64 : HHG_F32;
  for (int it = 0; it < o->nu1; ++it) HHG_TRY(mg_smooth<T>(H, L, b, x, o, s));
  HHG_TRY(hhg_op_apply(L.op, x, Buf<T>::y(L), dt, 1, s));
  residual_kernel<T><<<nblocks<T>(L.n), 256, 0, s>>>(L.n, b, Buf<T>::y(L), Buf<T>::r(L));
  HHG_TRY(mg_restrict<T>(H, l, Buf<T>::r(L), Buf<T>::b(C), s));
  HHG_CUDA_TRY(cudaMemsetAsync(Buf<T>::x(C), 0, sizeof(T) * C.n, s));
  HHG_TRY(vcycle<T>(H, l - 1, Buf<T>::b(C), Buf<T>::x(C), o, s));
  HHG_TRY(mg_prolongate<T>(H, l, Buf<T>::x(C), Buf<T>::y(L), s));
  axpy_kernel<T, T><<<nblocks<T>(L.n), 256, 0, s>>>(L.n, x, Buf<T>::y(L), T(1));
  for (int it = 0; it < o->nu2; ++it) HHG_TRY(mg_smooth<T>(H, L, b, x, o, s));
  HHG_CUDA_TRY(cudaGetLastError());
  return HHG_OK;
}

static int setup_mg(hhg_op* op, const hhg_mg_opts_t* o, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  std::unique_ptr<MGHierarchy> H(new MGHierarchy());
  H->L = op->level;
  H->coarse = o->coarse_level;
  if (H->coarse < 0 || H->coarse > H->L) return fail(HHG_E_ARG, "mg: coarse level %d outside 0..%d", H->coarse, H->L);
  H->n1 = op->kind == HHG_CURLCURL;
  H->lv.resize(H->L + 1);
  for (int l = H->coarse; l <= H->L; ++l) {
    MGLevel& lv = H->lv[l];
    if (l == H->L) {
      lv.op = op;
    } else {
      hhg_op_t* c = nullptr;
      if (H->n1)
        HHG_TRY(hhg_op_create_curlcurl(op->mesh, l, &op->coeff, &op->coeff2, op->bc, &c));
      else
        HHG_TRY(hhg_op_create(op->mesh, l, op->kind, op->degree, &op->coeff, op->bc, op->quad_degree, &c));
      lv.op = c;
      lv.owned = true;
      // the coarse operators take the fine one's FP64 arithmetic (double-float where it is set)
      if (op->d_dfx) HHG_TRY(hhg_op_set_fp64_arith(c, HHG_FP64_DOUBLE_FLOAT));
    }
    lv.n = lv.op->npts;
    for (double** p : {&lv.dinv64, &lv.x64, &lv.b64, &lv.r64, &lv.y64, &lv.d64})
      HHG_CUDA_TRY(cudaMalloc(p, sizeof(double) * lv.n));
    for (float** p : {&lv.dinv32, &lv.x32, &lv.b32, &lv.r32, &lv.y32, &lv.d32})
      HHG_CUDA_TRY(cudaMalloc(p, sizeof(float) * lv.n));
    HHG_TRY(hhg_op_diagonal(lv.op, lv.dinv64, HHG_F64, s));
    if (H->n1)
      invert_or_zero_kernel<double><<<nblocks<double>(lv.n), 256, 0, s>>>(lv.n, lv.dinv64);
    else
      invert_kernel<double><<<nblocks<double>(lv.n), 256, 0, s>>>(lv.n, lv.dinv64);
    convert_kernel<float, double><<<nblocks<float>(lv.n), 256, 0, s>>>(lv.n, lv.dinv64, lv.dinv32);
    HHG_CUDA_TRY(cudaGetLastError());
    if (l > H->coarse) {
      // lambda_max of D^{-1} A from a seeded counter-based start vector
      LevelArgs LA = level_args(lv.op->itf, lv.op->N);
      start_vector_kernel<<<dim3((unsigned)lv.op->itf->ncta, op->mesh->nmacro()), 256, 0, s>>>(LA, op->mesh->d_macros,
                                                                                             12345u, lv.x64);
      HHG_CUDA_TRY(cudaGetLastError());
      if (H->n1)
        HHG_TRY(launch_make_consistent_signed<double>(lv.op->itf, lv.x64, s));
      else
        HHG_TRY(launch_make_consistent<double>(lv.op->itf, lv.x64, 1, s));
      HHG_TRY(power_t<double>(lv.op, lv.dinv64, lv.x64, o->power_iters, &lv.lam, lv.y64, s));
    }
    if (H->n1 && l > H->coarse) {
      // the nodal part of the hybrid smoother: G^T A G over the level's P1 lattice is the P1
      // diffusion operator with coefficient beta (Dirichlet: interior vertices only)
      hhg_op_t* p = nullptr;
      HHG_TRY(hhg_op_create(op->mesh, l, HHG_DIFFUSION, 1, &op->coeff2, HHG_DIRICHLET, 2, &p));
      lv.pop = p;
      lv.np = p->npts;
      for (double** q : {&lv.pdinv64, &lv.px64, &lv.pb64, &lv.py64, &lv.pd64})
        HHG_CUDA_TRY(cudaMalloc(q, sizeof(double) * lv.np));
      for (float** q : {&lv.pdinv32, &lv.px32, &lv.pb32, &lv.py32, &lv.pd32})
        HHG_CUDA_TRY(cudaMalloc(q, sizeof(float) * lv.np));
      HHG_TRY(hhg_op_diagonal(p, lv.pdinv64, HHG_F64, s));
      invert_kernel<double><<<nblocks<double>(lv.np), 256, 0, s>>>(lv.np, lv.pdinv64);
      convert_kernel<float, double><<<nblocks<float>(lv.np), 256, 0, s>>>(lv.np, lv.pdinv64, lv.pdinv32);
      LevelArgs LP = level_args(p->itf, p->N);
      start_vector_kernel<<<dim3((unsigned)p->itf->ncta, op->mesh->nmacro()), 256, 0, s>>>(LP, op->mesh->d_macros,
                                                                                         54321u, lv.px64);
      HHG_CUDA_TRY(cudaGetLastError());
      HHG_TRY(launch_make_consistent<double>(p->itf, lv.px64, 1, s));
      HHG_TRY(power_t<double>(p, lv.pdinv64, lv.px64, o->power_iters, &lv.lam_p, lv.py64, s));
    }
  }
  HHG_CUDA_TRY(cudaMalloc(&H->xf64, sizeof(double) * op->npts));
  HHG_CUDA_TRY(cudaMalloc(&H->rf64, sizeof(double) * op->npts));
  // coarse level: dense matrix of the interior distinct points, inverted by Cholesky on the host
  {
    MGLevel& c = H->lv[H->coarse];
    const Interface* I = c.op->itf;
    const int N = c.op->N;
    const int64_t V = lattice_size(N);
    std::vector<uint8_t> nonowner(c.n, 0);
    for (int64_t g = 0; g < I->ngroups; ++g)
      for (int64_t t = I->h_ptr[g] + 1; t < I->h_ptr[g + 1]; ++t) nonowner[I->h_idx[t]] = 1;
    std::vector<int64_t> pos;
    for (int m = 0; m < op->mesh->nmacro(); ++m) {
      const uint32_t tb = op->mesh->macros[m].bnd_table;
      int64_t p = 0;
      for (int k = 0; k <= N; ++k)
        for (int j = 0; j + k <= N; ++j)
          for (int i = 0; i + j + k <= N; ++i, ++p) {
            const int z = (N - i - j - k == 0) | ((i == 0) << 1) | ((j == 0) << 2) | ((k == 0) << 3);
            const bool bnd = op->bc == HHG_DIRICHLET && ((tb >> z) & 1);
            const int64_t e = (int64_t)m * V + p;
            const bool dof = !H->n1 || ((i | j | k) & 1);   // Nedelec: edge midpoints only
            if (dof && !bnd && !nonowner[e]) pos.push_back(e);
          }
    }
    H->n0 = (int)pos.size();
    if (H->n0 > 4096) return fail(HHG_E_UNSUPPORTED, "mg: coarse level has %d interior points (max 4096)", H->n0);
    const int n0 = H->n0;
    std::vector<double> A((size_t)n0 * n0, 0.0), col(c.n);
    std::vector<double> e(c.n, 0.0);
    for (int r = 0; r < n0; ++r) {
      std::fill(e.begin(), e.end(), 0.0);
      e[pos[r]] = 1.0;
      HHG_CUDA_TRY(cudaMemcpyAsync(c.x64, e.data(), sizeof(double) * c.n, cudaMemcpyHostToDevice, s));
      if (H->n1)
        HHG_TRY(launch_make_consistent_signed<double>(I, c.x64, s));
      else
        HHG_TRY(launch_make_consistent<double>(I, c.x64, 1, s));
      HHG_TRY(hhg_op_apply(c.op, c.x64, c.y64, HHG_F64, 1, s));
      HHG_CUDA_TRY(cudaMemcpyAsync(col.data(), c.y64, sizeof(double) * c.n, cudaMemcpyDeviceToHost, s));
      HHG_CUDA_TRY(cudaStreamSynchronize(s));
      for (int q = 0; q < n0; ++q) A[(size_t)q * n0 + r] = col[pos[q]];
    }
    // Cholesky A = L L^T, then the inverse column by column
    std::vector<double> Lm(A);
    for (int j = 0; j < n0; ++j) {
      double d = Lm[(size_t)j * n0 + j];
      for (int k = 0; k < j; ++k) d -= Lm[(size_t)j * n0 + k] * Lm[(size_t)j * n0 + k];
      if (!(d > 0)) return fail(HHG_E_ARG, "mg: coarse matrix is not positive definite");
      d = std::sqrt(d);
      Lm[(size_t)j * n0 + j] = d;
      for (int i = j + 1; i < n0; ++i) {
        double v = Lm[(size_t)i * n0 + j];
        for (int k = 0; k < j; ++k) v -= Lm[(size_t)i * n0 + k] * Lm[(size_t)j * n0 + k];
        Lm[(size_t)i * n0 + j] = v / d;
      }
    }
    std::vector<double> Ainv((size_t)std::max(n0, 1) * std::max(n0, 1), 0.0), z(n0);
    for (int cix = 0; cix < n0; ++cix) {
      for (int i = 0; i < n0; ++i) {
        double v = i == cix ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) v -= Lm[(size_t)i * n0 + k] * z[k];
        z[i] = v / Lm[(size_t)i * n0 + i];
      }
      for (int i = n0 - 1; i >= 0; --i) {
        double v = z[i];
        for (int k = i + 1; k < n0; ++k) v -= Lm[(size_t)k * n0 + i] * Ainv[(size_t)k * n0 + cix];
        Ainv[(size_t)i * n0 + cix] = v / Lm[(size_t)i * n0 + i];
      }
    }
    HHG_CUDA_TRY(cudaMalloc(&H->Ainv, sizeof(double) * Ainv.size()));
    HHG_CUDA_TRY(cudaMalloc(&H->pos, sizeof(int64_t) * std::max<size_t>(pos.size(), 1)));
    HHG_CUDA_TRY(cudaMemcpy(H->Ainv, Ainv.data(), sizeof(double) * Ainv.size(), cudaMemcpyHostToDevice));
    if (!pos.empty()) HHG_CUDA_TRY(cudaMemcpy(H->pos, pos.data(), sizeof(int64_t) * pos.size(), cudaMemcpyHostToDevice));
  }
  HHG_CUDA_TRY(cudaStreamSynchronize(s));
  H->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  op->mg = H.release();
  return HHG_OK;
}

template <typename T>
static int fmg_t(MGHierarchy* H, const double* b, const hhg_mg_opts_t* o, cudaStream_t s) {
  // right-hand sides of every level by restriction, then coarse solve and one V-cycle per level
  MGLevel& F = H->lv[H->L];
  if (sizeof(T) == 8)
    HHG_CUDA_TRY(cudaMemcpyAsync(F.b64, b, sizeof(double) * F.n, cudaMemcpyDeviceToDevice, s));
  else
    convert_kernel<float, double><<<nblocks<float>(F.n), 256, 0, s>>>(F.n, b, F.b32);
  for (int l = H->L; l > H->coarse; --l)
    HHG_TRY(mg_restrict<T>(H, l, Buf<T>::b(H->lv[l]), Buf<T>::b(H->lv[l - 1]), s));
  HHG_TRY(coarse_solve<T>(H, Buf<T>::b(H->lv[H->coarse]), Buf<T>::x(H->lv[H->coarse]), s));
  for (int l = H->coarse + 1; l <= H->L; ++l) {
    HHG_TRY(mg_prolongate<T>(H, l, Buf<T>::x(H->lv[l - 1]), Buf<T>::x(H->lv[l]), s));
    // x_l is needed as the V-cycle's iterate; the level's y / r / d buffers are its scratch
    HHG_TRY(vcycle<T>(H, l, Buf<T>::b(H->lv[l]), Buf<T>::x(H->lv[l]), o, s));
  }
  return HHG_OK;
}

extern "C" int hhg_mg_default_opts(hhg_mg_opts_t* o) {
  if (!o) return fail(HHG_E_ARG, "mg_default_opts: null");
  o->nu1 = 2;
  o->nu2 = 2;
  o->cheb_order = 2;
  o->power_iters = 15;
  o->cheb_lo = 0.1;
  o->cheb_hi = 1.1;
  o->tol = 1e-10;
  o->max_iters = 50;
  o->mixed = 0;
  o->fmg = 1;
  o->coarse_level = 0;
  return HHG_OK;
}

extern "C" int hhg_mg_solve(hhg_op_t* op, const double* b, double* x, const hhg_mg_opts_t* opts, hhg_mg_stats_t* stats,
                            void* stream) {
  clear_error();
  if (!op || !b || !x || !opts) return fail(HHG_E_ARG, "mg_solve: null pointer");
  const bool n1 = op->kind == HHG_CURLCURL;
  if (op->bc != HHG_DIRICHLET)
    return fail(HHG_E_UNSUPPORTED, "mg_solve: needs a DIRICHLET operator");
  if (!n1 && (op->kind != HHG_DIFFUSION || (op->coeff.type != HHG_COEFF_CONST && op->coeff.type != HHG_COEFF_SIN3)))
    return fail(HHG_E_UNSUPPORTED, "mg_solve: needs a diffusion operator with CONST or SIN3 coefficient, or a "
                                   "curl-curl operator");
  if (n1 && (op->coeff.type != HHG_COEFF_CONST || op->coeff2.type != HHG_COEFF_CONST))
    return fail(HHG_E_UNSUPPORTED, "mg_solve: the curl-curl hierarchy takes CONST alpha and beta");
  if (opts->nu1 < 0 || opts->nu2 < 0 || opts->cheb_order < 1 || opts->max_iters < 0 || !(opts->tol > 0))
    return fail(HHG_E_ARG, "mg_solve: bad options");
  cudaStream_t s = (cudaStream_t)stream;
  if (op->mg && (op->mg->coarse != opts->coarse_level)) {
    destroy_mg(op->mg);
    op->mg = nullptr;
  }
  double setup_ms = 0.0;
  if (!op->mg) {
    HHG_TRY(setup_mg(op, opts, s));
    setup_ms = op->mg->setup_ms;
  }
  MGHierarchy* H = op->mg;
  MGLevel& F = H->lv[H->L];
  const int64_t n = F.n;
  // the events are released on every path, errors included
  struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } ev;
  HHG_CUDA_TRY(cudaEventCreate(&ev.e0));
  HHG_CUDA_TRY(cudaEventCreate(&ev.e1));
  HHG_CUDA_TRY(cudaEventRecord(ev.e0, s));
  int it = 0;
  double rel = 0.0;
  // FMG, then outer iterations; every exit of the body leaves the iteration count and the last
  // residual for the statistics
  auto body = [&]() -> int {
    double nb2 = 0.0;
    HHG_TRY(hhg_vec_dot(op->mesh, op->level, op->degree, b, b, HHG_F64, 1, &nb2, s));
    const double nb = std::sqrt(nb2);
    if (opts->fmg) {
      if (opts->mixed) {
        HHG_TRY(fmg_t<float>(H, b, opts, s));
        convert_kernel<double, float><<<nblocks<double>(n), 256, 0, s>>>(n, F.x32, x);
      } else {
        HHG_TRY(fmg_t<double>(H, b, opts, s));
        HHG_CUDA_TRY(cudaMemcpyAsync(x, F.x64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      }
    }
    for (;; ++it) {
      // outer residual in FP64
      HHG_TRY(hhg_op_apply(op, x, H->xf64, HHG_F64, 1, s));
      residual_kernel<double><<<nblocks<double>(n), 256, 0, s>>>(n, b, H->xf64, H->rf64);
      double r2 = 0.0;
      HHG_TRY(hhg_vec_dot(op->mesh, op->level, op->degree, H->rf64, H->rf64, HHG_F64, 1, &r2, s));
      rel = nb > 0 ? std::sqrt(r2) / nb : std::sqrt(r2);
      if (stats && it < 64) stats->residual_history[it] = rel;
      if (!std::isfinite(rel)) return fail(HHG_E_NAN, "mg_solve: residual is not finite");
      if (rel <= opts->tol) return HHG_OK;
      if (it >= opts->max_iters)
        return fail(HHG_E_NOT_CONVERGED, "mg_solve: relative residual %.3e after %d iterations", rel, it);
      // correction c = V(r) from zero, in the inner precision; x += c in FP64
      if (opts->mixed) {
        convert_kernel<float, double><<<nblocks<float>(n), 256, 0, s>>>(n, H->rf64, F.b32);
        HHG_CUDA_TRY(cudaMemsetAsync(F.x32, 0, sizeof(float) * n, s));
        HHG_TRY(vcycle<float>(H, H->L, F.b32, F.x32, opts, s));
        axpy_kernel<double, float><<<nblocks<double>(n), 256, 0, s>>>(n, x, F.x32, 1.0);
      } else {
        HHG_CUDA_TRY(cudaMemcpyAsync(F.b64, H->rf64, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        HHG_CUDA_TRY(cudaMemsetAsync(F.x64, 0, sizeof(double) * n, s));
        HHG_TRY(vcycle<double>(H, H->L, F.b64, F.x64, opts, s));
        axpy_kernel<double, double><<<nblocks<double>(n), 256, 0, s>>>(n, x, F.x64, 1.0);
      }
      HHG_CUDA_TRY(cudaGetLastError());
    }
  };
  const int status = body();
  float ms = 0.f;
  if (cudaEventRecord(ev.e1, s) == cudaSuccess && cudaEventSynchronize(ev.e1) == cudaSuccess)
    cudaEventElapsedTime(&ms, ev.e0, ev.e1);
  if (stats) {
    stats->iterations = it;
    stats->rel_residual = rel;
    stats->setup_ms = setup_ms;
    stats->solve_ms = ms;
  }
  return status;
}
