// Device helpers for the packed tetrahedral lattice of one macro (Section 2: implicit,
// analytical index maps; no stored connectivity).
#pragma once

#include <cstdint>

namespace hhg {

// Device copies of the class tables (same values as kClassOffsets / kP2Edges in mesh.cpp).
static __constant__ int kClassOffsetsD[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {1, 1, 0}},
    {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {0, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {1, 0, 0}},
    {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},
};
// The 15 P1 stencil offsets (same order as kStencil in mesh.cpp).
static __constant__ int kStencilD[15][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}, {1, -1, 1}, {-1, 1, -1}};
static __constant__ int kP2EdgesD[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// Number of lattice points with i+j+k <= s (V(s) = (s+1)(s+2)(s+3)/6; V(-1) = 0).
__device__ __forceinline__ int64_t dV(int64_t s) { return (s + 1) * (s + 2) * (s + 3) / 6; }

// First packed position of plane k (resolution N): V(N) - V(N-k).
__device__ __forceinline__ int64_t plane_start(int N, int k) { return dV(N) - dV(N - k); }

// Offset of row j inside a plane with s = N - k: sum_{j' < j} (s - j' + 1).
__device__ __forceinline__ int64_t row_start(int s, int j) {
  return (int64_t)j * (s + 1) - ((int64_t)j * (j - 1)) / 2;
}

__device__ __forceinline__ int64_t packed_index(int N, int i, int j, int k) {
  return plane_start(N, k) + row_start(N - k, j) + i;
}

// Inverse of packed_index: plane by the cubic V, row by the quadratic row_start.
__device__ __forceinline__ void decode_point(int64_t p, int N, int& i, int& j, int& k) {
  const int64_t R = dV(N) - p;   // plane k holds p iff V(s-1) < R <= V(s), s = N - k
  int s = (int)cbrtf(6.0f * (float)R) - 2;
  if (s < 0) s = 0;
  while (dV(s) < R) ++s;
  while (s > 0 && dV(s - 1) >= R) --s;
  k = N - s;
  const int64_t q = p - (dV(N) - dV(s));
  const float b = 2.0f * s + 3.0f;
  int jj = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * (float)q, 0.0f))));
  if (jj < 0) jj = 0;
  if (jj > s) jj = s;
  while (jj < s && row_start(s, jj + 1) <= q) ++jj;
  while (jj > 0 && row_start(s, jj) > q) --jj;
  j = jj;
  i = (int)(q - row_start(s, jj));
}

// Zero-set mask of the barycentric weights (N-i-j-k, i, j, k): bit a set iff weight a is 0.
__device__ __forceinline__ int zero_mask(int N, int i, int j, int k) {
  return (N - i - j - k == 0) | ((i == 0) << 1) | ((j == 0) << 2) | ((k == 0) << 3);
}

__device__ __forceinline__ bool on_dirichlet(uint32_t table, int N, int i, int j, int k) {
  return (table >> zero_mask(N, i, j, k)) & 1u;
}

__device__ __forceinline__ bool inside(int N, int i, int j, int k) {
  return i >= 0 && j >= 0 && k >= 0 && i + j + k <= N;
}

}  // namespace hhg
