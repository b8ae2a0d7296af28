// Macro mesh set-up: validation, boundary classification, interface groups, quadrature rules.
//
// Section 2: the coarse grid is an unstructured mesh of macro-tetrahedra; each
// is refined uniformly and addressed by implicit index maps.  The library keeps
// every macro's closure in its own packed block; points shared between macros
// (on macro faces, edges, vertices) are reconciled by "interface groups".
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <set>
#include <string>
#include <tuple>

#include "hhg_internal.h"

namespace hhg {

const int kClassOffsets[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},   // white up
    {{0, 1, 0}, {1, 0, 1}, {1, 0, 0}, {1, 1, 0}},   // octahedron tets around (0,1,0)-(1,0,1)
    {{0, 1, 0}, {1, 0, 1}, {1, 1, 0}, {0, 1, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 1, 1}, {0, 0, 1}},
    {{0, 1, 0}, {1, 0, 1}, {0, 0, 1}, {1, 0, 0}},
    {{1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}},   // white down
};
const int kClassShrink[6] = {0, 1, 1, 1, 1, 2};
const int kP2Edges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
// The 15 points of the P1 stencil: the point itself and its neighbours along the 7 edge directions.
const int kStencil[15][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0}, {0, 0, 1},  {0, 0, -1}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1},  {0, -1, 1}, {1, -1, 1}, {-1, 1, -1}};

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
void clear_error() { g_err.clear(); }

Interface::~Interface() {
  cudaFree(d_ptr);
  cudaFree(d_idx);
  cudaFree(d_bnd);
  cudaFree(d_cta_plane);
  cudaFree(d_cta_start);
  cudaFree(d_pstart);
  cudaFree(d_march_tasks);
  for (TileTasks& t : tile) cudaFree(t.d);
  cudaFree(d_sign);
}

// ---------------------------------------------------------------------------
// Quadrature rules (reference tetrahedron, volume 1/6).
//   degree 1: centroid.  degree 2: symmetric 4-point rule, barycentric (b,a,a,a)
//   with a = (5 - sqrt 5)/20.  degree 3..5: fully symmetric 14-point rule with
//   orbits (a1,a1,a1,1-3a1), (a2,a2,a2,1-3a2), (b,b,1/2-b,1/2-b) whose six
//   parameters solve the moment equations (Newton on the symmetric invariants).
// ---------------------------------------------------------------------------
static void orbit31(double a, std::vector<double>& xi) {
  for (int pos = 0; pos < 4; ++pos) {
    double lam[4] = {a, a, a, a};
    lam[pos] = 1.0 - 3.0 * a;
    xi.push_back(lam[1]);
    xi.push_back(lam[2]);
    xi.push_back(lam[3]);
  }
}
static void orbit22(double b, std::vector<double>& xi) {
  double c = 0.5 - b;
  // the six distinct arrangements of (b,b,c,c)
  const int pat[6][4] = {{0, 0, 1, 1}, {0, 1, 0, 1}, {0, 1, 1, 0}, {1, 0, 0, 1}, {1, 0, 1, 0}, {1, 1, 0, 0}};
  for (auto& p : pat) {
    double lam[4];
    for (int t = 0; t < 4; ++t) lam[t] = p[t] ? c : b;
    xi.push_back(lam[1]);
    xi.push_back(lam[2]);
    xi.push_back(lam[3]);
  }
}
static double fact(int k) {
  double r = 1;
  for (int i = 2; i <= k; ++i) r *= i;
  return r;
}
// Moment residuals of the 14-point family against all monomials of degree <= 5.
static void rule14(const double th[6], std::vector<double>& xi, std::vector<double>& w) {
  xi.clear();
  w.clear();
  orbit31(th[0], xi);
  orbit31(th[2], xi);
  orbit22(th[4], xi);
  for (int q = 0; q < 4; ++q) w.push_back(th[1]);
  for (int q = 0; q < 4; ++q) w.push_back(th[3]);
  for (int q = 0; q < 6; ++q) w.push_back(th[5]);
}
static void residual14(const double th[6], std::vector<double>& r) {
  std::vector<double> xi, w;
  rule14(th, xi, w);
  r.clear();
  for (int a = 0; a <= 5; ++a)
    for (int b = 0; a + b <= 5; ++b)
      for (int c = 0; a + b + c <= 5; ++c) {
        double s = 0;
        for (size_t q = 0; q < w.size(); ++q)
          s += w[q] * std::pow(xi[3 * q], a) * std::pow(xi[3 * q + 1], b) * std::pow(xi[3 * q + 2], c);
        r.push_back(s - fact(a) * fact(b) * fact(c) / fact(a + b + c + 3));
      }
}
// Solve the (consistent, overdetermined) moment system by Gauss-Newton with normal equations.
static bool solve14(double th[6]) {
  const double init[6] = {0.1, 1.0 / 84, 0.3, 1.0 / 84, 0.45, 1.0 / 84};
  std::memcpy(th, init, sizeof(init));
  std::vector<double> r, rp, rm;
  for (int it = 0; it < 100; ++it) {
    residual14(th, r);
    size_t m = r.size();
    std::vector<double> J(m * 6);
    for (int p = 0; p < 6; ++p) {
      double tp[6], tm[6];
      std::memcpy(tp, th, sizeof(tp));
      std::memcpy(tm, th, sizeof(tm));
      tp[p] += 1e-7;
      tm[p] -= 1e-7;
      residual14(tp, rp);
      residual14(tm, rm);
      for (size_t e = 0; e < m; ++e) J[e * 6 + p] = (rp[e] - rm[e]) / 2e-7;
    }
    double NtN[6][7] = {};
    for (int a = 0; a < 6; ++a) {
      for (int b = 0; b < 6; ++b)
        for (size_t e = 0; e < m; ++e) NtN[a][b] += J[e * 6 + a] * J[e * 6 + b];
      for (size_t e = 0; e < m; ++e) NtN[a][6] -= J[e * 6 + a] * r[e];
    }
    // Gaussian elimination with partial pivoting
    for (int c = 0; c < 6; ++c) {
      int piv = c;
      for (int rr = c + 1; rr < 6; ++rr)
        if (std::fabs(NtN[rr][c]) > std::fabs(NtN[piv][c])) piv = rr;
      for (int k = 0; k < 7; ++k) std::swap(NtN[c][k], NtN[piv][k]);
      if (NtN[c][c] == 0) return false;
      for (int rr = c + 1; rr < 6; ++rr) {
        double f = NtN[rr][c] / NtN[c][c];
        for (int k = c; k < 7; ++k) NtN[rr][k] -= f * NtN[c][k];
      }
    }
    double step[6];
    for (int c = 5; c >= 0; --c) {
      double s = NtN[c][6];
      for (int k = c + 1; k < 6; ++k) s -= NtN[c][k] * step[k];
      step[c] = s / NtN[c][c];
    }
    double mx = 0;
    for (int p = 0; p < 6; ++p) {
      th[p] += step[p];
      mx = std::max(mx, std::fabs(step[p]));
    }
    if (mx < 1e-17) break;
  }
  residual14(th, r);
  double mx = 0;
  for (double v : r) mx = std::max(mx, std::fabs(v));
  return mx < 1e-14;
}

int quad_rule(int degree, QuadRule* out) {
  out->xi.clear();
  out->w.clear();
  if (degree <= 1) {
    out->xi = {0.25, 0.25, 0.25};
    out->w = {1.0 / 6.0};
    return HHG_OK;
  }
  if (degree == 2) {
    orbit31((5.0 - std::sqrt(5.0)) / 20.0, out->xi);
    out->w.assign(4, 1.0 / 24.0);
    return HHG_OK;
  }
  if (degree <= 5) {
    static double th[6];
    static int solved = 0;   // 0 unknown, 1 ok, -1 failed
    if (solved == 0) solved = solve14(th) ? 1 : -1;
    if (solved < 0) return fail(HHG_E_UNSUPPORTED, "14-point quadrature rule did not converge");
    rule14(th, out->xi, out->w);
    return HHG_OK;
  }
  return fail(HHG_E_UNSUPPORTED, "quadrature degree %d not supported (1..5)", degree);
}

}  // namespace hhg

using namespace hhg;

// ---------------------------------------------------------------------------
// Mesh
// ---------------------------------------------------------------------------
hhg_mesh::~hhg_mesh() {
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(device);
  iface.clear();
  cudaFree(d_macros);
  cudaFree(d_scratch);
  cudaSetDevice(cur);
}

namespace {
using Face = std::array<int32_t, 3>;
using Edge = std::array<int32_t, 2>;

// Key of a lattice point: its (vertex id, integer barycentric weight) pairs with
// nonzero weight, sorted by vertex id.  Shared points have equal keys.
struct PointKey {
  uint64_t k[4];
  int64_t pos;
  uint8_t bnd;
  int8_t dir_tail_first;   // edge points: +1 if the canonical direction's tail has the smaller key
  bool operator<(const PointKey& o) const {
    for (int t = 0; t < 4; ++t)
      if (k[t] != o.k[t]) return k[t] < o.k[t];
    return pos < o.pos;
  }
  bool same(const PointKey& o) const {
    return k[0] == o.k[0] && k[1] == o.k[1] && k[2] == o.k[2] && k[3] == o.k[3];
  }
};

}  // namespace

extern "C" const char* hhg_last_error(void) { return g_err.c_str(); }

extern "C" int hhg_mesh_create(const double* vx, int64_t nv, const int32_t* tx, int64_t nt, int level,
                               hhg_mesh_t** out) {
  clear_error();
  if (!vx || !tx || !out || nv < 4 || nt < 1) return fail(HHG_E_ARG, "mesh_create: null pointer or empty mesh");
  if (level < 0 || level > 10) return fail(HHG_E_ARG, "mesh_create: level %d outside 0..10", level);
  *out = nullptr;
  std::unique_ptr<hhg_mesh> m(new hhg_mesh());
  m->level = level;
  cudaGetDevice(&m->device);
  m->vertices.assign(vx, vx + 3 * nv);
  m->tets.assign(tx, tx + 4 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 4; ++a)
      if (tx[4 * t + a] < 0 || tx[4 * t + a] >= nv) return fail(HHG_E_ARG, "mesh_create: vertex index out of range");
  // geometry and degeneracy
  m->macros.resize(nt);
  for (int64_t t = 0; t < nt; ++t) {
    MacroGeom& g = m->macros[t];
    const double* P[4];
    for (int a = 0; a < 4; ++a) {
      g.vid[a] = tx[4 * t + a];
      P[a] = vx + 3 * tx[4 * t + a];
    }
    double len = 0;
    for (int d = 0; d < 3; ++d) g.p0[d] = P[0][d];
    for (int a = 0; a < 3; ++a) {
      double l2 = 0;
      for (int d = 0; d < 3; ++d) {
        g.e[a][d] = P[a + 1][d] - P[0][d];
        l2 += g.e[a][d] * g.e[a][d];
      }
      len = std::max(len, std::sqrt(l2));
    }
    double det = g.e[0][0] * (g.e[1][1] * g.e[2][2] - g.e[1][2] * g.e[2][1]) -
                 g.e[0][1] * (g.e[1][0] * g.e[2][2] - g.e[1][2] * g.e[2][0]) +
                 g.e[0][2] * (g.e[1][0] * g.e[2][1] - g.e[1][1] * g.e[2][0]);
    if (!(std::fabs(det) / 6.0 > 1e-12 * len * len * len))
      return fail(HHG_E_DEGENERATE, "mesh_create: macro %lld is degenerate", (long long)t);
  }
  // faces: interior faces have two macros, boundary faces one
  std::map<Face, int> face_count;
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 4; ++a) {
      Face f;
      int c = 0;
      for (int b = 0; b < 4; ++b)
        if (b != a) f[c++] = tx[4 * t + b];
      std::sort(f.begin(), f.end());
      if (++face_count[f] > 2) return fail(HHG_E_NONMANIFOLD, "mesh_create: a face is shared by more than two macros");
    }
  std::set<Edge> bnd_edges;
  std::set<int32_t> bnd_verts;
  for (auto& kv : face_count)
    if (kv.second == 1) {
      const Face& f = kv.first;
      for (int a = 0; a < 3; ++a) {
        bnd_verts.insert(f[a]);
        for (int b = a + 1; b < 3; ++b) bnd_edges.insert(Edge{std::min(f[a], f[b]), std::max(f[a], f[b])});
      }
    }
  // macros around every vertex, edge and face (for the owner tables)
  std::map<std::vector<int32_t>, int> lowest;
  for (int64_t t = 0; t < nt; ++t)
    for (int z = 1; z < 15; ++z) {
      std::vector<int32_t> key;
      for (int a = 0; a < 4; ++a)
        if (!(z & (1 << a))) key.push_back(tx[4 * t + a]);
      std::sort(key.begin(), key.end());
      auto it = lowest.find(key);
      if (it == lowest.end() || it->second > (int)t) lowest[key] = (int)t;
    }
  // boundary table per macro, indexed by the zero set z of the weights (w0, w1, w2, w3)
  for (int64_t t = 0; t < nt; ++t) {
    MacroGeom& g = m->macros[t];
    uint32_t table = 0;
    for (int z = 1; z < 15; ++z) {
      int nz = __builtin_popcount(z);
      std::vector<int> rest;
      for (int a = 0; a < 4; ++a)
        if (!(z & (1 << a))) rest.push_back(a);
      bool b = false;
      if (nz == 1) {
        Face f{g.vid[rest[0]], g.vid[rest[1]], g.vid[rest[2]]};
        std::sort(f.begin(), f.end());
        b = face_count[f] == 1;
      } else if (nz == 2) {
        Edge e{std::min(g.vid[rest[0]], g.vid[rest[1]]), std::max(g.vid[rest[0]], g.vid[rest[1]])};
        b = bnd_edges.count(e) > 0;
      } else if (nz == 3) {
        b = bnd_verts.count(g.vid[rest[0]]) > 0;
      }
      if (b) table |= 1u << z;
    }
    g.bnd_table = table;
    uint32_t own = 1u;   // z = 0: interior points belong to this macro only
    for (int z = 1; z < 15; ++z) {
      std::vector<int32_t> key;
      for (int a = 0; a < 4; ++a)
        if (!(z & (1 << a))) key.push_back(g.vid[a]);
      std::sort(key.begin(), key.end());
      if (lowest[key] == (int)t) own |= 1u << z;
    }
    g.own_table = own;
  }
  HHG_CUDA_TRY(cudaMalloc(&m->d_macros, sizeof(MacroGeom) * nt));
  HHG_CUDA_TRY(cudaMemcpy(m->d_macros, m->macros.data(), sizeof(MacroGeom) * nt, cudaMemcpyHostToDevice));
  *out = m.release();
  return HHG_OK;
}

int hhg_mesh::scratch_reserve(size_t bytes) {
  if (bytes <= scratch_bytes) return HHG_OK;
  cudaFree(d_scratch);
  d_scratch = nullptr;
  scratch_bytes = 0;
  HHG_CUDA_TRY(cudaMalloc(&d_scratch, bytes));
  scratch_bytes = bytes;
  return HHG_OK;
}

extern "C" int hhg_mesh_destroy(hhg_mesh_t* mesh) {
  delete mesh;
  return HHG_OK;
}

// Build (once) the interface groups of (level, degree).
// Tasks of a plane-tile kernel on one macro lattice of resolution N: tiles of iw points along i
// and jw rows, k-chunks (from 32) halved until the list (times the macros it holds) has min_tasks
// tasks, heaviest first.  copies: the macros the list holds (nmacro() for one launch over all
// macros, 1 for a launch per macro, whose tasks then carry macro 0).
int hhg_mesh::build_tile_tasks(int64_t N, int64_t iw, int64_t jw, int copies, int64_t min_tasks, TileTasks* out) const {
  int kch = 32;
  std::vector<std::pair<int64_t, int4>> tasks;
  for (;;) {
    tasks.clear();
    for (int64_t kc = 0; kc * kch <= N; ++kc)
      for (int64_t ty = 0; ty * jw + kc * kch <= N; ++ty)
        for (int64_t tx = 0; tx * iw + ty * jw + kc * kch <= N; ++tx) {
          int64_t work = 0;
          for (int64_t k = kc * kch; k < std::min<int64_t>(kc * kch + kch, N + 1); ++k)
            for (int64_t j = ty * jw; j < ty * jw + jw; ++j) {
              const int64_t len = N - j - k + 1 - tx * iw;   // points of the row from the chunk start
              if (len > 0) work += std::min<int64_t>(len, iw);
            }
          tasks.push_back({work, int4{(int)tx, (int)ty, (int)kc, 0}});
        }
    if (kch <= 4 || (int64_t)tasks.size() * copies >= min_tasks) break;
    kch /= 2;
  }
  std::vector<std::pair<int64_t, int4>> all;
  for (int mac = 0; mac < copies; ++mac)
    for (auto& t : tasks) all.push_back({t.first, int4{t.second.x, t.second.y, t.second.z, mac}});
  std::stable_sort(all.begin(), all.end(), [](const std::pair<int64_t, int4>& a, const std::pair<int64_t, int4>& b) {
    return a.first > b.first;
  });
  std::vector<int4> tv(all.size());
  for (size_t t = 0; t < all.size(); ++t) tv[t] = all[t].second;
  out->kchunk = kch;
  out->n = (int64_t)tv.size();
  HHG_CUDA_TRY(cudaMalloc(&out->d, sizeof(int4) * tv.size()));
  HHG_CUDA_TRY(cudaMemcpy(out->d, tv.data(), sizeof(int4) * tv.size(), cudaMemcpyHostToDevice));
  return HHG_OK;
}

int hhg_mesh::interface(int lvl, int degree, const Interface** out) {
  if (lvl < 0 || lvl > level) return fail(HHG_E_ARG, "level %d outside 0..%d", lvl, level);
  if (degree != 1 && degree != 2) return fail(HHG_E_ARG, "degree must be 1 or 2");
  int key = lvl * 8 + degree;
  auto it = iface.find(key);
  if (it != iface.end()) {
    *out = it->second.get();
    return HHG_OK;
  }
  std::unique_ptr<Interface> I(new Interface());
  const int64_t N = (int64_t)degree << lvl;
  const int64_t V = lattice_size(N);
  std::vector<PointKey> keys;
  int64_t nbnd_points = 0;
  for (int mac = 0; mac < nmacro(); ++mac) {
    const MacroGeom& g = macros[mac];
    for (int64_t k = 0; k <= N; ++k)
      for (int64_t j = 0; j + k <= N; ++j) {
        int64_t m = N - k;
        int64_t rowbase = (V - lattice_size(N - k)) + j * (m + 1) - j * (j - 1) / 2;
        for (int64_t i = 0; i + j + k <= N; ++i) {
          int64_t w[4] = {N - i - j - k, i, j, k};
          int z = (w[0] == 0) | ((w[1] == 0) << 1) | ((w[2] == 0) << 2) | ((w[3] == 0) << 3);
          if (z == 0) {
            // interior of the macro: skip to the last point of the row
            i = std::max(i, N - j - k - 1);
            continue;
          }
          if ((g.bnd_table >> z) & 1) ++nbnd_points;
          PointKey pk;
          std::array<std::pair<int32_t, int64_t>, 4> pr;
          int c = 0;
          for (int a = 0; a < 4; ++a)
            if (w[a] > 0) pr[c++] = {g.vid[a], w[a]};
          std::sort(pr.begin(), pr.begin() + c);
          for (int t = 0; t < 4; ++t)
            pk.k[t] = t < c ? ((uint64_t)(uint32_t)pr[t].first << 32) | (uint64_t)pr[t].second : ~0ull;
          pk.pos = mac * V + rowbase + i;
          pk.bnd = (g.bnd_table >> z) & 1;
          pk.dir_tail_first = 1;
          if (degree == 2 && ((i | j | k) & 1)) {
            // edge midpoint: endpoints (p -+ d) / 2 along the canonical direction d of its parity;
            // orientation relative to a macro-independent order of the endpoints' keys
            const int pi = (int)(i & 1), pj = (int)(j & 1), pkk = (int)(k & 1);
            int d[3] = {pi, pj, pkk};
            if (pi && pj && !pkk) d[1] = -1;
            if (pi && !pj && pkk) d[2] = -1;
            if (!pi && pj && pkk) d[2] = -1;
            if (pi && pj && pkk) d[1] = -1;
            std::array<std::array<uint64_t, 4>, 2> ek;
            for (int side = 0; side < 2; ++side) {
              const int sg = side == 0 ? -1 : 1;
              const int64_t ti = (i + sg * d[0]) / 2, tj = (j + sg * d[1]) / 2, tk = (k + sg * d[2]) / 2;
              const int64_t n1 = N / 2;
              const int64_t wv[4] = {n1 - ti - tj - tk, ti, tj, tk};
              std::array<std::pair<int32_t, int64_t>, 4> pv;
              int cv = 0;
              for (int a = 0; a < 4; ++a)
                if (wv[a] > 0) pv[cv++] = {g.vid[a], wv[a]};
              std::sort(pv.begin(), pv.begin() + cv);
              for (int t = 0; t < 4; ++t)
                ek[side][t] = t < cv ? ((uint64_t)(uint32_t)pv[t].first << 32) | (uint64_t)pv[t].second : ~0ull;
            }
            pk.dir_tail_first = ek[0] < ek[1] ? 1 : -1;
          }
          keys.push_back(pk);
        }
      }
  }
  std::sort(keys.begin(), keys.end());
  std::vector<int64_t> ptr{0}, idx;
  std::vector<uint8_t> bnd;
  std::vector<int8_t> sgn;
  int64_t dup = 0, dup_bnd = 0;
  for (size_t a = 0; a < keys.size();) {
    size_t b = a + 1;
    while (b < keys.size() && keys[b].same(keys[a])) ++b;
    if (b - a >= 2) {
      for (size_t t = a; t < b; ++t) {
        idx.push_back(keys[t].pos);
        sgn.push_back((int8_t)(keys[t].dir_tail_first * keys[a].dir_tail_first));
      }
      ptr.push_back((int64_t)idx.size());
      uint8_t isb = keys[a].bnd;   // equal for all copies
      bnd.push_back(isb);
      dup += (int64_t)(b - a) - 1;
      if (isb) dup_bnd += (int64_t)(b - a) - 1;
    }
    a = b;
  }
  I->ngroups = (int64_t)bnd.size();
  I->nmembers = (int64_t)idx.size();
  I->ndof_total = nmacro() * V - dup;
  int64_t nb_unique = nbnd_points - dup_bnd;
  I->ndof_interior = I->ndof_total - nb_unique;
  // plane launch tables (32-bit in-macro indexing)
  if (V >= ((int64_t)1 << 31)) return fail(HHG_E_UNSUPPORTED, "level too fine for 32-bit in-macro indexing");
  {
    std::vector<int> cta_start(N + 2), pstart(N + 2), cta_plane;
    int64_t ncta = 0, p = 0;
    for (int64_t k = 0; k <= N + 1; ++k) {
      cta_start[k] = (int)ncta;
      pstart[k] = (int)p;
      if (k <= N) {
        const int64_t s = N - k, cnt = (s + 1) * (s + 2) / 2, nb = (cnt + 255) / 256;
        for (int64_t b = 0; b < nb; ++b) cta_plane.push_back((int)k);
        ncta += nb;
        p += cnt;
      }
    }
    I->ncta = ncta;
    HHG_CUDA_TRY(cudaMalloc(&I->d_cta_plane, sizeof(int) * cta_plane.size()));
    HHG_CUDA_TRY(cudaMalloc(&I->d_cta_start, sizeof(int) * cta_start.size()));
    HHG_CUDA_TRY(cudaMalloc(&I->d_pstart, sizeof(int) * pstart.size()));
    HHG_CUDA_TRY(cudaMemcpy(I->d_cta_plane, cta_plane.data(), sizeof(int) * cta_plane.size(), cudaMemcpyHostToDevice));
    HHG_CUDA_TRY(cudaMemcpy(I->d_cta_start, cta_start.data(), sizeof(int) * cta_start.size(), cudaMemcpyHostToDevice));
    HHG_CUDA_TRY(cudaMemcpy(I->d_pstart, pstart.data(), sizeof(int) * pstart.size(), cudaMemcpyHostToDevice));
  }
  // marching-kernel tasks: every tile with owned points, sorted by its number of cubes (longest
  // first), with the k-chunk shortened until there are enough tasks to fill the GPU
  {
    const int64_t n = (int64_t)1 << lvl;
    const int iw = march_iw((int)n), jw = march_jw((int)n);
    const int h = jw == kMarchWarps ? 0 : 1;   // overlapping column / row of cubes below the tile
    int kch = 32;
    std::vector<std::pair<int64_t, int4>> tasks;
    for (;;) {
      tasks.clear();
      for (int64_t kc = 0; kc * kch <= n; ++kc)
        for (int64_t ty = 0; ty * jw + kc * kch <= n; ++ty)
          for (int64_t tx = 0; tx * iw + ty * jw + kc * kch <= n; ++tx) {
            int64_t work = 1;   // the top layer still writes carried points
            for (int64_t ck = std::max<int64_t>(kc * kch - 1, 0); ck <= kc * kch + kch - 1; ++ck)
              for (int64_t cj = std::max<int64_t>(ty * jw - h, 0); cj <= ty * jw + jw - 1; ++cj) {
                const int64_t hi = std::min<int64_t>(tx * iw + iw - 1, n - 1 - cj - ck), lo = std::max<int64_t>(tx * iw - h, 0);
                if (hi >= lo) work += hi - lo + 1;
              }
            tasks.push_back({work, int4{(int)tx, (int)ty, (int)kc, 0}});
          }
      if (kch <= 4 || (int64_t)tasks.size() * nmacro() >= 4 * 152) break;
      kch /= 2;
    }
    std::vector<std::pair<int64_t, int4>> all;
    for (int mac = 0; mac < nmacro(); ++mac)
      for (auto& t : tasks) all.push_back({t.first, int4{t.second.x, t.second.y, t.second.z, mac}});
    std::stable_sort(all.begin(), all.end(), [](const std::pair<int64_t, int4>& a, const std::pair<int64_t, int4>& b) {
      return a.first > b.first;
    });
    std::vector<int4> tv(all.size());
    for (size_t t = 0; t < all.size(); ++t) tv[t] = all[t].second;
    I->march_kchunk = kch;
    I->n_march_tasks = (int64_t)tv.size();
    HHG_CUDA_TRY(cudaMalloc(&I->d_march_tasks, sizeof(int4) * tv.size()));
    HHG_CUDA_TRY(cudaMemcpy(I->d_march_tasks, tv.data(), sizeof(int4) * tv.size(), cudaMemcpyHostToDevice));
  }
  // plane-tile kernel tasks: (i-chunk, row group, k-chunk), sorted by their number of points
  // the per-macro list of the two-plane FP32 P2 kernel: longer k-chunks (its 8-plane prologue is paid
  // once per task) for about 4 tasks per SM; the others about 8 per SM
  HHG_TRY(build_tile_tasks(N, 128, kStencilWarps, 1, 4 * 152, &I->tile[0]));
  HHG_TRY(build_tile_tasks(N, 64, kStencilWarps, nmacro(), 8 * 152, &I->tile[1]));
  HHG_TRY(build_tile_tasks(N, 64, kStencilWarps, 1, 4 * 152, &I->tile[2]));
  I->h_ptr = ptr;
  I->h_idx = idx;
  I->h_bnd = bnd;
  if (I->ngroups > 0) {
    HHG_CUDA_TRY(cudaMalloc(&I->d_ptr, sizeof(int64_t) * ptr.size()));
    HHG_CUDA_TRY(cudaMalloc(&I->d_idx, sizeof(int64_t) * idx.size()));
    HHG_CUDA_TRY(cudaMalloc(&I->d_bnd, bnd.size()));
    HHG_CUDA_TRY(cudaMemcpy(I->d_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice));
    HHG_CUDA_TRY(cudaMemcpy(I->d_idx, idx.data(), sizeof(int64_t) * idx.size(), cudaMemcpyHostToDevice));
    HHG_CUDA_TRY(cudaMemcpy(I->d_bnd, bnd.data(), bnd.size(), cudaMemcpyHostToDevice));
    HHG_CUDA_TRY(cudaMalloc(&I->d_sign, sgn.size()));
    HHG_CUDA_TRY(cudaMemcpy(I->d_sign, sgn.data(), sgn.size(), cudaMemcpyHostToDevice));
  }
  *out = I.get();
  iface[key] = std::move(I);
  return HHG_OK;
}

extern "C" int hhg_vec_size(const hhg_mesh_t* mesh, int level, int degree, int64_t* n) {
  clear_error();
  if (!mesh || !n) return fail(HHG_E_ARG, "vec_size: null pointer");
  if (level < 0 || level > mesh->level) return fail(HHG_E_ARG, "vec_size: level %d outside 0..%d", level, mesh->level);
  if (degree != 1 && degree != 2) return fail(HHG_E_ARG, "vec_size: degree must be 1 or 2");
  *n = (int64_t)mesh->nmacro() * lattice_size((int64_t)degree << level);
  return HHG_OK;
}

extern "C" int hhg_dof_count(const hhg_mesh_t* mesh, int level, int degree, int64_t* total, int64_t* interior) {
  clear_error();
  if (!mesh || !total || !interior) return fail(HHG_E_ARG, "dof_count: null pointer");
  const Interface* I = nullptr;
  HHG_TRY(const_cast<hhg_mesh_t*>(mesh)->interface(level, degree, &I));
  *total = I->ndof_total;
  *interior = I->ndof_interior;
  return HHG_OK;
}
