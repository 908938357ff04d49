// Host side of dgsl: mesh ingest and connectivity (Sec. 2.1), orders, the
// reference operators of Sec. 2.4 and the FP64 per-edge blocks.
//
// Connectivity reading (Sec. 2.1 assigns left/right "randomly"): local edge k
// of triangle t joins (v_k, v_{k+1 mod 3}); edges are numbered by first
// encounter (triangles by id, k = 0,1,2); the first triangle to meet an edge
// is its left triangle l(j), the second its right r(j); (X1, X2) follow l's
// counter-clockwise order, so n_j points from l to r.
//
// Orders (not in the paper): reverse Cuthill-McKee over the triangle graph
// from triangle 0 (neighbours by increasing (degree, id)); greedy edge
// colouring over edges sorted by (min rank, max rank, id), the smallest
// colour unused by the edges of l(j) and r(j); internal edge order by
// (colour, min rank, max rank, id).
//
// Blocks: the gradient blocks of eq. ad5.2 from the reference-operator form
// of Sec. 2.4,
//   Q_ij = A_ij J_i . Q^{V,a,b} - |G_j| n_j sigma_ij Q^{L,a,b},  A_ij = A_i / 3,
// and the dual mass matrix of eq. MassMatrixD,
//   Mhat_j = A_lj M^L + A_rj M^R,
// inverted per edge by Cholesky.
#include "host.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <exception>
#include <mutex>
#include <numeric>
#include <set>
#include <thread>
#include <unordered_map>

namespace dgsl {
namespace {

template <class F>
void parallel_for(int64_t n, F&& f) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
  if (n < 4096 || nt == 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next{0};
  std::atomic<bool> failed{false};
  std::exception_ptr err;
  std::mutex err_mu;
  const int64_t chunk = 256;
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&] {
      try {
        for (;;) {
          if (failed.load()) break;
          int64_t s = next.fetch_add(chunk);
          if (s >= n) break;
          int64_t e = std::min(n, s + chunk);
          for (int64_t i = s; i < e; ++i) f(i);
        }
      } catch (...) {
        std::lock_guard<std::mutex> lk(err_mu);
        if (!err) err = std::current_exception();
        failed.store(true);
      }
    });
  for (auto& x : th) x.join();
  if (err) std::rethrow_exception(err);
}

// ---------------------------------------------------------------- basis

std::vector<std::pair<int, int>> node_ab(int p) {
  std::vector<std::pair<int, int>> out;
  for (int b = 0; b <= p; ++b)
    for (int a = 0; a <= p - b; ++a) out.push_back({a, b});
  return out;
}

std::vector<std::pair<int, int>> monomials(int p) {
  std::vector<std::pair<int, int>> out;
  for (int i = 0; i <= p; ++i)
    for (int j = 0; j <= p - i; ++j) out.push_back({i, j});
  return out;
}

// Inverse of a dense n x n matrix by Gauss-Jordan elimination with partial
// pivoting (row-major, in place into inv).
void invert(int n, std::vector<double> a, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
    if (a[(size_t)piv * n + c] == 0.0) throw Error(DGSL_EINVAL, "singular Vandermonde matrix");
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)c * n + k], a[(size_t)piv * n + k]);
        std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
      }
    double d = a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      a[(size_t)c * n + k] /= d;
      inv[(size_t)c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
}

struct Basis {
  int p, n;
  std::vector<std::pair<int, int>> mono;
  std::vector<double> C;  // C[m][k]: coefficient of monomial m in phi_k
  explicit Basis(int p_) : p(p_) {
    auto ab = node_ab(p);
    mono = monomials(p);
    n = (int)ab.size();
    std::vector<double> V((size_t)n * n);
    for (int r = 0; r < n; ++r) {
      double x = (double)ab[r].first / p, y = (double)ab[r].second / p;
      for (int m = 0; m < n; ++m) V[(size_t)r * n + m] = std::pow(x, mono[m].first) * std::pow(y, mono[m].second);
    }
    invert(n, V, C);
  }
  void eval(double x, double y, double* phi) const {
    for (int k = 0; k < n; ++k) phi[k] = 0.0;
    for (int m = 0; m < n; ++m) {
      double v = std::pow(x, mono[m].first) * std::pow(y, mono[m].second);
      for (int k = 0; k < n; ++k) phi[k] += C[(size_t)m * n + k] * v;
    }
  }
  void grad(double x, double y, double* gx, double* gy) const {
    for (int k = 0; k < n; ++k) gx[k] = gy[k] = 0.0;
    for (int m = 0; m < n; ++m) {
      int i = mono[m].first, j = mono[m].second;
      double dx = i > 0 ? i * std::pow(x, i - 1) * std::pow(y, j) : 0.0;
      double dy = j > 0 ? j * std::pow(x, i) * std::pow(y, j - 1) : 0.0;
      for (int k = 0; k < n; ++k) {
        gx[k] += C[(size_t)m * n + k] * dx;
        gy[k] += C[(size_t)m * n + k] * dy;
      }
    }
  }
};

// Gauss-Legendre rule on [0,1] by Newton iteration on P_n.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Collapsed-coordinate product rule on T_ref (exact to degree 2n-2).
void triangle_rule(int n, std::vector<double>& qx, std::vector<double>& qy, std::vector<double>& qw) {
  std::vector<double> t, w;
  gauss_legendre01(n, t, w);
  qx.clear();
  qy.clear();
  qw.clear();
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      qx.push_back(t[a]);
      qy.push_back(t[b] * (1.0 - t[a]));
      qw.push_back(w[a] * w[b] * (1.0 - t[a]));
    }
}

inline double min_image(double d, double P) { return d - P * std::nearbyint(d / P); }

}  // namespace

// ---------------------------------------------------------------- reference operators

RefOps build_reference_operators(int p) {
  if (p < 1 || p > 4) throw Error(DGSL_EINVAL, "degree p must be in 1..4");
  RefOps ro;
  ro.p = p;
  ro.nphi = n_phi_of(p);
  ro.npsi = n_psi_of(p);
  const int n = ro.nphi;
  Basis B(p);
  auto ab = node_ab(p);
  // dual index maps by node coincidence: the right half's local node (a, b)
  // sits at 1 - (a/p, b/p), which for a + b = p is the left node (b, a)
  ro.Lmap.resize(n);
  ro.Rmap.resize(n);
  int next = n;
  for (int m = 0; m < n; ++m) ro.Lmap[m] = m;
  for (int m = 0; m < n; ++m) {
    int a = ab[m].first, b = ab[m].second;
    if (a + b < p) {
      ro.Rmap[m] = next++;
    } else {
      int q = -1;
      for (int u = 0; u < n; ++u)
        if (ab[u].first == b && ab[u].second == a) q = u;
      ro.Rmap[m] = ro.Lmap[q];
    }
  }
  std::vector<double> qx, qy, qw, t, wt;
  triangle_rule(p + 2, qx, qy, qw);
  gauss_legendre01(p + 2, t, wt);
  const int nq = (int)qw.size();
  std::vector<double> phi(n), phk(n), gx(n), gy(n);
  ro.Mref.assign((size_t)n * n, 0.0);
  for (int q = 0; q < nq; ++q) {
    B.eval(qx[q], qy[q], phi.data());
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l) ro.Mref[(size_t)k * n + l] += qw[q] * phi[k] * phi[l];
  }
  const double nu[3][2] = {{0, 0}, {1, 0}, {0, 1}};
  const double bref[2] = {1.0 / 3.0, 1.0 / 3.0};
  ro.V.assign((size_t)3 * n * n * 2, 0.0);
  ro.Line.assign((size_t)3 * n * n, 0.0);
  ro.U.assign((size_t)3 * n * n, 0.0);
  for (int a = 0; a < 3; ++a) {
    const double* va = nu[a];
    const double* vb = nu[(a + 1) % 3];
    for (int q = 0; q < nq; ++q) {
      // xi = T_a^{-1}(z): b_ref -> (0,0), nu_a -> (1,0), nu_{a+1} -> (0,1)
      double xi = bref[0] + qx[q] * (va[0] - bref[0]) + qy[q] * (vb[0] - bref[0]);
      double eta = bref[1] + qx[q] * (va[1] - bref[1]) + qy[q] * (vb[1] - bref[1]);
      B.eval(qx[q], qy[q], phi.data());   // phi_m(z): dual half basis
      B.eval(xi, eta, phk.data());        // phi_k(T_a^{-1} z)
      B.grad(xi, eta, gx.data(), gy.data());
      for (int k = 0; k < n; ++k)
        for (int m = 0; m < n; ++m) {
          size_t o = (((size_t)a * n + k) * n + m) * 2;
          ro.V[o + 0] += qw[q] * gx[k] * phi[m];
          ro.V[o + 1] += qw[q] * gy[k] * phi[m];
          ro.U[((size_t)a * n + m) * n + k] += qw[q] * phi[m] * phk[k];
        }
    }
    for (size_t q = 0; q < t.size(); ++q) {
      double ex = va[0] + t[q] * (vb[0] - va[0]);
      double ey = va[1] + t[q] * (vb[1] - va[1]);
      B.eval(ex, ey, phk.data());
      B.eval(1.0 - t[q], t[q], phi.data());
      for (int k = 0; k < n; ++k)
        for (int m = 0; m < n; ++m) ro.Line[((size_t)a * n + k) * n + m] += wt[q] * phk[k] * phi[m];
    }
  }
  return ro;
}

// ---------------------------------------------------------------- mesh

HostMesh build_mesh(const dgsl_mesh& m) {
  if (!m.xy || !m.tri || m.n_vertices <= 0 || m.n_triangles <= 0)
    throw Error(DGSL_EINVAL, "mesh arrays must be non-empty");
  if (!(m.period[0] > 0.0) || !(m.period[1] > 0.0)) throw Error(DGSL_EINVAL, "periods must be positive");
  HostMesh hm;
  hm.nv = m.n_vertices;
  hm.ne = m.n_triangles;
  hm.period[0] = m.period[0];
  hm.period[1] = m.period[1];
  const int ne = hm.ne;
  const double Px = m.period[0], Py = m.period[1];
  hm.txy.resize((size_t)ne * 6);
  hm.tri_v.assign(m.tri, m.tri + 3 * (size_t)ne);
  for (int t = 0; t < ne; ++t) {
    int v[3];
    for (int k = 0; k < 3; ++k) {
      v[k] = m.tri[3 * (size_t)t + k];
      if (v[k] < 0 || v[k] >= m.n_vertices) throw Error(DGSL_EMESH, "vertex index out of range");
    }
    double x0 = m.xy[2 * (size_t)v[0]], y0 = m.xy[2 * (size_t)v[0] + 1];
    double* o = &hm.txy[(size_t)t * 6];
    o[0] = x0;
    o[1] = y0;
    for (int k = 1; k < 3; ++k) {
      o[2 * k] = x0 + min_image(m.xy[2 * (size_t)v[k]] - x0, Px);
      o[2 * k + 1] = y0 + min_image(m.xy[2 * (size_t)v[k] + 1] - y0, Py);
    }
    double e1x = o[2] - o[0], e1y = o[3] - o[1], e2x = o[4] - o[0], e2y = o[5] - o[1];
    double a2 = e1x * e2y - e1y * e2x;
    if (!(a2 > 0.0)) throw Error(DGSL_EMESH, "triangle with non-positive area (not CCW or degenerate)");
  }
  std::unordered_map<uint64_t, int32_t> key_to_edge;
  key_to_edge.reserve((size_t)ne * 2);
  hm.tri_edge.assign((size_t)ne * 3, -1);
  for (int t = 0; t < ne; ++t)
    for (int k = 0; k < 3; ++k) {
      int32_t a = m.tri[3 * (size_t)t + k], b = m.tri[3 * (size_t)t + (k + 1) % 3];
      if (a == b) throw Error(DGSL_EMESH, "degenerate edge");
      uint64_t key = a < b ? ((uint64_t)a << 32 | (uint32_t)b) : ((uint64_t)b << 32 | (uint32_t)a);
      auto it = key_to_edge.find(key);
      int32_t j;
      if (it == key_to_edge.end()) {
        j = (int32_t)(hm.lr.size() / 2);
        key_to_edge.emplace(key, j);
        hm.edge_vtx.push_back(a);
        hm.edge_vtx.push_back(b);
        hm.lr.push_back(t);
        hm.lr.push_back(-1);
        hm.loc.push_back((uint8_t)k);
        hm.loc.push_back(0xFF);
      } else {
        j = it->second;
        if (hm.lr[2 * (size_t)j + 1] != -1) throw Error(DGSL_EMESH, "edge shared by more than two triangles");
        if (hm.edge_vtx[2 * (size_t)j] != b || hm.edge_vtx[2 * (size_t)j + 1] != a)
          throw Error(DGSL_EMESH, "inconsistent orientation across an edge");
        if (hm.lr[2 * (size_t)j] == t) throw Error(DGSL_EMESH, "triangle meets the same edge twice");
        hm.lr[2 * (size_t)j + 1] = t;
        hm.loc[2 * (size_t)j + 1] = (uint8_t)k;
      }
      hm.tri_edge[(size_t)t * 3 + k] = j;
    }
  hm.nd = (int)(hm.lr.size() / 2);
  const int nd = hm.nd;
  for (int j = 0; j < nd; ++j)
    if (hm.lr[2 * (size_t)j + 1] < 0) throw Error(DGSL_EMESH, "boundary edge: only periodic (closed) meshes are supported");
  hm.shift.resize((size_t)nd * 2);
  for (int j = 0; j < nd; ++j) {
    int l = hm.lr[2 * j], r = hm.lr[2 * j + 1];
    int al = hm.loc[2 * j], ar = hm.loc[2 * j + 1];
    const double* Pl = &hm.txy[(size_t)l * 6];
    const double* Pr = &hm.txy[(size_t)r * 6];
    const double* x1l = Pl + 2 * al;
    const double* x1r = Pr + 2 * ((ar + 1) % 3);
    const double* x2l = Pl + 2 * ((al + 1) % 3);
    const double* x2r = Pr + 2 * ar;
    double sx = std::nearbyint((x1l[0] - x1r[0]) / Px);
    double sy = std::nearbyint((x1l[1] - x1r[1]) / Py);
    hm.shift[2 * (size_t)j] = (int8_t)sx;
    hm.shift[2 * (size_t)j + 1] = (int8_t)sy;
    if (std::fabs(x2l[0] - (x2r[0] + sx * Px)) > 1e-9 || std::fabs(x2l[1] - (x2r[1] + sy * Py)) > 1e-9)
      throw Error(DGSL_EMESH, "edge endpoints disagree across the periodic boundary");
  }
  // neighbours; reject triangle pairs that share two edges
  std::vector<int32_t> nb((size_t)ne * 3);
  for (int t = 0; t < ne; ++t)
    for (int k = 0; k < 3; ++k) {
      int j = hm.tri_edge[(size_t)t * 3 + k];
      nb[(size_t)t * 3 + k] = hm.lr[2 * j] == t ? hm.lr[2 * j + 1] : hm.lr[2 * j];
    }
  for (int t = 0; t < ne; ++t) {
    int a = nb[3 * t], b = nb[3 * t + 1], c = nb[3 * t + 2];
    if (a == b || b == c || a == c) throw Error(DGSL_EMESH, "two triangles share more than one edge (mesh too coarse)");
  }
  // reverse Cuthill-McKee
  std::vector<int> deg(ne);
  for (int t = 0; t < ne; ++t) {
    std::set<int> s(&nb[3 * (size_t)t], &nb[3 * (size_t)t] + 3);
    deg[t] = (int)s.size();
  }
  std::vector<char> seen(ne, 0);
  std::vector<int32_t> order;
  order.reserve(ne);
  for (int start = 0; start < ne; ++start) {
    if (seen[start]) continue;
    seen[start] = 1;
    std::deque<int> q{start};
    while (!q.empty()) {
      int t = q.front();
      q.pop_front();
      order.push_back(t);
      std::vector<int> cand;
      for (int k = 0; k < 3; ++k) {
        int u = nb[3 * (size_t)t + k];
        if (!seen[u] && std::find(cand.begin(), cand.end(), u) == cand.end()) cand.push_back(u);
      }
      std::sort(cand.begin(), cand.end(), [&](int x, int y) { return deg[x] != deg[y] ? deg[x] < deg[y] : x < y; });
      for (int u : cand) {
        seen[u] = 1;
        q.push_back(u);
      }
    }
  }
  std::reverse(order.begin(), order.end());
  hm.perm = order;
  hm.rank.resize(ne);
  for (int i = 0; i < ne; ++i) hm.rank[hm.perm[i]] = i;
  // greedy edge colouring
  std::vector<int64_t> lo(nd), hi(nd);
  for (int j = 0; j < nd; ++j) {
    int64_t a = hm.rank[hm.lr[2 * j]], b = hm.rank[hm.lr[2 * j + 1]];
    lo[j] = std::min(a, b);
    hi[j] = std::max(a, b);
  }
  std::vector<int32_t> visit(nd);
  std::iota(visit.begin(), visit.end(), 0);
  std::sort(visit.begin(), visit.end(), [&](int x, int y) {
    if (lo[x] != lo[y]) return lo[x] < lo[y];
    if (hi[x] != hi[y]) return hi[x] < hi[y];
    return x < y;
  });
  std::vector<int> col(nd, -1);
  int ncol = 0;
  for (int j : visit) {
    unsigned used = 0;
    for (int s = 0; s < 2; ++s) {
      int t = hm.lr[2 * j + s];
      for (int k = 0; k < 3; ++k) {
        int e = hm.tri_edge[3 * (size_t)t + k];
        if (e != j && col[e] >= 0) used |= 1u << col[e];
      }
    }
    int c = 0;
    while (used & (1u << c)) ++c;
    col[j] = c;
    ncol = std::max(ncol, c + 1);
  }
  hm.colour.resize(nd);
  for (int j = 0; j < nd; ++j) hm.colour[j] = (uint8_t)col[j];
  hm.edge_perm.resize(nd);
  std::iota(hm.edge_perm.begin(), hm.edge_perm.end(), 0);
  std::sort(hm.edge_perm.begin(), hm.edge_perm.end(), [&](int x, int y) {
    if (col[x] != col[y]) return col[x] < col[y];
    if (lo[x] != lo[y]) return lo[x] < lo[y];
    if (hi[x] != hi[y]) return hi[x] < hi[y];
    return x < y;
  });
  hm.edge_rank.resize(nd);
  for (int e = 0; e < nd; ++e) hm.edge_rank[hm.edge_perm[e]] = e;
  hm.colour_offsets.assign(ncol + 1, 0);
  for (int j = 0; j < nd; ++j) hm.colour_offsets[col[j] + 1]++;
  for (int c = 0; c < ncol; ++c) hm.colour_offsets[c + 1] += hm.colour_offsets[c];
  return hm;
}

// ---------------------------------------------------------------- blocks

namespace {
// Cholesky inverse of a symmetric positive definite n x n matrix.
void spd_inverse(int n, const double* A, double* out) {
  std::vector<double> L((size_t)n * n, 0.0), Li((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      if (i == j) {
        if (!(s > 0.0)) throw Error(DGSL_EMESH, "dual mass matrix not positive definite");
        L[(size_t)i * n + i] = std::sqrt(s);
      } else {
        L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
      }
    }
  for (int c = 0; c < n; ++c)  // forward solve L Li = I
    for (int i = 0; i < n; ++i) {
      double s = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * Li[(size_t)k * n + c];
      Li[(size_t)i * n + c] = s / L[(size_t)i * n + i];
    }
  for (int i = 0; i < n; ++i)  // A^{-1} = Li^T Li
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = std::max(i, j); k < n; ++k) s += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
      out[(size_t)i * n + j] = s;
    }
}
}  // namespace

HostBlocks build_blocks(const HostMesh& hm, const RefOps& ro) {
  HostBlocks hb;
  const int n = ro.nphi, np = ro.npsi, ne = hm.ne, nd = hm.nd;
  hb.p = ro.p;
  hb.nphi = n;
  hb.npsi = np;
  hb.ne = ne;
  hb.nd = nd;
  hb.area.resize(ne);
  for (int i = 0; i < ne; ++i) {
    const double* P = &hm.txy[(size_t)hm.perm[i] * 6];
    hb.area[i] = (P[2] - P[0]) * (P[5] - P[1]) - (P[3] - P[1]) * (P[4] - P[0]);
  }
  hb.G.assign((size_t)nd * 4 * n * n, 0.0);
  hb.Minv.assign((size_t)nd * np * np, 0.0);
  hb.Kd.assign((size_t)ne * n * n, 0.0);
  hb.Ko.assign((size_t)ne * 3 * n * n, 0.0);
  hb.nbr.assign((size_t)ne * 3, -1);
  hb.elr.resize((size_t)nd * 2);
  hb.eloc.resize((size_t)nd * 2);
  hb.Uloc.assign((size_t)nd * 2 * n * n, 0.0);
  // edges of one colour share no triangle, so a colour is processed in parallel
  for (int c = 0; c < hm.n_colours(); ++c) {
    int e0 = hm.colour_offsets[c], e1 = hm.colour_offsets[c + 1];
    parallel_for(e1 - e0, [&](int64_t off) {
      const int e = e0 + (int)off;
      const int j = hm.edge_perm[e];
      int tri[2] = {hm.lr[2 * j], hm.lr[2 * j + 1]};
      int al = hm.loc[2 * j], ar = hm.loc[2 * j + 1];
      int alpha[2] = {al, ar};
      const double* Pl = &hm.txy[(size_t)tri[0] * 6];
      double X1[2] = {Pl[2 * al], Pl[2 * al + 1]};
      double X2[2] = {Pl[2 * ((al + 1) % 3)], Pl[2 * ((al + 1) % 3) + 1]};
      double dx = X2[0] - X1[0], dy = X2[1] - X1[1];
      double glen = std::hypot(dx, dy);
      double nrm[2] = {dy / glen, -dx / glen};
      double A[2];
      double* Ge = &hb.G[(size_t)e * 4 * n * n];
      for (int s = 0; s < 2; ++s) {
        const double* P = &hm.txy[(size_t)tri[s] * 6];
        double a = P[2] - P[0], b = P[4] - P[0], cc = P[3] - P[1], d = P[5] - P[1];
        double Ai = a * d - b * cc;
        A[s] = Ai;
        // (A_i/3) J(T_i)[dd][comp] with J(T_i) = J(T_i^{-1})^{-1}
        double AJ[2][2] = {{d / 3.0, -b / 3.0}, {-cc / 3.0, a / 3.0}};
        double sg = s == 0 ? 1.0 : -1.0;  // sigma_ij
        const int aa = alpha[s];
        for (int comp = 0; comp < 2; ++comp)
          for (int m = 0; m < n; ++m)
            for (int k = 0; k < n; ++k) {
              size_t vo = (((size_t)aa * n + k) * n + m) * 2;
              double vol = AJ[0][comp] * ro.V[vo] + AJ[1][comp] * ro.V[vo + 1];
              double line = ro.Line[((size_t)aa * n + k) * n + m];
              Ge[(((size_t)s * 2 + comp) * n + m) * n + k] = vol - sg * glen * nrm[comp] * line;
            }
        for (int m = 0; m < n; ++m)
          for (int k = 0; k < n; ++k)
            hb.Uloc[(((size_t)e * 2 + s) * n + m) * n + k] = (Ai / 3.0) * ro.U[((size_t)aa * n + m) * n + k];
      }
      // Mhat_j = A_lj M^L + A_rj M^R, A_ij = A_i/3 (eq. MassMatrixD)
      std::vector<double> Mh((size_t)np * np, 0.0);
      for (int s = 0; s < 2; ++s) {
        const std::vector<int>& map = s == 0 ? ro.Lmap : ro.Rmap;
        for (int m = 0; m < n; ++m)
          for (int q = 0; q < n; ++q) Mh[(size_t)map[m] * np + map[q]] += (A[s] / 3.0) * ro.Mref[(size_t)m * n + q];
      }
      double* Mi = &hb.Minv[(size_t)e * np * np];
      spd_inverse(np, Mh.data(), Mi);
      // couplings K_ab = sum_comp G_a^T Mhat^{-1} G_b
      std::vector<double> W((size_t)2 * 2 * np * n, 0.0);  // [side][comp][npsi][nphi]
      for (int s = 0; s < 2; ++s) {
        const std::vector<int>& map = s == 0 ? ro.Lmap : ro.Rmap;
        for (int comp = 0; comp < 2; ++comp)
          for (int r = 0; r < np; ++r)
            for (int k = 0; k < n; ++k) {
              double acc = 0.0;
              for (int m = 0; m < n; ++m)
                acc += Mi[(size_t)r * np + map[m]] * Ge[(((size_t)s * 2 + comp) * n + m) * n + k];
              W[(((size_t)s * 2 + comp) * np + r) * n + k] = acc;
            }
      }
      int ti[2] = {hm.rank[tri[0]], hm.rank[tri[1]]};
      for (int s = 0; s < 2; ++s) {
        hb.elr[2 * (size_t)e + s] = ti[s];
        hb.eloc[2 * (size_t)e + s] = (uint8_t)alpha[s];
      }
      for (int sa = 0; sa < 2; ++sa) {
        const std::vector<int>& mapa = sa == 0 ? ro.Lmap : ro.Rmap;
        for (int sb = 0; sb < 2; ++sb) {
          double* dst = sa == sb ? &hb.Kd[(size_t)ti[sa] * n * n]
                                 : &hb.Ko[((size_t)ti[sa] * 3 + alpha[sa]) * n * n];
          for (int k = 0; k < n; ++k)
            for (int l = 0; l < n; ++l) {
              double acc = 0.0;
              for (int comp = 0; comp < 2; ++comp)
                for (int m = 0; m < n; ++m)
                  acc += Ge[(((size_t)sa * 2 + comp) * n + m) * n + k] *
                         W[(((size_t)sb * 2 + comp) * np + mapa[m]) * n + l];
              dst[(size_t)k * n + l] += acc;
            }
        }
        hb.nbr[(size_t)ti[sa] * 3 + alpha[sa]] = ti[1 - sa];
      }
    });
  }
  // S = G^T Mhat^-1 G is symmetric (eq. pressure_final), but the two sides of
  // an edge compute their transposed blocks with different rounding.  The
  // stored couplings are made exactly symmetric (each pair of transposed
  // entries replaced by its mean), as CG assumes: with the difference form's
  // zero row sums the column sums then vanish too, and the FP32 / BF16 copies
  // rounded from these values are symmetric as well.
  parallel_for(nd, [&](int64_t e) {
    double* A = &hb.Ko[((size_t)hb.elr[2 * e] * 3 + hb.eloc[2 * e]) * n * n];
    double* B = &hb.Ko[((size_t)hb.elr[2 * e + 1] * 3 + hb.eloc[2 * e + 1]) * n * n];
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l) {
        const double v = 0.5 * (A[(size_t)k * n + l] + B[(size_t)l * n + k]);
        A[(size_t)k * n + l] = v;
        B[(size_t)l * n + k] = v;
      }
  });
  parallel_for(ne, [&](int64_t i) {
    double* D = &hb.Kd[(size_t)i * n * n];
    for (int k = 0; k < n; ++k)
      for (int l = k + 1; l < n; ++l) {
        const double v = 0.5 * (D[(size_t)k * n + l] + D[(size_t)l * n + k]);
        D[(size_t)k * n + l] = v;
        D[(size_t)l * n + k] = v;
      }
  });
  return hb;
}

std::vector<double> mref_inverse(const RefOps& ro) {
  std::vector<double> inv;
  invert(ro.nphi, ro.Mref, inv);
  return inv;
}

void sl_rule(int p, std::vector<double>& pts, std::vector<double>& w) {
  std::vector<double> qx, qy;
  triangle_rule(p + 1, qx, qy, w);
  pts.resize(2 * qx.size());
  for (size_t g = 0; g < qx.size(); ++g) {
    pts[2 * g] = qx[g];
    pts[2 * g + 1] = qy[g];
  }
}

SLHost build_sl_host(const HostMesh& hm, const RefOps& ro) {
  SLHost s;
  s.p = ro.p;
  s.nphi = ro.nphi;
  const int ne = hm.ne, n = ro.nphi;
  const double Px = hm.period[0], Py = hm.period[1];
  s.tri.assign((size_t)ne * 16, 0.0);
  s.nbr.assign((size_t)ne * 4, 0);
  for (int ti = 0; ti < ne; ++ti) {
    const int t = hm.perm[ti];
    const double* P = &hm.txy[(size_t)t * 6];
    double* o = &s.tri[(size_t)ti * 16];
    const double e1x = P[2] - P[0], e1y = P[3] - P[1], e2x = P[4] - P[0], e2y = P[5] - P[1];
    const double det = e1x * e2y - e1y * e2x;
    o[0] = P[0];
    o[1] = P[1];
    o[2] = e1x;
    o[3] = e1y;
    o[4] = e2x;
    o[5] = e2y;
    o[6] = e2y / det;   // xi  = j00 dx + j01 dy
    o[7] = -e2x / det;
    o[8] = -e1y / det;  // eta = j10 dx + j11 dy
    o[9] = e1x / det;
    for (int k = 0; k < 3; ++k) {
      const int j = hm.tri_edge[(size_t)t * 3 + k];
      const int l = hm.lr[2 * j], r = hm.lr[2 * j + 1];
      // shift: periods to add to r's frame to reach l's
      const double sx = hm.shift[2 * (size_t)j] * Px, sy = hm.shift[2 * (size_t)j + 1] * Py;
      const bool is_l = l == t;
      o[10 + 2 * k] = is_l ? -sx : sx;
      o[11 + 2 * k] = is_l ? -sy : sy;
      s.nbr[(size_t)ti * 4 + k] = hm.rank[is_l ? r : l];
      // local index of the same edge in that neighbour, 2 bits per edge
      s.nbr[(size_t)ti * 4 + 3] |= (int32_t)hm.loc[2 * (size_t)j + (is_l ? 1 : 0)] << (2 * k);
    }
  }
  Basis b(ro.p);
  s.mono_c = b.C;
  std::vector<double> qx, qy, qw;
  triangle_rule(ro.p + 1, qx, qy, qw);
  s.ng = (int)qw.size();
  s.pts.resize((size_t)s.ng * 2);
  s.w = qw;
  std::vector<double> Minv;
  invert(n, ro.Mref, Minv);
  s.q.assign((size_t)n * s.ng, 0.0);
  std::vector<double> phi(n);
  for (int g = 0; g < s.ng; ++g) {
    s.pts[2 * g] = qx[g];
    s.pts[2 * g + 1] = qy[g];
    b.eval(qx[g], qy[g], phi.data());
    for (int k = 0; k < n; ++k) {
      double a = 0.0;
      for (int l = 0; l < n; ++l) a += Minv[(size_t)k * n + l] * phi[l];
      s.q[(size_t)k * s.ng + g] = a * qw[g];
    }
  }
  return s;
}

void node_coords(const HostMesh& hm, const RefOps& ro, int grid, double* out) {
  const int p = ro.p, n = ro.nphi;
  auto ab = node_ab(p);
  if (grid == DGSL_MAIN) {
    for (int i = 0; i < hm.ne; ++i) {
      const double* P = &hm.txy[(size_t)hm.perm[i] * 6];
      for (int k = 0; k < n; ++k) {
        double xi = (double)ab[k].first / p, eta = (double)ab[k].second / p;
        double* o = out + ((size_t)i * n + k) * 2;
        o[0] = P[0] + xi * (P[2] - P[0]) + eta * (P[4] - P[0]);
        o[1] = P[1] + xi * (P[3] - P[1]) + eta * (P[5] - P[1]);
      }
    }
    return;
  }
  const int np = ro.npsi;
  for (int e = 0; e < hm.nd; ++e) {
    int j = hm.edge_perm[e];
    int l = hm.lr[2 * j], r = hm.lr[2 * j + 1];
    int al = hm.loc[2 * j], ar = hm.loc[2 * j + 1];
    const double* Pl = &hm.txy[(size_t)l * 6];
    const double* Pr = &hm.txy[(size_t)r * 6];
    double bl[2] = {(Pl[0] + Pl[2] + Pl[4]) / 3.0, (Pl[1] + Pl[3] + Pl[5]) / 3.0};
    double br[2] = {(Pr[0] + Pr[2] + Pr[4]) / 3.0, (Pr[1] + Pr[3] + Pr[5]) / 3.0};
    const double* X1l = Pl + 2 * al;
    const double* X2l = Pl + 2 * ((al + 1) % 3);
    const double* X1r = Pr + 2 * ((ar + 1) % 3);
    const double* X2r = Pr + 2 * ar;
    double sh[2] = {hm.shift[2 * j] * hm.period[0], hm.shift[2 * j + 1] * hm.period[1]};
    for (int m = 0; m < n; ++m) {
      double xi = (double)ab[m].first / p, eta = (double)ab[m].second / p;
      double* o = out + ((size_t)e * np + ro.Lmap[m]) * 2;
      for (int d = 0; d < 2; ++d) o[d] = bl[d] + xi * (X1l[d] - bl[d]) + eta * (X2l[d] - bl[d]);
      if (ro.Rmap[m] >= n) {
        double* q = out + ((size_t)e * np + ro.Rmap[m]) * 2;
        for (int d = 0; d < 2; ++d) q[d] = br[d] + xi * (X2r[d] - br[d]) + eta * (X1r[d] - br[d]) + sh[d];
      }
    }
  }
}

}  // namespace dgsl
