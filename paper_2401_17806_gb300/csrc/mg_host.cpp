// Host setup of the two-level multigrid preconditioner: vertex numbering,
// coarse patterns, smoothed-aggregation levels and the dense coarsest solve
// (FP64; see mg_host.h for the method).
#include "mg_host.h"

#include <algorithm>
#include <cmath>

namespace dgsl {

namespace {

// Rows of sorted, unique column lists -> CSR pattern (values zero).
CsrD from_rows(std::vector<std::vector<int32_t>>& rows, int m) {
  CsrD a;
  a.n = (int)rows.size();
  a.m = m;
  a.rp.assign(a.n + 1, 0);
  for (int i = 0; i < a.n; ++i) {
    auto& r = rows[i];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    a.rp[i + 1] = a.rp[i] + (int32_t)r.size();
  }
  a.ci.resize(a.rp[a.n]);
  for (int i = 0; i < a.n; ++i) std::copy(rows[i].begin(), rows[i].end(), a.ci.begin() + a.rp[i]);
  a.v.assign(a.ci.size(), 0.0);
  return a;
}

// Greedy two-pass aggregation on a graph with sorted rows (see mg_host.h).
int aggregate(const CsrD& g, std::vector<int32_t>& agg) {
  const int n = g.n;
  agg.assign(n, -1);
  int na = 0;
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_nb = true;
    for (int k = g.rp[i]; k < g.rp[i + 1]; ++k)
      if (agg[g.ci[k]] >= 0) {
        free_nb = false;
        break;
      }
    if (!free_nb) continue;
    for (int k = g.rp[i]; k < g.rp[i + 1]; ++k) agg[g.ci[k]] = na;
    agg[i] = na;
    ++na;
  }
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    int a = -1;
    for (int k = g.rp[i]; k < g.rp[i + 1]; ++k)
      if (agg[g.ci[k]] >= 0) {
        a = agg[g.ci[k]];
        break;
      }
    agg[i] = a >= 0 ? a : na++;
  }
  return na;
}

CsrD transpose(const CsrD& a) {
  CsrD t;
  t.n = a.m;
  t.m = a.n;
  t.rp.assign(t.n + 1, 0);
  for (int32_t c : a.ci) ++t.rp[c + 1];
  for (int i = 0; i < t.n; ++i) t.rp[i + 1] += t.rp[i];
  t.ci.resize(a.ci.size());
  t.v.resize(a.v.size());
  std::vector<int32_t> pos(t.rp.begin(), t.rp.end() - 1);
  for (int i = 0; i < a.n; ++i)  // rows in order: the columns of t come out sorted
    for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
      const int32_t p = pos[a.ci[k]]++;
      t.ci[p] = i;
      t.v[p] = a.v[k];
    }
  return t;
}

// C = A B (Gustavson, structural: every column reached is kept, also when its
// sum is zero; columns sorted).
CsrD multiply(const CsrD& a, const CsrD& b) {
  CsrD c;
  c.n = a.n;
  c.m = b.m;
  c.rp.assign(c.n + 1, 0);
  std::vector<int32_t> mark(b.m, -1);
  std::vector<double> acc(b.m, 0.0);
  std::vector<int32_t> cols;
  for (int i = 0; i < a.n; ++i) {
    cols.clear();
    for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
      const int j = a.ci[k];
      const double av = a.v[k];
      for (int q = b.rp[j]; q < b.rp[j + 1]; ++q) {
        const int c2 = b.ci[q];
        if (mark[c2] != i) {
          mark[c2] = i;
          acc[c2] = 0.0;
          cols.push_back(c2);
        }
        acc[c2] += av * b.v[q];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t c2 : cols) {
      c.ci.push_back(c2);
      c.v.push_back(acc[c2]);
    }
    c.rp[i + 1] = (int32_t)c.ci.size();
  }
  return c;
}

double gershgorin(const CsrD& a) {
  double lam = 0.0;
  for (int i = 0; i < a.n; ++i) {
    double s = 0.0, d = 0.0;
    for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
      s += std::fabs(a.v[k]);
      if (a.ci[k] == i) d = a.v[k];
    }
    if (!(d > 0.0)) throw Error(DGSL_EINVAL, "multigrid: a coarse operator has a non-positive diagonal");
    lam = std::max(lam, s / d);
  }
  return lam;
}

double diag_of(const CsrD& a, int i) {
  const int64_t k = csr_find(a, i, i);
  return k >= 0 ? a.v[k] : 0.0;
}

// In-place Cholesky of the leading m x m block of the row-major n x n matrix.
void cholesky(std::vector<double>& a, int n, int m) {
  for (int j = 0; j < m; ++j) {
    double d = a[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
    if (!(d > 0.0)) throw Error(DGSL_EINVAL, "multigrid: the coarsest operator is not positive definite");
    const double l = std::sqrt(d);
    a[(size_t)j * n + j] = l;
    for (int r = j + 1; r < m; ++r) {
      double v = a[(size_t)r * n + j];
      for (int k = 0; k < j; ++k) v -= a[(size_t)r * n + k] * a[(size_t)j * n + k];
      a[(size_t)r * n + j] = v / l;
    }
  }
}

// Dense coarsest solve.  Regular: A^-1.  Singular (kernel span{1}): with
// E = [[0, 0], [0, A11^-1]] (DOF 0 grounded) the operator Pi E Pi, Pi the
// projection to mean zero: for a right-hand side of zero sum it is the
// pseudo-inverse (the mean-zero solution).
std::vector<double> coarsest_inverse(const CsrD& a, bool singular) {
  const int n = a.n;
  std::vector<double> d((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) d[(size_t)i * n + a.ci[k]] += 0.5 * a.v[k];
  for (int i = 0; i < n; ++i)  // symmetrised
    for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) d[(size_t)a.ci[k] * n + i] += 0.5 * a.v[k];
  const int off = singular ? 1 : 0;
  const int m = n - off;
  std::vector<double> s((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) s[(size_t)i * m + j] = d[(size_t)(i + off) * n + j + off];
  cholesky(s, m, m);
  std::vector<double> inv((size_t)n * n, 0.0), y(m);
  for (int c = 0; c < m; ++c) {  // column c of the inverse: L L^T y = e_c
    for (int i = 0; i < m; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= s[(size_t)i * m + k] * y[k];
      y[i] = v / s[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < m; ++k) v -= s[(size_t)k * m + i] * y[k];
      y[i] = v / s[(size_t)i * m + i];
    }
    for (int i = 0; i < m; ++i) inv[(size_t)(i + off) * n + c + off] = y[i];
  }
  if (!singular) return inv;
  // Pi inv Pi: subtract row means, then column means
  for (int i = 0; i < n; ++i) {
    double mu = 0.0;
    for (int j = 0; j < n; ++j) mu += inv[(size_t)i * n + j];
    mu /= n;
    for (int j = 0; j < n; ++j) inv[(size_t)i * n + j] -= mu;
  }
  for (int j = 0; j < n; ++j) {
    double mu = 0.0;
    for (int i = 0; i < n; ++i) mu += inv[(size_t)i * n + j];
    mu /= n;
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + j] -= mu;
  }
  return inv;
}

}  // namespace

int64_t csr_find(const CsrD& a, int i, int j) {
  const int32_t* b = a.ci.data() + a.rp[i];
  const int32_t* e = a.ci.data() + a.rp[i + 1];
  const int32_t* p = std::lower_bound(b, e, j);
  return (p != e && *p == j) ? (int64_t)(p - a.ci.data()) : -1;
}

void mg_vertex_numbering(const HostMesh& hm, MGHost& mg) {
  const int ne = hm.ne;
  std::vector<int32_t> id(hm.nv, -1);
  mg.cvid.assign((size_t)ne * 3, -1);
  int nv = 0;
  for (int t = 0; t < ne; ++t) {
    const int tn = hm.perm[t];
    for (int m = 0; m < 3; ++m) {
      const int v = hm.tri_v[(size_t)tn * 3 + m];
      if (id[v] < 0) id[v] = nv++;
      mg.cvid[(size_t)t * 3 + m] = id[v];
    }
  }
  mg.nv = nv;
  mg.v2t_ptr.assign(nv + 1, 0);
  for (int32_t v : mg.cvid) ++mg.v2t_ptr[v + 1];
  for (int v = 0; v < nv; ++v) mg.v2t_ptr[v + 1] += mg.v2t_ptr[v];
  mg.v2t.resize(mg.cvid.size());
  std::vector<int32_t> pos(mg.v2t_ptr.begin(), mg.v2t_ptr.end() - 1);
  for (int k = 0; k < 3 * ne; ++k) mg.v2t[pos[mg.cvid[k]]++] = k;  // (t, m) ascending
}

CsrD mg_coarse_pattern(const MGHost& mg, int ne, const std::vector<int32_t>& nbr) {
  std::vector<std::vector<int32_t>> rows(mg.nv);
  for (int t = 0; t < ne; ++t) {
    const int tt[4] = {t, nbr[(size_t)t * 3], nbr[(size_t)t * 3 + 1], nbr[(size_t)t * 3 + 2]};
    for (int a = 0; a < 3; ++a) {
      auto& r = rows[mg.cvid[(size_t)t * 3 + a]];
      for (int u = 0; u < 4; ++u)
        for (int b = 0; b < 3; ++b) r.push_back(mg.cvid[(size_t)tt[u] * 3 + b]);
    }
  }
  return from_rows(rows, mg.nv);
}

CsrD mg_vertex_graph(const MGHost& mg, int ne) {
  std::vector<std::vector<int32_t>> rows(mg.nv);
  for (int t = 0; t < ne; ++t)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) rows[mg.cvid[(size_t)t * 3 + a]].push_back(mg.cvid[(size_t)t * 3 + b]);
  return from_rows(rows, mg.nv);
}

void mg_build_levels(MGHost& mg, const CsrD& A0, const CsrD& G0, bool singular) {
  mg.lv.clear();
  mg.lv.emplace_back();
  mg.lv.back().A = A0;
  CsrD G = G0;
  while (mg.lv.back().A.n > kMGCoarsest) {
    MGLevelH& L = mg.lv.back();
    const int n = L.A.n;
    std::vector<int32_t> agg;
    const int na = aggregate(G, agg);
    if (na > 0.8 * n) break;
    // P = T - omega D^-1 A T on the pattern of T + A T
    const double omega = (4.0 / 3.0) / gershgorin(L.A);
    std::vector<std::vector<int32_t>> prow(n);
    for (int i = 0; i < n; ++i) {
      prow[i].push_back(agg[i]);
      for (int k = L.A.rp[i]; k < L.A.rp[i + 1]; ++k) prow[i].push_back(agg[L.A.ci[k]]);
    }
    CsrD P = from_rows(prow, na);
    for (int i = 0; i < n; ++i) {
      const double s = omega / diag_of(L.A, i);
      P.v[csr_find(P, i, agg[i])] += 1.0;
      for (int k = L.A.rp[i]; k < L.A.rp[i + 1]; ++k) P.v[csr_find(P, i, agg[L.A.ci[k]])] -= s * L.A.v[k];
    }
    CsrD R = transpose(P);
    CsrD An = multiply(R, multiply(L.A, P));
    // aggregate graph: T^T G T
    std::vector<std::vector<int32_t>> grow(na);
    for (int i = 0; i < n; ++i)
      for (int k = G.rp[i]; k < G.rp[i + 1]; ++k) grow[agg[i]].push_back(agg[G.ci[k]]);
    G = from_rows(grow, na);
    L.agg = std::move(agg);
    L.P = std::move(P);
    L.R = std::move(R);
    mg.lv.emplace_back();
    mg.lv.back().A = std::move(An);
  }
  for (auto& L : mg.lv) {
    const double w = (4.0 / 3.0) / gershgorin(L.A);
    L.wd.resize(L.A.n);
    for (int i = 0; i < L.A.n; ++i) L.wd[i] = w / diag_of(L.A, i);
  }
  mg.nc = mg.lv.back().A.n;
  if (mg.nc > 16 * kMGCoarsest) throw Error(DGSL_EINVAL, "multigrid: the aggregation stalled above the dense size");
  mg.C = coarsest_inverse(mg.lv.back().A, singular);
  const int nc = mg.nc;  // exactly symmetric (the kernels read it by columns)
  for (int i = 0; i < nc; ++i)
    for (int j = i + 1; j < nc; ++j) {
      const double v = 0.5 * (mg.C[(size_t)i * nc + j] + mg.C[(size_t)j * nc + i]);
      mg.C[(size_t)i * nc + j] = v;
      mg.C[(size_t)j * nc + i] = v;
    }
}

}  // namespace dgsl
