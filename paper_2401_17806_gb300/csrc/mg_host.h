// Host side of the two-level multigrid preconditioner of dgsl (an extension:
// the paper runs CG unpreconditioned).  Coarse space: continuous
// piecewise-linear functions on the mesh vertices; the vertex-level operator
// A_0 = Pc^T A Pc is solved approximately by one V(1,1)-cycle of smoothed
// aggregation (Vanek, Mandel and Brezina 1996), built here in FP64:
//  - vertex numbering by first appearance over the triangles in RCM order;
//  - A_0 on the combinatorial pattern {vertices of t} x {vertices of t and of
//    its edge neighbours};
//  - greedy two-pass aggregation on a graph (never on values): the mesh-edge
//    graph of the vertices, then the aggregate graph T^T G T per level;
//  - tentative T, smoothed P = T - omega_P D^-1 A T with omega_P = (4/3) /
//    lambda_G (Gershgorin bound of D^-1 A), next level P^T A P on the boolean
//    product pattern (cancelled entries kept as explicit zeros);
//  - down to <= 256 DOFs (or an aggregation step that removes < 20%), then a
//    dense inverse: for the pressure operator (kernel span{1}) the solution is
//    grounded at DOF 0 (Cholesky of the rest) and shifted to mean zero, which
//    for the consistent right-hand sides of the cycle is the pseudo-inverse.
#pragma once

#include <cstdint>
#include <vector>

#include "host.h"

namespace dgsl {

struct CsrD {
  int n = 0, m = 0;               // rows, columns
  std::vector<int32_t> rp, ci;    // row pointers [n + 1], sorted column indices
  std::vector<double> v;
};

struct MGLevelH {
  CsrD A;                         // operator of this level
  std::vector<double> wd;         // Jacobi weights omega_J / a_ii
  CsrD P, R;                      // prolongation to this level from the next (n x n_next) and R = P^T
  std::vector<int32_t> agg;       // aggregate of every DOF (empty on the coarsest level)
};

struct MGHost {
  int nv = 0;                     // vertex DOFs (level 0)
  std::vector<int32_t> cvid;      // [ne][3] coarse DOF of each vertex of each internal triangle
  std::vector<int32_t> v2t_ptr, v2t;  // vertex -> incident (t * 3 + m), sorted by (t, m)
  std::vector<MGLevelH> lv;       // lv.back() is the dense coarsest level
  std::vector<double> C;          // coarsest solve, dense row-major [nc][nc]
  int nc = 0;
};

constexpr int kMGCoarsest = 256;

// Vertex numbering and incidence (depends on the mesh only).
void mg_vertex_numbering(const HostMesh& hm, MGHost& mg);
// Pattern of A_0 from the internal neighbour table nbr [ne][3].
CsrD mg_coarse_pattern(const MGHost& mg, int ne, const std::vector<int32_t>& nbr);
// The mesh-edge graph of the vertices (with the diagonal).
CsrD mg_vertex_graph(const MGHost& mg, int ne);
// Index of (i, j) in a CSR pattern (-1 if absent).
int64_t csr_find(const CsrD& a, int i, int j);
// The smoothed-aggregation levels below A0 (values on its pattern), built on
// graph G0; singular: the pressure operator (kernel span{1}).
void mg_build_levels(MGHost& mg, const CsrD& A0, const CsrD& G0, bool singular);

}  // namespace dgsl
