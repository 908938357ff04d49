// Host-side data structures of the dgsl library: mesh connectivity, orders,
// reference operators of Sec. 2.4 and FP64 block precompute.
#pragma once

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dgsl.h"

namespace dgsl {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

inline int n_phi_of(int p) { return (p + 1) * (p + 2) / 2; }
inline int n_psi_of(int p) { return (p + 1) * (p + 1); }

// Element-independent matrices of Sec. 2.4 on the reference triangle.
//   Mref[k][l]     = int_Tref phi_k phi_l                              (eq. MassMatrixM)
//   V[a][k][m][d]  = int_Tref (d_d phi_k)(T_a^{-1} z) phi_m(z) dz      (volume part, D^{V,a,.})
//   Line[a][k][m]  = int_0^1 phi_k(nu_a + t (nu_{a+1} - nu_a)) phi_m(1 - t, t) dt
//                                                                      (line part, D^{L,a,.})
//   U[a][m][k]     = int_Tref phi_m(z) phi_k(T_a^{-1} z) dz            (eq. u)
// where T_a^{-1} maps T_ref onto the sub-triangle (b_ref, nu_a, nu_{a+1}).
// The dual halves carry phi_m with dual index Lmap[m] (left) / Rmap[m] (right).
struct RefOps {
  int p = 0, nphi = 0, npsi = 0;
  std::vector<int> Lmap, Rmap;
  std::vector<double> Mref, V, Line, U;
};
RefOps build_reference_operators(int p);

struct HostMesh {
  int nv = 0, ne = 0, nd = 0;
  double period[2] = {1.0, 1.0};
  std::vector<double> txy;             // [ne][3][2] unwrapped vertices
  std::vector<int32_t> tri_v;          // [ne][3] vertex ids as given, natural numbering
  std::vector<int32_t> edge_vtx, lr;   // [nd][2], natural numbering
  std::vector<uint8_t> loc;            // [nd][2]
  std::vector<int8_t> shift;           // [nd][2]
  std::vector<int32_t> tri_edge;       // [ne][3]
  std::vector<int32_t> perm, rank;     // perm[internal] = natural, rank = inverse
  std::vector<int32_t> edge_perm, edge_rank;
  std::vector<uint8_t> colour;         // natural edge numbering
  std::vector<int32_t> colour_offsets; // [n_colours + 1]
  int n_colours() const { return (int)colour_offsets.size() - 1; }
};
HostMesh build_mesh(const dgsl_mesh& m);

// FP64 blocks, internal numbering.
struct HostBlocks {
  int p = 0, nphi = 0, npsi = 0, ne = 0, nd = 0;
  std::vector<double> area;      // [ne] A_i = 2|T_i|
  std::vector<double> G;         // [nd][2 side][2 comp][nphi m][nphi k]
  std::vector<double> Minv;      // [nd][npsi][npsi]
  std::vector<double> Kd;        // [ne][nphi][nphi]     diagonal coupling block
  std::vector<double> Ko;        // [ne][3][nphi][nphi]  block to neighbour across local edge k
  std::vector<int32_t> nbr;      // [ne][3] internal neighbour index
  std::vector<int32_t> elr;      // [nd][2] internal (l, r)
  std::vector<uint8_t> eloc;     // [nd][2]
  std::vector<double> Uloc;      // [nd][2 side][nphi m][nphi k] = A_ij U[a][m][k]
};
HostBlocks build_blocks(const HostMesh& hm, const RefOps& ro);

void node_coords(const HostMesh& hm, const RefOps& ro, int grid, double* out);

// Semi-Lagrangian walk (Sec. 2.5): per-triangle records in internal order
// (see SLTri in kernels.h) and the reference data of degree p:
//   mono_c[m][k]  coefficient of monomial m = x^i y^j ((i, j) with i = 0..p
//                 outer, j = 0..p-i inner) in phi_k;
//   pts[g][2], w[g]  the collapsed Gauss-Legendre rule, (p+1)^2 points;
//   q[k][g] = sum_l (Mref^-1)[k][l] phi_l(pts_g) w_g  (the projection of
//                 eq. intstage; |J_i| cancels against Mbar_i = A_i Mref).
struct SLHost {
  int p = 0, nphi = 0, ng = 0;
  std::vector<double> tri;  // [ne][16] doubles: v0 (2), e1 (2), e2 (2), J^-1 (4), translations (3 x 2)
  std::vector<int32_t> nbr; // [ne][4]: neighbours across local edges 0..2 (internal); word 3 holds,
                            // in bits 2k..2k+1, the local index of edge k in the neighbour across it
  std::vector<double> mono_c, pts, w, q;
};
SLHost build_sl_host(const HostMesh& hm, const RefOps& ro);
// Mref^-1 (row-major), for the inverse main-grid mass matrix Mbar_i^-1 = Mref^-1 / A_i.
std::vector<double> mref_inverse(const RefOps& ro);
// The quadrature rule of SLHost alone (no mesh needed).
void sl_rule(int p, std::vector<double>& pts, std::vector<double>& w);

}  // namespace dgsl
