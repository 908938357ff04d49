// Device-side operator layout and kernel launchers of dgsl (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace dgsl {

// Device copy of one operator.  All arrays are in internal order.
//
// Assembled couplings K = G^T Mhat^{-1} G: for triangle row i and column
// slot b (b = 0: i itself, b = 1..3: neighbour across local edge b-1) the
// block K_b(i) is N_phi x N_phi.  Element (row = i*N_phi + k, c = b*N_phi + kk)
// with c in [0, 4 N_phi) is stored at  vals[(c / VEC) * n_dof * VEC + row * VEC + c % VEC],
// VEC = 16 / sizeof(value): each thread (one matrix row) reads 16-byte
// vectors and a warp reads 512 contiguous bytes per load.
struct DevOp {
  int p = 0, nphi = 0, npsi = 0, ne = 0, nd = 0, ncol = 0;
  int64_t n = 0;                   // n_dof
  int device = 0;
  int ne_pad = 0;                  // row stride of cols: ne rounded up to a multiple of 4
  int32_t* cols = nullptr;         // [4][ne_pad] (padding entries are 0)
  double* K64 = nullptr;           // assembled, FP64
  float* K32 = nullptr;            // assembled, FP32
  uint16_t* K16 = nullptr;         // assembled, BF16 bits
  double* area = nullptr;          // [ne]  A_i = 2|T_i|
  double* Mref = nullptr;          // [nphi][nphi]
  double* Mrefinv = nullptr;       // [nphi][nphi]
  // factored per-edge blocks (optional)
  double* G = nullptr;             // [nd][2][2][nphi][nphi]
  double* Minv = nullptr;          // [nd][npsi][npsi]
  double* Uloc = nullptr;          // [nd][2][nphi][nphi]  A_ij U[a][m][k]
  int32_t* elr = nullptr;          // [nd][2]
  int32_t* tedge = nullptr;        // [ne][3]  2*internal_edge + side
  int colour_offsets[9] = {0};
};

// Dual-index tables (filled once per device): for degree p,
// lmap[p][m], rmap[p][m]: dual index of the left / right local node m;
// dl[p][l], dr[p][l]: local node of dual index l on the left / right half (-1 if none).
void upload_dual_tables(int device);

// ---- applies (stream-ordered, asynchronous)
cudaError_t launch_apply_assembled_f64(const DevOp& op, double coefK, double coefM, const double* x,
                                       double* y, cudaStream_t s);
cudaError_t launch_apply_assembled_f32(const DevOp& op, float coefK, const float* x, float* y,
                                       cudaStream_t s);
cudaError_t launch_apply_factored_f64(const DevOp& op, double coefK, double coefM, const double* x,
                                      double* y, cudaStream_t s);
cudaError_t launch_d2m_rhs(const DevOp& op, const double* vhat, double* b, cudaStream_t s);
cudaError_t launch_m2d(const DevOp& op, const double* vbar, double* vhat, cudaStream_t s);
cudaError_t launch_div(const DevOp& op, const double* vhat, double* y, cudaStream_t s);
cudaError_t launch_velocity_update(const DevOp& op, double coef, const double* F, const double* pr, double* v,
                                   cudaStream_t s);
// y = Mbar^-1 x (per triangle Mref^-1 x_i / A_i) for ncomp main fields of n values
// (y must not alias x).
cudaError_t launch_mass_inv(const DevOp& op, const double* x, double* y, int ncomp, cudaStream_t s);
// y = 2 a - prev, then prev = a (n values; y may be a).
cudaError_t launch_extrapolate(const double* a, double* prev, double* y, int64_t n, cudaStream_t s);

// ---- vector helpers for the refinement loop
// Sum over rows of sum_c (a_c x_c)^2 (FP64 couplings of coefK K + coefM Mbar,
// the self coupling included) into part[2 * block] (k_apply.cu): the rounding
// floor of the FP64 residual.
cudaError_t launch_residual_floor_f64(const DevOp& op, double coefK, double coefM, const double* x, double* part,
                                      int max_parts, int* nparts, cudaStream_t s);
// r = b - A x (FP64 assembled form, A = coefM Mbar + coefK K), optional mean
// projection of b; partial sums of r.r written to part[nblocks]; returns the
// number of CTAs used (<= max_parts).
cudaError_t launch_residual_f64(const DevOp& op, double coefK, double coefM, int mean_zero,
                                const double* b, const double* x, double b_mean, double* r,
                                double* part, int max_parts, int* nparts, cudaStream_t s);
cudaError_t launch_sum2(const double* v, int64_t n, double* part, int max_parts, int* nparts,
                        cudaStream_t s);  // part[j] = (sum v, sum v*v) over CTA j's share
cudaError_t launch_scale_to_f32(const double* v, double scale, float* out, int64_t n, cudaStream_t s);
cudaError_t launch_axpy_f32_to_f64(double a, const float* d, double* x, int64_t n, cudaStream_t s);
cudaError_t launch_remove_mean_f64(double* x, const double* sum_dev, int64_t n, cudaStream_t s);
cudaError_t launch_axpy_f64(double a, const double* d, double* x, int64_t n, cudaStream_t s);
// part[0] = sum_j part[2 j] (fixed order, one CTA)
cudaError_t launch_sum_to_first(double* part, int nparts, cudaStream_t s);

// ---- persistent conjugate gradients (cooperative launch)
// Solves A d = r0 from d = 0 with A = coefM Mbar + coefK K (assembled form in
// the vector type's precision).  r0 is consumed.  Iterates until
// ||r|| <= stop_rel ||r0|| or max_iters.  Result words in `res`:
//   res->iters, res->rr (final recursive r.r), res->status.
struct CGResult {
  int iters;
  int status;
  double rr0;
  double rr;
};
struct CGWork {
  void* vec = nullptr;    // cg_vec_bytes(op, precond): p, x, r, w, s (r, w, s double-buffered; with the
                          // preconditioner also u), per-triangle padded
  double* part = nullptr; // 2 x max_parts x 4 partial sums (6 with the preconditioner; epoch parity)
  GridBarrier* bar = nullptr;
  CGResult* res = nullptr;
  int max_parts = 0;
};
// ---- block-Jacobi preconditioner (an extension)
// P = blockdiag(P_i), P_i = D_i^-1 with D_i = coefK K_0(i) + coefM A_i Mref,
// the diagonal N_phi x N_phi block of A on triangle i, by Cholesky in FP64.
// The preconditioned CG streams the couplings of A P (block (i, j) = A_ij P_j,
// the mass term folded into the diagonal block; the layout of DevOp's K
// arrays) and P itself (element (row, l) at ((l / VP) n + row) VP + l % VP,
// VP = 16 / sizeof(value), padding columns 0).
struct PrecondOp {
  const void* ap = nullptr;    // couplings of A P: FP32, FP64 or BF16 bits (the CG's coupling type)
  const void* pinv = nullptr;  // P: FP32, or FP64 for the FP64 CG
};
// type: 0 FP32 couplings, 1 FP64, 2 BF16 (P in FP32 for 0 and 2, FP64 for 1)
size_t precond_ap_bytes(const DevOp& op, int type);
size_t precond_pinv_bytes(const DevOp& op, int type);
// Builds P in FP64 into p64 (precond_pinv_bytes(op, 1) bytes), A P into ap and
// P in the vector type into pinv (for type 1 pinv may be p64).  *bad (device
// int, zeroed by the caller) becomes 1 if a diagonal block is not positive
// definite.  Needs the FP64 couplings.
cudaError_t launch_build_precond(const DevOp& op, double coefK, double coefM, int type, void* ap, void* pinv,
                                 double* p64, int* bad, cudaStream_t s);

// pre: nullptr for plain CG, else the preconditioned operator built by
// launch_build_precond for the same coefK, coefM and coupling type.
cudaError_t launch_cg_f64(const DevOp& op, double coefK, double coefM, int mean_zero, double* x,
                          double* r, const PrecondOp* pre, double stop_rel, int max_iters, const CGWork& w,
                          uint64_t timeout_ns, cudaStream_t s, int* grid_used);
cudaError_t launch_cg_f32(const DevOp& op, int bf16, float coefK, float coefM, int mean_zero, float* x,
                          float* r, const PrecondOp* pre, double stop_rel, int max_iters, const CGWork& w,
                          uint64_t timeout_ns, cudaStream_t s, int* grid_used);
int cg_max_blocks(const DevOp& op, int prec);
size_t cg_vec_bytes(const DevOp& op, int precond);
// Bounded-wait self-test (see k_cg.cu): records kStatusTimeout in bar->status.
cudaError_t launch_selftest_wait(GridBarrier* bar, int which, uint64_t timeout_ns, cudaStream_t s);
// FMA throughput probe (k_cg.cu): blocks x 256 threads, 8 chains of iters FMAs
// each; out holds blocks * 256 values of the vector type.
cudaError_t launch_fma_rate(int fp64, void* out, int blocks, int iters, cudaStream_t s);

// ---- semi-Lagrangian trajectories and transport (Sec. 2.5, eq. intstage; k_sl.cu)
// Device copy of SLHost (host.h): per-triangle records [ne][16] doubles
// (v0, e1, e2, J^-1, frame translations across local edges 0..2), neighbours
// [ne][4], and the reference data of degree p.
struct SLDev {
  int p = 0, nphi = 0, ng = 0, ne = 0;
  const double* tri = nullptr;
  const int32_t* nbr = nullptr;   // [ne][4]: 3 neighbours, then their local edge indices (2 bits each)
  const double* mono_c = nullptr;  // [nphi][nphi]
  const double* pts = nullptr;     // [ng][2]
  const double* q = nullptr;       // [nphi][ng]
};
constexpr int kSLMaxFields = 8;
// Feet of the ne * ng trajectories (foot [ne * ng][2] in the containing
// triangle's frame, cell and steps [ne * ng], each optional) and the
// transported fields cstar = projection of c at the feet (nf <= 8 fields of n
// values).  vbar: [2][n] main-grid velocity.  Workspace: vmono [ne][2][nphi],
// cmono [nf][ne][nphi].  *err (zeroed by the caller) becomes 1 if a
// trajectory crossed more than max_steps cells (its walk stops there).
cudaError_t launch_sl_transport(const SLDev& g, int64_t n, double dt, const double* vbar, const double* c, int nf,
                                double* cstar, double* foot, int32_t* cell, int32_t* steps, int max_steps,
                                double* vmono, double* cmono, int* err, cudaStream_t s);
// An IMEX Runge-Kutta tableau of ns <= 4 stages: explicit At (strictly lower)
// with weights b, and the implicit A (ai, with its diagonal; weights b too).
struct SLTableau {
  int ns = 0;
  double at[4][4] = {};
  double b[4] = {};
  double ai[4][4] = {};
};
// The tableaux of App. A for R = 0, 1, 2 (false for another R).
bool sl_tableau(int R, SLTableau& t);
// As launch_sl_transport, but the feet come from the stage trajectories of the
// tableau (each stage point and the foot reached from the previous point along
// a straight segment): x^E_s = x - dt sum_{j<s} at[s][j] vbar(x^E_j),
// x_F = x - dt sum_j b_j vbar(x^E_j).  steps: the cells crossed by all the
// segments of a trajectory.
cudaError_t launch_sl_stages(const SLDev& g, int64_t n, double dt, const SLTableau& tab, const double* vbar,
                             const double* c, int nf, double* cstar, double* foot, int32_t* cell, int32_t* steps,
                             int max_steps, double* vmono, double* cmono, int* err, cudaStream_t s);
// The stage velocities V_j = vbar(x^E_j) of every trajectory alone (no foot):
// vout [ns][ne * ng][2].
cudaError_t launch_sl_stage_velocities(const SLDev& g, int64_t n, double dt, const SLTableau& tab, const double* vbar,
                                       double* vout, double* vmono, int max_steps, int* err, cudaStream_t s);
// Stage s (0-based) of the SL-IMEX advection-diffusion step: a[j] = a_{s,j}
// (j <= s) and shift[j] = c_s - c_j of the implicit tableau.
struct SLStage {
  int s = 0;
  double a[4] = {};
  double shift[4] = {};
};
// ci = projection (eq. intstage) of C^n(x - dt sum_{j<=s} a[j] V_j) +
// sum_{j<s} dt a[j] H_j(x - shift[j] dt V_j) over every Gauss point x;
// fields: 1 + s fields of n values, fstride apart (C^n, H_0, ..., H_{s-1});
// V as launch_sl_stage_velocities; cmono workspace [1 + s][ne][nphi].
cudaError_t launch_sl_advdiff_stage(const SLDev& g, int64_t n, int64_t fstride, double dt, const SLStage& st,
                                    const double* V, const double* fields, double* cmono, double* ci, int max_steps,
                                    int* err, cudaStream_t s);
// V_s (s = st.s) of every trajectory: the two-component main-grid field
// field2 (components fstride apart) at x - dt sum_{j<s} st.a[j] V_j; vmono
// workspace [ne][2][nphi].
cudaError_t launch_sl_stage_velocity(const SLDev& g, int64_t fstride, double dt, const SLStage& st,
                                     const double* field2, double* V, double* vmono, int max_steps, int* err,
                                     cudaStream_t s);
// h = (cst - ci) * inv, n values.
cudaError_t launch_sl_flux(const double* cst, const double* ci, double inv, double* h, int64_t n, cudaStream_t s);

void count_launch(int n = 1);
uint64_t launch_count();

}  // namespace dgsl
