/*
 * dgsl — GB300-native implicit-stage solver library for the staggered
 * semi-Lagrangian IMEX DG method of Tavelli & Boscheri.
 *
 * The library builds, from a periodic triangulation and a degree p, the
 * operators of the implicit stage (Sec. 2.3-2.4) and solves
 *
 *   pressure Schur system (eq. pressure_final, eq. pressure_IMEX):
 *       S p = b,   S = dt^2 * G^T Mhat^{-1} G          (symmetric, PSD)
 *   implicit diffusion / viscosity system (eq. ad5, lambda = nu):
 *       H v = b,   H = Mbar + nu*dt * G^T Mhat^{-1} G  (SPD)
 *
 * with G the gradient operator of eq. ad5.2 (blocks Q_ij), Mhat the C0 dual
 * mass matrix of eq. Mj (one (p+1)^2 block per edge quad) and Mbar the main
 * mass matrix of eq. Mi.  Because D = -Q^T (Sec. 2.3), the paper's left-hand
 * side sum_j D_ij Mhat_j^{-1}(Q_lj p_l + Q_rj p_r) equals -(G^T Mhat^{-1} G p)_i;
 * the library exposes the positive semidefinite sign, so a caller holding the
 * paper's right-hand side passes its negation.
 *
 * Conventions for every call below
 *  - Every call returns an int status (DGSL_OK = 0).  No C++ exception
 *    crosses this boundary.  dgsl_last_error() returns a thread-local
 *    message for the last failing call on the calling thread.
 *  - "device pointer": memory on the operator's CUDA device, owned by the
 *    caller (e.g. a PyTorch tensor's data_ptr()); "host pointer": ordinary
 *    host memory owned by the caller.  The library never retains caller
 *    pointers after a call returns unless the call says so (dgsl_submit).
 *  - "stream" is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Device-pointer calls are asynchronous on that stream
 *    unless stated otherwise.
 *  - Vector layout (internal order): triangles are renumbered by reverse
 *    Cuthill-McKee and edges by (colour, RCM key).  A main-grid vector is
 *    double[n_tri][n_phi] with triangle t at internal position t; a scalar
 *    dual-grid field is double[n_edge][n_psi] in internal edge order; a
 *    vector dual field is double[2][n_edge][n_psi] (x component first).
 *    dgsl_query_maps() returns perm (internal -> natural triangle id) and
 *    edge_perm (internal -> natural edge id).  Several right-hand sides are
 *    stored one after another (rhs-major).
 *  - Local DOF order: main node k of T_ref is (a/p, b/p), a + b <= p,
 *    b-major then a.  Dual DOF order: the n_phi nodes of the left half, then
 *    the right-half nodes off the diagonal, in the same order.
 */
#ifndef DGSL_H
#define DGSL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
enum {
  DGSL_OK = 0,
  DGSL_EINVAL = 1,      /* bad argument (NULL, size, degree out of 1..4, ...) */
  DGSL_EMESH = 2,       /* inverted / degenerate / non-manifold / too coarse mesh */
  DGSL_ENOMEM = 3,      /* host or device allocation failed */
  DGSL_EBUDGET = 4,     /* request can never fit the server's memory budget */
  DGSL_ENOTCONV = 5,    /* max_iters reached; best iterate returned */
  DGSL_ETIMEOUT = 6,    /* a bounded device wait expired */
  DGSL_EPENDING = 7,    /* dgsl_poll: request not finished yet */
  DGSL_ECUDA = 8,       /* CUDA runtime error */
  DGSL_ENODEVICE = 9    /* called a device path on a host-only operator */
};

/* Thread-local message of the last failing call ("" if none). */
const char* dgsl_last_error(void);

/* Library version string. */
const char* dgsl_version(void);

/* Number of kernels this library has launched in this process. */
uint64_t dgsl_launch_count(void);

/* ------------------------------------------------------------ mesh */
/* Periodic triangulation (Sec. 2.1).  Host pointers, caller-owned, copied
 * during dgsl_build_operators and never retained.
 *   xy  : double[n_vertices][2] vertex coordinates
 *   tri : int32[n_triangles][3] counter-clockwise vertex ids (after each
 *         triangle's vertices are moved to their minimum image relative to
 *         its first vertex)
 *   period : the torus periods in x and y (> 0). */
typedef struct {
  int32_t n_vertices;
  const double* xy;
  int32_t n_triangles;
  const int32_t* tri;
  double period[2];
} dgsl_mesh;

typedef struct dgsl_operator dgsl_operator;

enum { DGSL_STORE_F64 = 1, DGSL_STORE_F32 = 2, DGSL_STORE_BF16 = 4 };

typedef struct {
  int32_t host_only;   /* 1: build host maps and FP64 blocks only (no GPU) */
  int32_t device;      /* CUDA device ordinal */
  int32_t store;       /* DGSL_STORE_* mask of block copies kept on device
                          (0 = F64|F32) */
  int32_t factored;    /* 1: also keep the per-edge G / Mhat^{-1} blocks */
  void* stream;        /* cudaStream_t of the build's host-to-device copies
                          (NULL: legacy default stream); the build returns
                          after they have completed on it */
} dgsl_build_opts;

/* Builds connectivity (left/right triangles by first encounter), the RCM
 * order, the greedy edge colouring, the geometry and, from the reference
 * operators of Sec. 2.4, the per-edge blocks G_lj, G_rj, Mhat_j^{-1} and
 * the assembled couplings K = G^T Mhat^{-1} G (4 blocks per triangle row).
 * p in 1..4.  opts may be NULL (defaults).  On success *out owns all host
 * and device storage; release it with dgsl_destroy_operator.
 * Errors: EINVAL, EMESH (inverted, degenerate, non-manifold or a periodic
 * mesh so coarse that two triangles share two edges), ENOMEM, ECUDA. */
int dgsl_build_operators(const dgsl_mesh* mesh, int p, const dgsl_build_opts* opts,
                         dgsl_operator** out);
void dgsl_destroy_operator(dgsl_operator* op);

typedef struct {
  int32_t p, n_phi, n_psi;
  int32_t n_tri, n_edge, n_colours;
  int64_t n_dof;          /* n_tri * n_phi */
  int64_t n_dual;         /* n_edge * n_psi */
  int64_t device_bytes;   /* device memory held by the operator */
  int32_t host_only;
  int32_t device;
} dgsl_info;
int dgsl_operator_info(const dgsl_operator* op, dgsl_info* out);

/* Host copies of the index maps (caller-allocated host arrays; any member
 * may be NULL to skip it).  Natural numbering unless noted.
 *   edge_vtx [n_edge][2]  (X1, X2): counter-clockwise in the left triangle
 *   lr       [n_edge][2]  left, right triangle
 *   loc      [n_edge][2]  local edge index (0..2) in left, right
 *   shift    [n_edge][2]  periods added to the right triangle's frame
 *   tri_edge [n_tri][3]   edge of local edge k = (v_k, v_{k+1 mod 3})
 *   perm     [n_tri]      internal -> natural triangle
 *   edge_perm[n_edge]     internal -> natural edge
 *   colour   [n_edge]     colour of each natural edge
 *   colour_offsets [n_colours + 1] internal edge ranges per colour */
typedef struct {
  int32_t* edge_vtx;
  int32_t* lr;
  uint8_t* loc;
  int8_t* shift;
  int32_t* tri_edge;
  int32_t* perm;
  int32_t* edge_perm;
  uint8_t* colour;
  int32_t* colour_offsets;
} dgsl_maps;
int dgsl_query_maps(const dgsl_operator* op, dgsl_maps* out);

enum { DGSL_MAIN = 0, DGSL_DUAL = 1 };
/* Physical coordinates of the nodal DOFs, host double[n][2] in internal
 * order: grid DGSL_MAIN -> n_tri*n_phi nodes (each triangle in its own
 * unwrapped frame); DGSL_DUAL -> n_edge*n_psi nodes (in the left triangle's
 * frame). */
int dgsl_node_coords(const dgsl_operator* op, int grid, double* xy);

/* The neighbour tables of the semi-Lagrangian walk (Sec. 2.5), host arrays
 * in internal triangle order, each optional: nbr int32[n_tri][4] (the
 * neighbours across local edges 0..2, then in bits 2k..2k+1 of the fourth
 * word the local index of edge k in that neighbour) and trans
 * double[n_tri][3][2] (the whole periods that carry a point of the triangle's
 * frame into the neighbour's frame across local edge k).  Pure host call;
 * also for host-only operators. */
int dgsl_query_sl_tables(const dgsl_operator* op, int32_t* nbr, double* trans);

/* Host FP64 copies of the assembled couplings of K = G^T Mhat^{-1} G (the
 * Schur operator is dt^2 K, eq. pressure_final; the viscous one Mbar + nu dt K,
 * eq. ad5), internal triangle order (any pointer may be NULL):
 *   Kd  [n_tri][n_phi k][n_phi l]     block (i, i): row (i, k), column (i, l)
 *   Ko  [n_tri][3][n_phi k][n_phi l]  block (i, nbr[i][e]) across local edge e
 *   nbr [n_tri][3]                    the neighbour across local edge e
 * These are the values the device copies are made from (FP64 as is, FP32 and
 * BF16 rounded, with the self coupling stored as 0 in the difference form).
 * Kept only for host_only or factored builds (DGSL_EINVAL otherwise).  Pure
 * host call. */
int dgsl_query_couplings(const dgsl_operator* op, double* Kd, double* Ko, int32_t* nbr);

/* Host FP64 copies of the blocks, internal edge order (any may be NULL):
 *   G    [n_edge][2 side][2 comp][n_phi m][n_phi k] = Q_{s,j}[L_s(m), k, comp]
 *        (eq. ad5.2 restricted to the dual nodes of side s)
 *   Minv [n_edge][n_psi][n_psi]   Mhat_j^{-1}
 *   Mref [n_phi][n_phi]           Mbar_ref (eq. MassMatrixM)
 *   area [n_tri]                  A_i = 2|T_i| (internal order) */
int dgsl_query_blocks(const dgsl_operator* op, double* G, double* Minv, double* Mref,
                      double* area);

/* ------------------------------------------------------------ applies */
/* Forms of the Schur / Helmholtz matvec. */
enum {
  DGSL_FORM_ASSEMBLED = 0,  /* stored couplings K (4 blocks per triangle row) */
  DGSL_FORM_FACTORED = 1    /* stored G, Mhat^{-1} per edge, edge-coloured phases */
};

/* y = dt^2 G^T Mhat^{-1} G x  (eq. pressure_final, PSD sign).
 * x, y: device double[n_rhs][n_dof], internal order, may not alias.
 * form: DGSL_FORM_*; FACTORED needs opts.factored at build time. */
int dgsl_apply_schur(const dgsl_operator* op, int form, double dt, const double* x, double* y,
                     int n_rhs, void* stream);

/* Same in FP32 (FP32 blocks and vectors, FP32 accumulation). */
int dgsl_apply_schur_f32(const dgsl_operator* op, float dt, const float* x, float* y, int n_rhs,
                         void* stream);

/* y = (Mbar + nu_dt G^T Mhat^{-1} G) x  (eq. ad5 with lambda*dt = nu_dt). */
int dgsl_apply_helmholtz(const dgsl_operator* op, double nu_dt, const double* x, double* y,
                         int n_rhs, void* stream);

/* b_i = sum_{j in S_i} U_ij^T vhat_j (eq. d2m times Mbar_i; eq. u), for
 * n_rhs scalar dual fields vhat [n_rhs][n_edge][n_psi] -> b [n_rhs][n_dof]. */
int dgsl_project_d2m_rhs(const dgsl_operator* op, const double* vhat, double* b, int n_rhs,
                         void* stream);

/* vhat_j = Mhat_j^{-1} (U_lj vbar_l + U_rj vbar_r) (eq. m2d), for n_rhs scalar
 * main fields vbar [n_rhs][n_dof] -> vhat [n_rhs][n_edge][n_psi]. */
int dgsl_project_m2d(const dgsl_operator* op, const double* vbar, double* vhat, int n_rhs,
                     void* stream);

/* y = G^T vhat = -sum_j D_ij vhat_j (eqs. ins.1 / D), vhat a vector dual field
 * [n_rhs][2][n_edge][n_psi] -> y [n_rhs][n_dof]. */
int dgsl_apply_div(const dgsl_operator* op, const double* vhat, double* y, int n_rhs,
                   void* stream);

/* Velocity update of the pressure projection (eq. nc.2 solved for the new
 * dual velocity, its gravity / buoyancy source terms left to the caller):
 *   v_j = F_j - coef Mhat_j^{-1} (Q_lj p_l + Q_rj p_r)
 * for n_rhs vector dual fields F, v [n_rhs][2][n_edge][n_psi] and main fields
 * p [n_rhs][n_dof] (device, internal orders; v may be F).  coef = dt for the
 * paper's pressure; for the p of dgsl_cg_solve(DGSL_SCHUR, dt, b = G^T F)
 * (S = dt^2 G^T Mhat^-1 G) coef = dt^2, and then G^T v = b - S p: the
 * divergence of v is the pressure solve's residual (eq. nc.1).  Needs an
 * operator built with opts.factored (DGSL_EINVAL otherwise). */
int dgsl_velocity_update(const dgsl_operator* op, double coef, const double* F, const double* p,
                         double* v, int n_rhs, void* stream);

/* ------------------------------------------------------------ semi-Lagrangian transport */
/* The quadrature rule of dgsl_sl_transport for degree p (1..4): the
 * collapsed Gauss-Legendre rule on T_ref with n_g = (p+1)^2 points (exact to
 * degree 2p+1); pts [n_g][2] (xi, eta) and w [n_g] (sum 1/2), host arrays,
 * each optional.  Pure host call. */
int dgsl_sl_quadrature(int p, double* pts, double* w, int32_t* n_g);

/* Semi-Lagrangian transport on the main grid (Sec. 2.5, eq. lagrtrj; the
 * Gauss-point projection of eq. intstage).  The characteristic of every
 * quadrature point x_g of every triangle is followed backward over dt
 * (forward if dt < 0) in straight Euler pieces, cell by cell: from x in
 * triangle T with T's velocity polynomial v at x, the ray x - s v either
 * ends in T after the time left (the foot) or leaves T through the edge whose
 * opposite barycentric coordinate first reaches 0 (ties: the lowest local
 * edge), and the walk continues in the neighbour across it (periodic
 * neighbours by a frame translation), with no global search.  A walk sent
 * back through the edge it entered a cell by may do so once; sent across
 * that edge again at once, it is held there (the foot is that point, the
 * time left dropped: the velocity on both sides points at the edge).  The fields are
 * evaluated at the feet in the containing triangles and projected back:
 *   cstar_i = Mbar_i^{-1} sum_g phi(xi_g) c(x_F(x_g)) w_g |J_i|.
 *  - vbar: device double[2][n_dof], the main-grid velocity (two components,
 *    each [n_tri][N_phi] nodal coefficients in internal order).
 *  - c, cstar: device double[n_fields][n_dof] (n_fields 0..8; cstar must not
 *    alias c or vbar).
 *  - foot: device double[n_tri * n_g][2], the foot of trajectory
 *    (triangle i, point g) at index i n_g + g, in the frame of the triangle
 *    that contains it (its vertices unwrapped around its first vertex); cell:
 *    device int32[n_tri * n_g], that triangle (internal index); steps: device
 *    int32[n_tri * n_g], the cells crossed.  Each may be NULL.
 * Synchronous (reads a status word).  Returns DGSL_ENOTCONV if a trajectory
 * crossed more than 65536 cells (its walk stops there). */
int dgsl_sl_transport(const dgsl_operator* op, double dt, const double* vbar, const double* c,
                      double* cstar, int n_fields, double* foot, int32_t* cell, int32_t* steps,
                      void* stream);

/* Semi-Lagrangian transport with the stage trajectories of the IMEX scheme
 * of degree R (Sec. 3, the explicit tableau (A~, b) of App. A: R = 0 Euler,
 * R = 1 two stages, R = 2 four stages with the printed six digits), for a
 * field carried by a steady main-grid velocity vbar without diffusion.
 * Every Gauss point x follows
 *   x^E_s = x - dt sum_{j<s} a~_{s,j} V_j,  V_j = vbar(x^E_j),
 *   x_F   = x - dt sum_j b_j V_j,
 * each stage point located by walking the straight segment from the
 * previous one (the first from x, the foot from the last), cell by cell, as
 * in dgsl_sl_transport (so vbar is evaluated with the polynomial of the cell
 * reached).  The feet converge at order R + 1 in dt.
 * The fields are evaluated at x_F and projected as in dgsl_sl_transport.
 * Arguments, outputs and errors as dgsl_sl_transport (steps: the cells
 * crossed by all segments of a trajectory); DGSL_EINVAL for R outside 0..2. */
int dgsl_sl_transport_imex(const dgsl_operator* op, int R, double dt, const double* vbar,
                           const double* c, double* cstar, int n_fields, double* foot,
                           int32_t* cell, int32_t* steps, void* stream);

/* ------------------------------------------------------------ solves */
enum { DGSL_SCHUR = 0, DGSL_HELMHOLTZ = 1 };
enum {
  DGSL_PREC_F64 = 0,       /* FP64 CG on FP64 blocks */
  DGSL_PREC_F32_IR = 1,    /* FP32 inner CG, FP64 iterative refinement */
  DGSL_PREC_BF16_IR = 2    /* BF16-stored blocks, FP32 inner CG, FP64 refinement */
};

enum {
  DGSL_PRECOND_NONE = 0,         /* plain CG, as the paper runs it (default) */
  DGSL_PRECOND_BLOCK_JACOBI = 1, /* CG preconditioned by the inverse N_phi x N_phi
                                    diagonal blocks of A (one per triangle) */
  DGSL_PRECOND_MULTIGRID = 2     /* PCG with a two-level multigrid preconditioner:
                                    damped block-Jacobi smoothing and a continuous
                                    P1 vertex coarse space solved by one
                                    smoothed-aggregation V-cycle (see
                                    dgsl_apply_multigrid) */
};

typedef struct {
  double tol;            /* target ||b - A x||_2 / ||b||_2 (default 1e-10) */
  int32_t max_iters;     /* cap on CG iterations, all refinements (default 200000) */
  int32_t precision;     /* DGSL_PREC_* */
  int32_t use_x0;        /* 1: x holds the initial guess */
  double inner_tol;      /* inner CG relative tolerance under refinement (1e-3) */
  int32_t max_refine;    /* refinement steps cap (default 30) */
  int32_t form;          /* DGSL_FORM_* of the FP64 operator */
  int32_t precond;       /* DGSL_PRECOND_* (default NONE) */
  int32_t pad;
} dgsl_solve_opts;

typedef struct {
  int32_t status;        /* DGSL_OK or DGSL_ENOTCONV / DGSL_ETIMEOUT */
  int32_t iters;         /* CG iterations (sum over refinements) */
  int32_t refinements;   /* outer FP64 refinement steps */
  int32_t cg_launches;   /* persistent CG launches (one per refinement step) */
  double relres;         /* final ||b - A x|| / ||b|| with the FP64 operator */
  double cg_kernel_ms;   /* device time of those launches (CUDA events on the
                            solve's stream) */
  int32_t grid;          /* CTAs of the persistent CG launches */
  int32_t pad;
  double relres_floor;   /* dgsl_cg_solve, status DGSL_ENOTCONV only (else 0):
                            the expected relative residual of the exact
                            solution rounded to FP64, from the returned x and
                            the FP64 couplings (each value's rounding error
                            uniform in +-2^-53, independent).  No FP64 vector
                            has a residual far below it: a relres within a
                            small multiple of it is at FP64's own accuracy.
                            The engine and the no-allocation solve leave 0. */
} dgsl_solve_info;

/* Solves A x = b for kind DGSL_SCHUR (A = S with dt = coef) or
 * DGSL_HELMHOLTZ (A = H with nu_dt = coef) by matrix-free CG (Sec. 2.3,
 * after eq. pressure_final), with x0 = 0 unless use_x0, stopping at the
 * relative residual tol.  With precond = DGSL_PRECOND_BLOCK_JACOBI the inner
 * CG is preconditioned by P = blockdiag(D_i)^-1, D_i the diagonal block of A on
 * triangle i (an extension; the paper's CG is unpreconditioned): the operator
 * builds P on first use for each (kind, coef, precision) and keeps the blocks
 * of the last four such systems (N_phi values per row, rounded up to 4 in
 * FP32 or 2 in FP64; about 48 / 80 bytes per DOF at p = 3); DGSL_EINVAL if a
 * diagonal block is not positive definite.  With precond =
 * DGSL_PRECOND_MULTIGRID the inner solve is PCG with the two-level
 * preconditioner of dgsl_apply_multigrid (built on first use per system; the
 * inner iterations then stay nearly constant as the mesh is refined).  For
 * DGSL_SCHUR, b is projected to mean zero and x
 * is returned with sum(x) = 0 (coefficient space).  b, x: device
 * double[n_rhs][n_dof] in internal order; info: host array [n_rhs] or NULL.
 * Blocks the calling thread until the solves finish (it reads the status
 * words back).  Returns DGSL_ENOTCONV (x = last iterate) if any right-hand
 * side missed tol within max_iters. */
int dgsl_cg_solve(const dgsl_operator* op, int kind, double coef, const double* b, double* x,
                  int n_rhs, const dgsl_solve_opts* opts, dgsl_solve_info* info, void* stream);

/* The two-level multigrid preconditioner M of DGSL_PRECOND_MULTIGRID (an
 * extension: the paper runs CG unpreconditioned, with iteration counts that
 * grow like 1/h; the operators are those of eq. pressure_final and eq. ad5).
 * For A = S (kind DGSL_SCHUR, dt = coef) or H (DGSL_HELMHOLTZ, nu_dt = coef):
 *   x1 = 0.7 D^-1 r,   x2 = x1 + Pc V(Pc^T (r - A x1)),
 *   z  = x2 + 0.7 D^-1 (r - A x2),
 * D = blockdiag of A's N_phi x N_phi diagonal blocks; Pc interpolates
 * continuous piecewise-linear functions on the mesh vertices at each
 * triangle's nodes (vertices numbered by first appearance over the triangles
 * in internal order); V is one V(1,1)-cycle of smoothed aggregation on
 * A_0 = Pc^T A Pc: greedy two-pass aggregation on the mesh-edge graph of the
 * vertices (then on the aggregate graphs), prolongations
 * P = T - (4/3 / lambda_G) diag(A)^-1 A T (lambda_G the Gershgorin bound of
 * diag(A)^-1 A), Galerkin levels down to <= 256 DOFs, damped Jacobi
 * smoothing (weight 4/3 / lambda_G), and a dense coarsest inverse (for S the
 * mean-zero pseudo-inverse).  The operator builds the hierarchy on first use
 * per (kind, coef, precision) and keeps the last four.
 * dgsl_apply_multigrid applies z = M r once: precision DGSL_PREC_F64 with
 * double r, z and FP64 couplings; DGSL_PREC_F32_IR (FP32 couplings) or
 * DGSL_PREC_BF16_IR (BF16 couplings in the two smoother residuals) with float
 * r, z; device vectors [n_dof] in internal order.  Synchronous.  In the solve
 * with DGSL_PREC_BF16_IR the PCG matvec, which defines the system solved,
 * keeps the FP32 couplings (both must be stored): BF16 rounding of the
 * couplings moves the small eigenvalues of the pressure operator, and only
 * the preconditioner may be that inexact.  DGSL_EINVAL if a block of D or the
 * coarsest operator is not positive definite. */
int dgsl_apply_multigrid(const dgsl_operator* op, int kind, double coef, int precision, const void* r,
                         void* z, void* stream);

typedef struct {
  int32_t n_levels;       /* coarse levels, the vertex level first, the dense one last */
  int32_t n_vertices;     /* DOFs of the vertex level */
  int32_t sizes[16];      /* DOFs of each level */
} dgsl_mg_info;
/* The hierarchy of dgsl_apply_multigrid for (kind, coef) (integer data, for
 * checks): info; cvid (host int32[n_tri][3], natural triangle order, or NULL):
 * the vertex-level DOF of each triangle vertex; agg (host int32, or NULL):
 * the aggregate of every DOF of levels 0 .. n_levels-2, concatenated.  The
 * aggregation depends on the mesh only.  Synchronous. */
int dgsl_query_multigrid(const dgsl_operator* op, int kind, double coef, dgsl_mg_info* info, int32_t* cvid,
                         int32_t* agg);

void dgsl_default_solve_opts(dgsl_solve_opts* opts);

/* Failure-detection self-test (no counterpart in the paper; the persistent
 * solvers' waits are bounded): which = 0 runs the persistent CG's grid barrier
 * expecting one CTA more than are launched, which = 1 waits on an mbarrier that
 * no copy completes.  Each wait gives up after timeout_s (0 < timeout_s <= 5),
 * the kernel records the timeout and returns; *status receives DGSL_ETIMEOUT
 * if it did (DGSL_OK otherwise) and the device stays usable.  Synchronous. */
int dgsl_selftest_wait_timeout(int device, int which, double timeout_s, int* status);

/* Measured FMA throughput of the device (no counterpart in the paper: the
 * denominator of the roofline of the FP64-ALU-bound kernels, the
 * semi-Lagrangian walk above all).  fp64 = 1 times FP64, 0 FP32: 3 warm-up and
 * 10 timed launches (CUDA events on a private stream) of SMs x 8 blocks of 256
 * threads, each thread running 8 independent FMA chains; *flops_per_s receives
 * 2 x FMAs / second.  Allocates a small output buffer (freed before return).
 * Synchronous; DGSL_EINVAL for a bad argument, DGSL_ECUDA on a CUDA error. */
int dgsl_measure_fma_rate(int device, int fp64, double* flops_per_s);

/* Same solve as dgsl_cg_solve (precond must be DGSL_PRECOND_NONE: the fixed
 * scratch has no room for the preconditioner's blocks; else DGSL_EINVAL), for
 * callers that cannot allocate device memory when they solve: real-time loops
 * and services that reserve all device memory at start-up under a fixed budget
 * (an allocation mid-run could fail or stall them), and hosts whose own
 * allocator owns the GPU's memory.  This entry point calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its scratch is one fixed device array
 * inside the library (about 28 MB: thirteen vectors of 262,144 doubles plus
 * reduction slots) that every GPU which loads the library's code holds until
 * the process exits.  The paper has no counterpart; this is a deployment
 * convenience.
 *  - Limit: op's n_dof <= 262,144 (per right-hand side); larger operators are
 *    rejected with DGSL_EINVAL before anything runs.
 *  - The array is reserved on a device when the library's code is loaded there.
 *    Under CUDA's default lazy module loading that happens at the first call of
 *    this entry point on that device, which also looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current: make one call
 *    (any small solve) before reserving the rest of the memory budget.
 *  - It cannot run while its stream is being captured into a CUDA graph: the
 *    refinement loop copies the residual norm to the host and synchronises the
 *    stream after every step.  A call on a capturing stream (or one whose
 *    capture state cannot be read) returns DGSL_EINVAL before enqueuing
 *    anything, leaving the capture intact.
 *  - Every call on a device shares the one array, which keeps whatever the last
 *    call left in it; everything a solve needs zeroed is cleared by the call.
 *    Calls are serialized by a lock and return only after their GPU work has
 *    finished; two solves that overlapped on the GPU would race on the array.
 *  - The grids and reduction order are those of dgsl_cg_solve, so the result is
 *    the same, bit for bit.  Arguments, results and errors as dgsl_cg_solve,
 *    except that info->cg_kernel_ms is reported as 0 (no timing events are
 *    created). */
int dgsl_cg_solve_noalloc(const dgsl_operator* op, int kind, double coef, const double* b,
                          double* x, int n_rhs, const dgsl_solve_opts* opts,
                          dgsl_solve_info* info, void* stream);

/* ------------------------------------------------------------ Navier-Stokes step */
/* One first-order semi-Lagrangian semi-implicit step of the incompressible
 * Navier-Stokes equations on the staggered grids: the one-stage (R = 0, Euler)
 * tableau of App. A applied to the splitting of Sec. 3, without temperature
 * or gravity.
 *  1. vbar = L_dm(vhat_in) (eq. d2m), the main-grid velocity;
 *  2. c = vbar transported by itself over dt (dgsl_sl_transport, Sec. 2.5);
 *  3. (Mbar + nu dt K) vbar* = Mbar c per component (eq. ad5, lambda = nu);
 *  4. vhat* = L_md(vbar*) (eq. m2d);
 *  5. S p = G^T vhat* with S = dt^2 G^T Mhat^-1 G (eq. pressure_final);
 *  6. vhat_out = vhat* - dt^2 Mhat^-1 G p (eq. nc.2), so that G^T vhat_out = 0.
 * vhat_in, vhat_out: device double[2][n_dual] (may alias); p_out: device
 * double[n_dof] in internal order, or NULL: receives p of step 5.  opts
 * govern the three solves (tolerance, precision, preconditioner); the
 * Helmholtz solves start from c, and the pressure solve starts from the
 * contents of p_out when opts->use_x0 is set and p_out is given (the last
 * step's pressure), else from 0.  With opts->use_x0 == 2 and p_out it starts
 * from the linear extrapolation 2 p^n - p^{n-1}: the operator keeps the
 * pressure of the last step called this way (the first such call only
 * records it).  Steps of another run on the same operator only make that
 * guess worse; the result still meets opts->tol.  info: host array of 3 or NULL (Helmholtz x,
 * Helmholtz y, Schur).  Needs an operator built with opts.factored.
 * Synchronous.  Returns the first non-OK solve status, or DGSL_ENOTCONV if a
 * trajectory crossed more than 65536 cells. */
int dgsl_ns_step(const dgsl_operator* op, double dt, double nu, const double* vhat_in,
                 double* vhat_out, double* p_out, const dgsl_solve_opts* opts,
                 dgsl_solve_info* info, void* stream);

/* One semi-Lagrangian IMEX step of the incompressible Navier-Stokes
 * equations (no temperature or gravity) with the tableaux of App. A,
 * R = 0, 1, 2.  Stages as dgsl_advdiff_step for the two main-grid velocity
 * components, starting from vbar^n = L_dm(vhat_in) (eq. d2m), with:
 *  - the stage velocity of each trajectory V_s = vbar^E_s(x^E_s), where the
 *    explicit stage field vbar^E_s is formed like the implicit stage value
 *    with the explicit row a~_s and shifts c~_s - c_j (V_1 = vbar^n(x));
 *  - per stage: the viscous solves (Mbar + a_ss dt nu K) vbar* = Mbar vbar^I
 *    (eq. ad5), vhat* = L_md(vbar*) (eq. m2d), the pressure solve
 *    S pi = G^T vhat* with S = (a_ss dt)^2 G^T Mhat^-1 G (eq. pressure_final)
 *    and vhat_s = vhat* - (a_ss dt)^2 Mhat^-1 G pi (eq. nc.2);
 *  - the stage flux Hhat_s = (vhat_s - L_md(vbar^I_s)) / (a_ss dt) on the dual
 *    grid, shifted as its main-grid copy L_dm(Hhat_s);
 *  - vhat_out = vhat_Ns (stiffly accurate tableaux).
 * vhat_in, vhat_out: device double[2][n_dual] (may alias); p_out: device
 * double[n_dof] or NULL (the last stage's pi; with opts->use_x0 its contents
 * start the first pressure solve, and every later stage starts from the
 * previous one); info: host array of 3 Ns (per stage: Helmholtz x, y,
 * Schur) or NULL.  Needs an operator built with opts.factored.
 * Synchronous.  Errors as dgsl_advdiff_step. */
int dgsl_ns_imex_step(const dgsl_operator* op, int R, double dt, double nu, const double* vhat_in,
                      double* vhat_out, double* p_out, const dgsl_solve_opts* opts,
                      dgsl_solve_info* info, void* stream);

/* ------------------------------------------------------------ advection-diffusion step */
/* One semi-Lagrangian IMEX step of the advection-diffusion model (Sec. 3 and
 * its advection-diffusion subsection; tableaux of App. A, R = 0, 1, 2):
 * dC/dt + vbar . grad C = alpha Laplacian C for a main-grid scalar C carried
 * by the steady main-grid velocity vbar.  With V_j the stage velocities of
 * the Gauss-point trajectories (as dgsl_sl_transport_imex) and the implicit
 * tableau (A, c), each stage s
 *  1. forms C^I_s = proj[C^n(x - dt sum_{j<=s} a_{s,j} V_j)
 *                        + sum_{j<s} dt a_{s,j} H_j(x - (c_s - c_j) dt V_j)]
 *     at every Gauss point x (the earlier stage fluxes taken where the
 *     characteristic was at their stage; eq. intstage projection);
 *  2. solves (Mbar + a_{s,s} dt alpha K) C*_s = Mbar C^I_s (eq. ad5, the
 *     Helmholtz system of dgsl_cg_solve, started from C^I_s);
 *  3. keeps H_s = (C*_s - C^I_s) / (a_{s,s} dt).
 * The tableaux are stiffly accurate: c_out = C*_{Ns}.  Every point is
 * reached from x along a straight segment, cell by cell.
 *  - vbar: device double[2][n_dof]; c_in, c_out: device double[n_dof]
 *    (internal order; may alias).
 *  - opts govern the Ns diffusion solves; info: host array of Ns (1, 2, 4)
 *    or NULL.
 * Synchronous.  Returns the first non-OK solve status, DGSL_ENOTCONV if a
 * segment crossed more than 65536 cells, DGSL_EINVAL for R outside 0..2,
 * dt <= 0 or alpha < 0. */
int dgsl_advdiff_step(const dgsl_operator* op, int R, double dt, double alpha, const double* vbar,
                      const double* c_in, double* c_out, const dgsl_solve_opts* opts,
                      dgsl_solve_info* info, void* stream);

/* ------------------------------------------------------------ batched engine and serving */
/* One solve request: op's Schur (coef = dt) or Helmholtz (coef = nu*dt)
 * system with n_rhs right-hand sides (0 or 1: one; at most 8): b and x device
 * double[n_rhs][n_dof] in op's internal order (caller-owned, kept alive until
 * the request completes).  tol <= 0 selects 1e-10.  The right-hand sides of a
 * request share every pass over op's couplings; each has its own refinement
 * and inner CG and gets the same result, bit for bit, as when solved alone.
 * The request's dgsl_solve_info reports the first non-OK status and the
 * largest iteration count, refinement count and relative residual over its
 * right-hand sides. */
typedef struct {
  const dgsl_operator* op;
  int32_t kind;
  int32_t n_rhs;
  double coef;
  const double* b;
  double* x;
  double tol;
} dgsl_request;

typedef struct {
  int32_t precision;        /* DGSL_PREC_F32_IR (default) or DGSL_PREC_BF16_IR */
  int32_t max_iters;        /* CG iterations per request (default 200000) */
  double inner_tol;         /* inner FP32 CG tolerance (default 1e-3) */
  int32_t max_refine;       /* refinement steps per request (default 30) */
  int32_t device;           /* CUDA device (all operators must live there) */
  int64_t hbm_budget_bytes; /* server: cap on workspace + resident operators (0 = 150e9) */
  int64_t idle_us;          /* server: how long an idle engine waits for work (default 500) */
  int32_t precond;          /* DGSL_PRECOND_* for every request (default NONE); with
                               BLOCK_JACOBI each operator keeps the couplings of A P and
                               P of its systems (see dgsl_cg_solve), counted in the budget;
                               with MULTIGRID the requests are not packed into the
                               persistent engine (a multigrid iteration is a sequence of
                               per-level launches): each runs the library's multigrid
                               solve on one of 8 worker streams, requests of different
                               operators concurrently, those of one operator in turn;
                               each operator's growth (hierarchy, workspace) is charged
                               to the budget */
  int32_t pad;
} dgsl_engine_opts;

void dgsl_default_engine_opts(dgsl_engine_opts* opts);

/* Solves n independent requests (any operators, degrees and sizes on one
 * device) in ONE persistent cooperative launch: each request runs its own FP64
 * iterative refinement around an FP32 (or BF16-coupling) Chronopoulos-Gear CG
 * (eq. pressure_final / eq. ad5), all requests advancing together with one grid
 * barrier per pass.  Results and errors per request in infos[n] (host), as for
 * dgsl_cg_solve.  Blocks until all requests finish; allocates its workspace for
 * the call.  n <= 4096.  The BF16 path needs operators built with
 * DGSL_STORE_BF16.  Returns the first non-OK request status, else DGSL_OK. */
int dgsl_cg_solve_batch(const dgsl_request* reqs, int n, const dgsl_engine_opts* opts,
                        dgsl_solve_info* infos, void* stream);

/* Serving: a request loop with continuous batching.  dgsl_submit queues a
 * request and returns at once; a scheduler thread admits queued requests while
 * their workspace plus every operator they reference fits hbm_budget_bytes,
 * publishes them to the running persistent engine (which picks them up at its
 * next pass, overlapping them with the solves already on the device) or
 * launches one, and collects completions.  The workspace arena is reserved at
 * create time, so no device allocation happens while the engine runs.
 * Errors: DGSL_EBUDGET from dgsl_submit if a request can never fit. */
typedef struct dgsl_server dgsl_server;
typedef struct {
  int64_t submitted, completed, queued, in_flight;
  int64_t engine_launches;
  int64_t bytes_in_use;     /* workspace + operators of requests in flight */
  int64_t admitted_running; /* requests published to an engine launch that was
                               already running, and admitted and finished by it
                               (continuous batching: they joined solves already
                               on the device) */
} dgsl_server_stats;

int dgsl_server_create(const dgsl_engine_opts* opts, dgsl_server** out);
int dgsl_submit(dgsl_server* srv, const dgsl_request* req, uint64_t* ticket);
/* DGSL_OK (info filled; the request's final status is info->status),
 * DGSL_EPENDING, or DGSL_EINVAL for an unknown ticket.  A ticket can be polled
 * until it is reported done once; after that it is forgotten. */
int dgsl_poll(dgsl_server* srv, uint64_t ticket, dgsl_solve_info* info);
/* Polls n tickets at once: done[i] = 1 and infos[i] filled for each ticket that
 * finished (it is then forgotten, as with dgsl_poll), done[i] = 0 if pending,
 * -1 if unknown.  Returns the number of finished tickets (>= 0) or a negative
 * status on bad arguments. */
int dgsl_poll_many(dgsl_server* srv, const uint64_t* tickets, int n, dgsl_solve_info* infos,
                   int32_t* done);
/* Removes a request that has not been admitted yet (DGSL_OK); an admitted one
 * runs to completion (DGSL_EPENDING). */
int dgsl_cancel(dgsl_server* srv, uint64_t ticket);
int dgsl_server_get_stats(dgsl_server* srv, dgsl_server_stats* out);
/* Waits for requests in flight, stops the engine and frees the server. */
void dgsl_server_destroy(dgsl_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* DGSL_H */
