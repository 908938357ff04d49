// Semi-Lagrangian trajectories and transport of dgsl (Sec. 2.5, eq. lagrtrj,
// and the Gauss-point projection of eq. intstage) on the main grid.
//
// Every quadrature point x_g of every main triangle follows its characteristic
// backward over dt in straight (Euler) pieces, one cell at a time: from x in
// triangle T, with T's DG velocity v at x, the backward ray x - s v either
// stays in T for the time left (the foot) or leaves T through the edge whose
// opposite barycentric coordinate first reaches 0; the walk moves to that
// exit point, into the neighbour's frame (a whole number of periods), and
// continues with the neighbour's velocity polynomial.  No global search.
// Where the backward rays on both sides of an edge point at it (the DG
// velocity jumps there), the walk would bounce across it forever with pieces
// of zero length: leaving a cell through the edge it entered by is allowed
// once, and a second bounce on the same edge holds the trajectory there (the
// foot is the current point, the time left is dropped).  At
// the foot the transported fields are evaluated with the polynomials of the
// triangle that contains it, and each triangle's values are projected back:
//   c*_i = Mref^-1 sum_g phi(xi_g) w_g c(x_F(x_g))      (Mbar_i = A_i Mref, |J_i| = A_i).
//
// One thread per trajectory (FP64: the walk's decisions are geometric), the
// NG = (p+1)^2 trajectories of a triangle in consecutive threads of one block,
// so the projection reads them from shared memory.  Velocity and fields are
// first converted to monomial coefficients per cell, so each step evaluates
// v by nested Horner (P(P+1)/2 + P FMAs per component).  Candidate exits are
// compared by cross-multiplication; one division per crossed edge.
#include <cmath>

#include "kernels.h"

namespace dgsl {

template <int P>
struct SLDeg {
  static constexpr int NPHI = (P + 1) * (P + 2) / 2;
  static constexpr int NG = (P + 1) * (P + 1);
  static constexpr int TPB = 128 / NG;  // triangles per block of 128 threads
};

// Value at (x, y) of sum_{i+j<=P} a_ij x^i y^j, coefficients in the order
// i = 0..P outer, j = 0..P-i inner, by nested Horner (y inside, then x):
// P(P+1)/2 + P FMAs.
template <int P>
__device__ __forceinline__ double sl_poly(const double* __restrict__ a, double x, double y) {
  double v = 0.0;
#pragma unroll
  for (int i = P; i >= 0; --i) {
    const int o = i * (P + 1) - i * (i - 1) / 2;  // offset of (i, 0)
    double r = __ldg(a + o + (P - i));
#pragma unroll
    for (int j = P - i - 1; j >= 0; --j) r = fma(r, y, __ldg(a + o + j));
    v = i == P ? r : fma(v, x, r);
  }
  return v;
}

// Nodal to monomial coefficients, a[m] = sum_k C[m][k] u[k], for nf fields of
// n values ([nf][ne][NPHI] in), written [cell][nf][NPHI] (vel: the
// components of a cell together) or [nf][ne][NPHI].
template <int NPHI>
__global__ void k_sl_mono(const double* __restrict__ in, int64_t n, int ne, int nf, const double* __restrict__ C,
                          double* __restrict__ out, int vel) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nf * ne * NPHI) return;
  const int m = (int)(t % NPHI);
  const int64_t fc = t / NPHI;
  const int f = (int)(fc / ne), cell = (int)(fc - (int64_t)f * ne);
  const double* u = in + (int64_t)f * n + (int64_t)cell * NPHI;
  double a = 0.0;
#pragma unroll
  for (int k = 0; k < NPHI; ++k) a = fma(__ldg(C + m * NPHI + k), __ldg(u + k), a);
  out[vel ? ((int64_t)cell * nf + f) * NPHI + m : ((int64_t)f * ne + cell) * NPHI + m] = a;
}

// Velocity of the walk: the cell's DG polynomial (times sgn) at (xi, eta).
template <int P>
struct SLPolyVel {
  const double* vmono;
  double sgn;
  __device__ __forceinline__ void operator()(int cell, double xi, double eta, double& vx, double& vy) const {
    constexpr int NPHI = SLDeg<P>::NPHI;
    const double* a = vmono + (int64_t)cell * 2 * NPHI;
    vx = sgn * sl_poly<P>(a, xi, eta);
    vy = sgn * sl_poly<P>(a + NPHI, xi, eta);
  }
};

// A constant velocity: the straight segment to a given point.
struct SLConstVel {
  double vx, vy;
  __device__ __forceinline__ void operator()(int, double, double, double& ox, double& oy) const {
    ox = vx;
    oy = vy;
  }
};

// The walk from (x, y) in `cell` along x - s v over the time tau (see the file
// header); on return (x, y) is the foot in the frame of `cell`.  Returns the
// cells crossed; sets *err and stops after max_steps.
template <class Vel>
__device__ __forceinline__ int sl_walk_path(const SLDev& g, double& x, double& y, int& cell, double tau, const Vel& vel,
                                            int max_steps, int* err) {
  int steps = 0, kin = -1;  // kin: local edge of `cell` the walk entered by
  bool bounced = false;     // it entered by leaving the last cell through its entry edge
  for (;;) {
    const double* C = g.tri + (int64_t)cell * 16;
    const double j00 = __ldg(C + 6), j01 = __ldg(C + 7), j10 = __ldg(C + 8), j11 = __ldg(C + 9);
    const double dx = x - __ldg(C + 0), dy = y - __ldg(C + 1);
    const double xi = fma(j00, dx, j01 * dy), eta = fma(j10, dx, j11 * dy);
    double vx, vy;
    vel(cell, xi, eta, vx, vy);
    if (vx == 0.0 && vy == 0.0) break;  // no motion: the foot is here
    const double dxi = fma(j00, vx, j01 * vy), deta = fma(j10, vx, j11 * vy);
    // barycentrics of vertices 0, 1, 2 and their rates along x - s v
    const double lam[3] = {1.0 - xi - eta, xi, eta};
    const double rate[3] = {dxi + deta, -dxi, -deta};
    int kx = -1;
    double bn = 0.0, bd = 1.0;  // exit parameter bn / bd
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int o = k == 0 ? 2 : k - 1;  // vertex opposite local edge k: (k + 2) mod 3
      if (rate[o] < 0.0) {
        const double nn = fmax(lam[o], 0.0), dd = -rate[o];
        if (kx < 0 || nn * bd < bn * dd) {
          kx = k;
          bn = nn;
          bd = dd;
        }
      }
    }
    if (kx < 0 || bn >= tau * bd) {  // the foot is in this cell
      x = fma(-tau, vx, x);
      y = fma(-tau, vy, y);
      break;
    }
    if (kx == kin && bounced) break;  // a second bounce on the same edge: held here
    const double s = bn / bd;
    x = fma(-s, vx, x) + __ldg(C + 10 + 2 * kx);
    y = fma(-s, vy, y) + __ldg(C + 11 + 2 * kx);
    tau -= s;
    bounced = kx == kin;
    kin = (__ldg(g.nbr + (int64_t)cell * 4 + 3) >> (2 * kx)) & 3;
    cell = __ldg(g.nbr + (int64_t)cell * 4 + kx);
    if (++steps > max_steps) {  // bounded walk: reported, never a hang
      atomicExch(err, 1);
      break;
    }
  }
  return steps;
}

// Reference coordinates of (x, y) (in the frame of `cell`).
__device__ __forceinline__ void sl_ref(const SLDev& g, int cell, double x, double y, double& xi, double& eta) {
  const double* C = g.tri + (int64_t)cell * 16;
  const double dx = x - __ldg(C + 0), dy = y - __ldg(C + 1);
  xi = fma(__ldg(C + 6), dx, __ldg(C + 7) * dy);
  eta = fma(__ldg(C + 8), dx, __ldg(C + 9) * dy);
}

// Outputs of one trajectory: foot, cell, steps (each optional) and the fields
// at the foot into the block's shared values.
template <int P>
__device__ __forceinline__ void sl_record(const SLDev& g, int64_t tr, double x, double y, int cell, int steps,
                                          const double* __restrict__ cmono, int nf, double (*s_val)[128],
                                          double* __restrict__ foot, int32_t* __restrict__ cellout,
                                          int32_t* __restrict__ stepsout) {
  constexpr int NPHI = SLDeg<P>::NPHI;
  double xf, yf;
  sl_ref(g, cell, x, y, xf, yf);
  if (foot) {
    foot[2 * tr] = x;
    foot[2 * tr + 1] = y;
  }
  if (cellout) cellout[tr] = cell;
  if (stepsout) stepsout[tr] = steps;
  for (int f = 0; f < nf; ++f) s_val[f][threadIdx.x] = sl_poly<P>(cmono + ((int64_t)f * g.ne + cell) * NPHI, xf, yf);
}

// eq. intstage for the block's triangles: thread (triangle, k) of the block.
template <int P>
__device__ __forceinline__ void sl_project(const SLDev& g, int64_t n, int nf, const double (*s_val)[128],
                                           double* __restrict__ cstar) {
  using D = SLDeg<P>;
  constexpr int NPHI = D::NPHI, NG = D::NG, TPB = D::TPB;
  if ((int)threadIdx.x < TPB * NPHI) {
    const int l2 = threadIdx.x / NPHI, k = threadIdx.x - l2 * NPHI;
    const int t2 = blockIdx.x * TPB + l2;
    if (t2 < g.ne)
      for (int f = 0; f < nf; ++f) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < NG; ++q) acc = fma(__ldg(g.q + k * NG + q), s_val[f][l2 * NG + q], acc);
        cstar[(int64_t)f * n + (int64_t)t2 * NPHI + k] = acc;
      }
  }
}

template <int P>
__global__ void __launch_bounds__(128) k_sl_walk(SLDev g, int64_t n, double dt, const double* __restrict__ vmono,
                                                 const double* __restrict__ cmono, int nf, double* __restrict__ cstar,
                                                 double* __restrict__ foot, int32_t* __restrict__ cellout,
                                                 int32_t* __restrict__ stepsout, int max_steps, int* err) {
  using D = SLDeg<P>;
  constexpr int NG = D::NG, TPB = D::TPB;
  __shared__ double s_val[kSLMaxFields][128];
  const int lt = threadIdx.x / NG, gq = threadIdx.x - lt * NG;
  const int ti = blockIdx.x * TPB + lt;
  if (lt < TPB && ti < g.ne) {
    const double* T = g.tri + (int64_t)ti * 16;
    const double xi0 = __ldg(g.pts + 2 * gq), eta0 = __ldg(g.pts + 2 * gq + 1);
    double x = __ldg(T + 0) + xi0 * __ldg(T + 2) + eta0 * __ldg(T + 4);
    double y = __ldg(T + 1) + xi0 * __ldg(T + 3) + eta0 * __ldg(T + 5);
    int cell = ti;
    // dt < 0: forward, the same walk with -v over |dt|
    const SLPolyVel<P> vel{vmono, dt < 0.0 ? -1.0 : 1.0};
    const int steps = sl_walk_path(g, x, y, cell, fabs(dt), vel, max_steps, err);
    sl_record<P>(g, (int64_t)ti * NG + gq, x, y, cell, steps, cmono, nf, s_val, foot, cellout, stepsout);
  }
  __syncthreads();
  sl_project<P>(g, n, nf, s_val, cstar);
}

// Stage trajectories of the explicit IMEX tableau (At, b) with NS stages:
// x^E_s = x - dt sum_{j<s} At[s][j] V_j with V_j = vbar(x^E_j), and the foot
// x_F = x - dt sum_j b_j V_j.  A point's cell does not depend on the path to
// it, so each point is reached from the previous one along the straight
// segment between them, cell by cell (the stage points of R = 2 lie at 0.44,
// 0.72 and 1 times the step: walking each one from x would cross about three
// times as many cells).
template <int P, int NS>
__global__ void __launch_bounds__(128) k_sl_stages(SLDev g, int64_t n, double dt, SLTableau tab,
                                                   const double* __restrict__ vmono, const double* __restrict__ cmono,
                                                   int nf, double* __restrict__ cstar, double* __restrict__ foot,
                                                   int32_t* __restrict__ cellout, int32_t* __restrict__ stepsout,
                                                   int max_steps, int* err, double* __restrict__ vout) {
  using D = SLDeg<P>;
  constexpr int NPHI = D::NPHI, NG = D::NG, TPB = D::TPB;
  __shared__ double s_val[kSLMaxFields][128];
  const int lt = threadIdx.x / NG, gq = threadIdx.x - lt * NG;
  const int ti = blockIdx.x * TPB + lt;
  if (lt < TPB && ti < g.ne) {
    const double* T = g.tri + (int64_t)ti * 16;
    const double xi0 = __ldg(g.pts + 2 * gq), eta0 = __ldg(g.pts + 2 * gq + 1);
    const double x0 = __ldg(T + 0) + xi0 * __ldg(T + 2) + eta0 * __ldg(T + 4);
    const double y0 = __ldg(T + 1) + xi0 * __ldg(T + 3) + eta0 * __ldg(T + 5);
    double Vx[NS], Vy[NS];
    int steps = 0;
    double x = x0, y = y0, px = 0.0, py = 0.0;  // the current point is x - dt (px, py)
    int cell = ti;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (s > 0) {
        double dx = 0.0, dy = 0.0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
          dx = fma(tab.at[s][j], Vx[j], dx);
          dy = fma(tab.at[s][j], Vy[j], dy);
        }
        // the segment to x - dt (dx, dy): the walk with the constant velocity dt (dx - px, dy - py) over time 1
        steps += sl_walk_path(g, x, y, cell, 1.0, SLConstVel{dt * (dx - px), dt * (dy - py)}, max_steps, err);
        px = dx;
        py = dy;
      }
      double xi, eta;
      sl_ref(g, cell, x, y, xi, eta);
      const double* a = vmono + (int64_t)cell * 2 * NPHI;
      Vx[s] = sl_poly<P>(a, xi, eta);
      Vy[s] = sl_poly<P>(a + NPHI, xi, eta);
      if (vout) {  // the stage velocities alone: [NS][trajectory][2]
        const int64_t o = ((int64_t)s * g.ne * NG + (int64_t)ti * NG + gq) * 2;
        vout[o] = Vx[s];
        vout[o + 1] = Vy[s];
      }
    }
    double dx = 0.0, dy = 0.0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      dx = fma(tab.b[j], Vx[j], dx);
      dy = fma(tab.b[j], Vy[j], dy);
    }
    if (!vout) {
      steps += sl_walk_path(g, x, y, cell, 1.0, SLConstVel{dt * (dx - px), dt * (dy - py)}, max_steps, err);
      sl_record<P>(g, (int64_t)ti * NG + gq, x, y, cell, steps, cmono, nf, s_val, foot, cellout, stepsout);
    }
  }
  __syncthreads();
  sl_project<P>(g, n, nf, s_val, cstar);
}

template <int P>
static cudaError_t run_sl(const SLDev& g, int64_t n, double dt, const double* vbar, const double* c, int nf,
                          double* cstar, double* foot, int32_t* cell, int32_t* steps, int max_steps, double* vmono,
                          double* cmono, int* err, cudaStream_t s) {
  using D = SLDeg<P>;
  const int64_t tv = (int64_t)2 * g.ne * D::NPHI;
  k_sl_mono<D::NPHI><<<(int)((tv + 255) / 256), 256, 0, s>>>(vbar, n, g.ne, 2, g.mono_c, vmono, 1);
  int launches = 2;
  if (nf > 0) {
    const int64_t tc = (int64_t)nf * g.ne * D::NPHI;
    k_sl_mono<D::NPHI><<<(int)((tc + 255) / 256), 256, 0, s>>>(c, n, g.ne, nf, g.mono_c, cmono, 0);
    ++launches;
  }
  k_sl_walk<P><<<(g.ne + D::TPB - 1) / D::TPB, 128, 0, s>>>(g, n, dt, vmono, cmono, nf, cstar, foot, cell, steps,
                                                            max_steps, err);
  count_launch(launches);
  return cudaGetLastError();
}

template <int P, int NS>
static cudaError_t run_sl_stages(const SLDev& g, int64_t n, double dt, const SLTableau& tab, const double* vbar,
                                 const double* c, int nf, double* cstar, double* foot, int32_t* cell, int32_t* steps,
                                 int max_steps, double* vmono, double* cmono, int* err, double* vout, cudaStream_t s) {
  using D = SLDeg<P>;
  const int64_t tv = (int64_t)2 * g.ne * D::NPHI;
  k_sl_mono<D::NPHI><<<(int)((tv + 255) / 256), 256, 0, s>>>(vbar, n, g.ne, 2, g.mono_c, vmono, 1);
  int launches = 2;
  if (nf > 0) {
    const int64_t tc = (int64_t)nf * g.ne * D::NPHI;
    k_sl_mono<D::NPHI><<<(int)((tc + 255) / 256), 256, 0, s>>>(c, n, g.ne, nf, g.mono_c, cmono, 0);
    ++launches;
  }
  k_sl_stages<P, NS><<<(g.ne + D::TPB - 1) / D::TPB, 128, 0, s>>>(g, n, dt, tab, vmono, cmono, nf, cstar, foot, cell,
                                                                  steps, max_steps, err, vout);
  count_launch(launches);
  return cudaGetLastError();
}

template <int P>
static cudaError_t run_sl_stages_p(const SLDev& g, int64_t n, double dt, const SLTableau& tab, const double* vbar,
                                   const double* c, int nf, double* cstar, double* foot, int32_t* cell,
                                   int32_t* steps, int max_steps, double* vmono, double* cmono, int* err,
                                   double* vout, cudaStream_t s) {
  switch (tab.ns) {
    case 1: return run_sl_stages<P, 1>(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, vout, s);
    case 2: return run_sl_stages<P, 2>(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, vout, s);
    case 4: return run_sl_stages<P, 4>(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, vout, s);
  }
  return cudaErrorInvalidValue;
}

// The tableaux of App. A (eq. IMEX1-IMEX3), explicit and implicit: R = 0
// Euler, R = 1 the two-stage scheme with gamma = 1 - 1/sqrt(2) and
// beta = 1/(2 gamma), R = 2 the four-stage scheme with its six printed digits.
bool sl_tableau(int R, SLTableau& t) {
  t = SLTableau{};
  if (R == 0) {
    t.ns = 1;
    t.b[0] = 1.0;
    t.ai[0][0] = 1.0;
  } else if (R == 1) {
    const double gm = 1.0 - 1.0 / std::sqrt(2.0);
    t.ns = 2;
    t.at[1][0] = 1.0 / (2.0 * gm);
    t.b[0] = 1.0 - gm;
    t.b[1] = gm;
    t.ai[0][0] = gm;
    t.ai[1][0] = 1.0 - gm;
    t.ai[1][1] = gm;
  } else if (R == 2) {
    const double gm = 0.435866;
    t.ns = 4;
    t.at[1][0] = gm;
    t.at[2][0] = 1.437745;
    t.at[2][1] = -0.719812;
    t.at[3][0] = 0.916993;
    t.at[3][1] = 0.5;
    t.at[3][2] = -0.416993;
    t.b[0] = 0.0;
    t.b[1] = 1.208496;
    t.b[2] = -0.644363;
    t.b[3] = gm;
    t.ai[0][0] = gm;
    t.ai[1][1] = gm;
    t.ai[2][1] = 0.282066;
    t.ai[2][2] = gm;
    t.ai[3][1] = 1.208496;
    t.ai[3][2] = -0.644363;
    t.ai[3][3] = gm;
  } else {
    return false;
  }
  return true;
}

static cudaError_t stages_dispatch(const SLDev& g, int64_t n, double dt, const SLTableau& tab, const double* vbar,
                                   const double* c, int nf, double* cstar, double* foot, int32_t* cell,
                                   int32_t* steps, int max_steps, double* vmono, double* cmono, int* err,
                                   double* vout, cudaStream_t s) {
  if (nf < 0 || nf > kSLMaxFields || g.ne < 1 || !vbar || (nf > 0 && (!c || !cstar || !cmono)) ||
      (tab.ns != 1 && tab.ns != 2 && tab.ns != 4))
    return cudaErrorInvalidValue;
  switch (g.p) {
    case 1: return run_sl_stages_p<1>(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, vout, s);
    case 2: return run_sl_stages_p<2>(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, vout, s);
    case 3: return run_sl_stages_p<3>(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, vout, s);
    case 4: return run_sl_stages_p<4>(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, vout, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sl_stages(const SLDev& g, int64_t n, double dt, const SLTableau& tab, const double* vbar,
                             const double* c, int nf, double* cstar, double* foot, int32_t* cell, int32_t* steps,
                             int max_steps, double* vmono, double* cmono, int* err, cudaStream_t s) {
  return stages_dispatch(g, n, dt, tab, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, nullptr,
                         s);
}

cudaError_t launch_sl_stage_velocities(const SLDev& g, int64_t n, double dt, const SLTableau& tab, const double* vbar,
                                       double* vout, double* vmono, int max_steps, int* err, cudaStream_t s) {
  if (!vout) return cudaErrorInvalidValue;
  return stages_dispatch(g, n, dt, tab, vbar, nullptr, 0, nullptr, nullptr, nullptr, nullptr, max_steps, vmono,
                         nullptr, err, vout, s);
}

// Stage s of the SL-IMEX advection-diffusion step at every Gauss point x:
//   C^n(x - dt sum_{j<=s} a_{s,j} V_j) + sum_{j<s} dt a_{s,j} H_j(x - (c_s - c_j) dt V_j),
// each point reached from x along a straight segment (fields in monomial form:
// cmono [1 + s][ne][nphi], C^n first, then H_0..H_{s-1}), projected by
// eq. intstage into ci.
template <int P>
__global__ void __launch_bounds__(128) k_sl_advdiff_stage(SLDev g, int64_t n, double dt, SLStage st,
                                                          const double* __restrict__ V,
                                                          const double* __restrict__ cmono, double* __restrict__ ci,
                                                          int max_steps, int* err) {
  using D = SLDeg<P>;
  constexpr int NPHI = D::NPHI, NG = D::NG, TPB = D::TPB;
  __shared__ double s_val[kSLMaxFields][128];
  const int lt = threadIdx.x / NG, gq = threadIdx.x - lt * NG;
  const int ti = blockIdx.x * TPB + lt;
  if (lt < TPB && ti < g.ne) {
    const double* T = g.tri + (int64_t)ti * 16;
    const double xi0 = __ldg(g.pts + 2 * gq), eta0 = __ldg(g.pts + 2 * gq + 1);
    const double x0 = __ldg(T + 0) + xi0 * __ldg(T + 2) + eta0 * __ldg(T + 4);
    const double y0 = __ldg(T + 1) + xi0 * __ldg(T + 3) + eta0 * __ldg(T + 5);
    const int64_t nt = (int64_t)g.ne * NG, tr = (int64_t)ti * NG + gq;
    double vx[4], vy[4];
    for (int j = 0; j <= st.s; ++j) {
      vx[j] = __ldg(V + 2 * (j * nt + tr));
      vy[j] = __ldg(V + 2 * (j * nt + tr) + 1);
    }
    // C^n at the implicit foot x^I_s
    double dx = 0.0, dy = 0.0;
    for (int j = 0; j <= st.s; ++j) {
      dx = fma(st.a[j], vx[j], dx);
      dy = fma(st.a[j], vy[j], dy);
    }
    double x = x0, y = y0, xi, eta;
    int cell = ti;
    sl_walk_path(g, x, y, cell, 1.0, SLConstVel{dt * dx, dt * dy}, max_steps, err);
    sl_ref(g, cell, x, y, xi, eta);
    double acc = sl_poly<P>(cmono + (int64_t)cell * NPHI, xi, eta);
    // the earlier stage fluxes, shifted along the characteristic
    for (int j = 0; j < st.s; ++j) {
      if (st.a[j] == 0.0) continue;
      const double h = st.shift[j] * dt;
      x = x0;
      y = y0;
      cell = ti;
      sl_walk_path(g, x, y, cell, 1.0, SLConstVel{h * vx[j], h * vy[j]}, max_steps, err);
      sl_ref(g, cell, x, y, xi, eta);
      acc = fma(dt * st.a[j], sl_poly<P>(cmono + ((int64_t)(1 + j) * g.ne + cell) * NPHI, xi, eta), acc);
    }
    s_val[0][threadIdx.x] = acc;
  }
  __syncthreads();
  sl_project<P>(g, n, 1, s_val, ci);
}

__global__ void k_sl_flux(const double* __restrict__ cst, const double* __restrict__ ci, double inv,
                          double* __restrict__ h, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) h[i] = (cst[i] - ci[i]) * inv;
}

// V_s of every trajectory: the two-component field (monomials vmono
// [cell][2][nphi]) at x - dt sum_{j<s} a[j] V_j, reached along the straight
// segment; V [stages][trajectory][2].
template <int P>
__global__ void __launch_bounds__(128) k_sl_stage_velocity(SLDev g, double dt, SLStage st, double* __restrict__ V,
                                                           const double* __restrict__ vmono, int max_steps, int* err) {
  using D = SLDeg<P>;
  constexpr int NPHI = D::NPHI, NG = D::NG;
  const int64_t nt = (int64_t)g.ne * NG;
  const int64_t tr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tr >= nt) return;
  const int ti = (int)(tr / NG), gq = (int)(tr - (int64_t)ti * NG);
  const double* T = g.tri + (int64_t)ti * 16;
  const double xi0 = __ldg(g.pts + 2 * gq), eta0 = __ldg(g.pts + 2 * gq + 1);
  double x = __ldg(T + 0) + xi0 * __ldg(T + 2) + eta0 * __ldg(T + 4);
  double y = __ldg(T + 1) + xi0 * __ldg(T + 3) + eta0 * __ldg(T + 5);
  double dx = 0.0, dy = 0.0;
  for (int j = 0; j < st.s; ++j) {
    dx = fma(st.a[j], V[2 * (j * nt + tr)], dx);
    dy = fma(st.a[j], V[2 * (j * nt + tr) + 1], dy);
  }
  int cell = ti;
  sl_walk_path(g, x, y, cell, 1.0, SLConstVel{dt * dx, dt * dy}, max_steps, err);
  double xi, eta;
  sl_ref(g, cell, x, y, xi, eta);
  const double* a = vmono + (int64_t)cell * 2 * NPHI;
  V[2 * (st.s * nt + tr)] = sl_poly<P>(a, xi, eta);
  V[2 * (st.s * nt + tr) + 1] = sl_poly<P>(a + NPHI, xi, eta);
}

template <int P>
static cudaError_t run_stage_velocity(const SLDev& g, int64_t fstride, double dt, const SLStage& st,
                                      const double* field2, double* V, double* vmono, int max_steps, int* err,
                                      cudaStream_t s) {
  using D = SLDeg<P>;
  const int64_t tv = (int64_t)2 * g.ne * D::NPHI;
  k_sl_mono<D::NPHI><<<(int)((tv + 255) / 256), 256, 0, s>>>(field2, fstride, g.ne, 2, g.mono_c, vmono, 1);
  const int64_t nt = (int64_t)g.ne * D::NG;
  k_sl_stage_velocity<P><<<(int)((nt + 127) / 128), 128, 0, s>>>(g, dt, st, V, vmono, max_steps, err);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_sl_stage_velocity(const SLDev& g, int64_t fstride, double dt, const SLStage& st,
                                     const double* field2, double* V, double* vmono, int max_steps, int* err,
                                     cudaStream_t s) {
  if (st.s < 0 || st.s > 3 || g.ne < 1 || !field2 || !V || !vmono) return cudaErrorInvalidValue;
  switch (g.p) {
    case 1: return run_stage_velocity<1>(g, fstride, dt, st, field2, V, vmono, max_steps, err, s);
    case 2: return run_stage_velocity<2>(g, fstride, dt, st, field2, V, vmono, max_steps, err, s);
    case 3: return run_stage_velocity<3>(g, fstride, dt, st, field2, V, vmono, max_steps, err, s);
    case 4: return run_stage_velocity<4>(g, fstride, dt, st, field2, V, vmono, max_steps, err, s);
  }
  return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t run_advdiff_stage(const SLDev& g, int64_t n, int64_t fstride, double dt, const SLStage& st,
                                     const double* V, const double* fields, double* cmono, double* ci, int max_steps,
                                     int* err, cudaStream_t s) {
  using D = SLDeg<P>;
  const int nf = 1 + st.s;
  const int64_t tc = (int64_t)nf * g.ne * D::NPHI;
  k_sl_mono<D::NPHI><<<(int)((tc + 255) / 256), 256, 0, s>>>(fields, fstride, g.ne, nf, g.mono_c, cmono, 0);
  k_sl_advdiff_stage<P><<<(g.ne + D::TPB - 1) / D::TPB, 128, 0, s>>>(g, n, dt, st, V, cmono, ci, max_steps, err);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_sl_advdiff_stage(const SLDev& g, int64_t n, int64_t fstride, double dt, const SLStage& st,
                                    const double* V, const double* fields, double* cmono, double* ci, int max_steps,
                                    int* err, cudaStream_t s) {
  if (st.s < 0 || st.s > 3 || g.ne < 1 || !V || !fields || !cmono || !ci || fstride < n) return cudaErrorInvalidValue;
  switch (g.p) {
    case 1: return run_advdiff_stage<1>(g, n, fstride, dt, st, V, fields, cmono, ci, max_steps, err, s);
    case 2: return run_advdiff_stage<2>(g, n, fstride, dt, st, V, fields, cmono, ci, max_steps, err, s);
    case 3: return run_advdiff_stage<3>(g, n, fstride, dt, st, V, fields, cmono, ci, max_steps, err, s);
    case 4: return run_advdiff_stage<4>(g, n, fstride, dt, st, V, fields, cmono, ci, max_steps, err, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sl_flux(const double* cst, const double* ci, double inv, double* h, int64_t n, cudaStream_t s) {
  k_sl_flux<<<(int)((n + 255) / 256), 256, 0, s>>>(cst, ci, inv, h, n);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_sl_transport(const SLDev& g, int64_t n, double dt, const double* vbar, const double* c, int nf,
                                double* cstar, double* foot, int32_t* cell, int32_t* steps, int max_steps,
                                double* vmono, double* cmono, int* err, cudaStream_t s) {
  if (nf < 0 || nf > kSLMaxFields || g.ne < 1 || !vbar || (nf > 0 && (!c || !cstar || !cmono)))
    return cudaErrorInvalidValue;
  switch (g.p) {
    case 1: return run_sl<1>(g, n, dt, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, s);
    case 2: return run_sl<2>(g, n, dt, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, s);
    case 3: return run_sl<3>(g, n, dt, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, s);
    case 4: return run_sl<4>(g, n, dt, vbar, c, nf, cstar, foot, cell, steps, max_steps, vmono, cmono, err, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dgsl
