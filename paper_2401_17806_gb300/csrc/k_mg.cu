// Two-level multigrid preconditioned CG (an extension: the paper runs CG
// unpreconditioned, and its iteration counts grow like 1/h).
//
// Fine level: the DG pressure space of degree p, damped block-Jacobi
// smoothing with omega_f = 0.7 (A <= 2 blockdiag(A), so the smoother
// contracts).  Coarse space: continuous piecewise-linear functions on the
// vertices, A_0 = Pc^T A Pc, solved approximately by one V(1,1)-cycle of
// smoothed aggregation (levels built on the host, mg_host.cpp).  One
// application z = M r:
//   x1 = omega_f D^-1 r;  x2 = x1 + Pc V(Pc^T (r - A x1));
//   z  = x2 + omega_f D^-1 (r - A x2).
// The outer iteration is textbook PCG (z = M r, alpha = (r, z) / (p, A p),
// beta = (r, z)_new / (r, z)_old), with the mean of A p and of z removed for
// the pressure operator (kernel span{1}).
//
// GB300 layout: the fine-level kernels stream the operator's assembled
// couplings (16-byte loads, one thread per matrix row) and keep a tile of
// TB = 128 / N_phi triangles per 128-thread CTA, so the per-triangle blocks of
// D^-1 (the interleaved layout of the block-Jacobi preconditioner) and the
// restriction to the three vertices work on shared memory.  The couplings are
// streamed twice per iteration (A p, and r - A x1); the post-smoothing residual
// r - A x2 is formed as (r - A x1) - (A Pc) e0 from 12 precomputed
// coefficients per row of A Pc.  Every reduction is
// deterministic: per-CTA partial sums, and the last CTA to arrive sums them in
// CTA order.  The coarse levels are small CSR matrices (one thread per row)
// and a dense coarsest inverse.  Scalars live in device memory, so an
// iteration is a fixed sequence of launches that the host replays without
// reading anything back; the host checks convergence every few iterations,
// and a finished solve turns the remaining launches into early returns.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "kassembled.cuh"
#include "mg.h"

namespace dgsl {

constexpr int kMGThreads = 128;
constexpr double kOmegaF = 0.7;
constexpr int kMGBatch = 4;  // PCG iterations launched between host checks (even)

struct MGRed {
  unsigned int count;
  unsigned int pad[31];
  double out[8];
};

struct MGState {
  double rz[2];  // (r, z) of the current direction, double-buffered by iteration parity
  double rr0, rr;
  double stop2;
  int it, done, max_iters, status;
};

struct MGFine {
  const void* vals;    // couplings of the PCG matvec (the operator solved)
  const void* svals;   // couplings of the smoother residuals (BF16 for type 2)
  const int32_t* cols;
  int ne_pad, ne;
  int64_t n;
  const double* area;
  const double* Mref;
  double coefK, coefM;
  int mean_zero;
  const void* dinv;
  const int32_t* cvid;
};

// Barycentric coordinates of node k (b-major then a; node (a/p, b/p)).
template <int NPHI, typename V>
__device__ __forceinline__ void node_lam(int k, V (&l)[3]) {
  constexpr int P = NPHI == 3 ? 1 : NPHI == 6 ? 2 : NPHI == 10 ? 3 : 4;
  int b = 0;
  while (k > P - b) {
    k -= P - b + 1;
    ++b;
  }
  l[1] = (V)k / (V)P;
  l[2] = (V)b / (V)P;
  l[0] = V(1) - l[1] - l[2];
}

// Deterministic grid-wide sum of v[0..NW): CTA sums in thread order, per-CTA
// partials, then the last CTA to arrive sums them in CTA order into red->out.
template <int NW>
__device__ __forceinline__ void grid_reduce(double (&v)[NW], double* part, MGRed* red) {
  __shared__ int s_last;
  block_sum<NW>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NW; ++i) part[(size_t)blockIdx.x * NW + i] = v[i];
    __threadfence();
    const unsigned t = atomicAdd(&red->count, 1u);
    s_last = t == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double tot[NW];
    sum_partials<NW>(part, (int)gridDim.x, tot);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < NW; ++i) red->out[i] = tot[i];
      red->count = 0;
      __threadfence();
    }
  }
}

// Row of A x (difference form) with the coupled blocks gathered straight from
// global memory (L1 / L2): staging a tile's blocks in shared memory first was
// measured slower here (the extra CTA barriers per tile cost more than the
// repeated loads).  x is always one of the system's own vectors (allocated
// here, so aligned): for even N_phi the blocks are read two values per load.
template <int NPHI, typename T, typename V>
__device__ __forceinline__ V mg_row(const void* vals, const MGFine& f, int64_t row, const V* x) {
  V y = (V)f.coefK * assembled_row<NPHI, T, V, false, DiffForm<T>::value, NPHI % 2 == 0>(
                         static_cast<const T*>(vals), f.cols, f.ne_pad, f.n, row, x);
  if (f.coefM != 0.0) y += (V)f.coefM * mass_row<NPHI, V, false>(f.area, f.Mref, row, x);
  return y;
}

// omega_f (D^-1 s)_row for the row's triangle block held in s (N_phi values).
template <int NPHI, typename V>
__device__ __forceinline__ V mg_bj(const MGFine& f, int64_t row, const V* s) {
  constexpr int VP = 16 / (int)sizeof(V);
  const V* d = static_cast<const V*>(f.dinv);
  V acc = V(0);
#pragma unroll
  for (int l = 0; l < NPHI; ++l) acc = fma(__ldg(d + ((int64_t)(l / VP) * f.n + row) * VP + l % VP), s[l], acc);
  return (V)kOmegaF * acc;
}

// q = A p; reduction (p.q, sum q, sum p)
template <int NPHI, typename T, typename V>
__global__ void __launch_bounds__(kMGThreads) k_mg_matvec(MGFine f, const V* __restrict__ p, V* __restrict__ q,
                                                         double* part, MGRed* red, const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  constexpr int TB = kMGThreads / NPHI, ROWS = TB * NPHI;
  const int ntile = (f.ne + TB - 1) / TB;
  V a0 = V(0), a1 = V(0), a2 = V(0);
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t row = (int64_t)tile * ROWS + threadIdx.x;
    if (threadIdx.x < ROWS && row < f.n) {
      const V y = mg_row<NPHI, T, V>(f.vals, f, row, p);
      q[row] = y;
      const V pv = p[row];
      a0 = fma(pv, y, a0);
      a1 += y;
      a2 += pv;
    }
  }
  double v[3] = {(double)a0, (double)a1, (double)a2};
  grid_reduce<3>(v, part, red);
}

// INIT: r = b, x = 0; else x += alpha p, r -= alpha (q - mean q).  Then
// x1 = omega_f D^-1 r; reduction (r.r, sum r).
template <int NPHI, typename V, bool INIT>
__global__ void __launch_bounds__(kMGThreads) k_mg_update(MGFine f, const V* __restrict__ b, const V* __restrict__ p,
                                                         const V* __restrict__ q, V* __restrict__ x, V* __restrict__ r,
                                                         V* __restrict__ x1, const MGRed* red_mv, const MGState* st,
                                                         int par, double* part, MGRed* red) {
  if (*((volatile const int*)&st->done)) return;
  constexpr int TB = kMGThreads / NPHI, ROWS = TB * NPHI;
  __shared__ V s_r[kMGThreads];
  __shared__ V s_sc[2];
  if (!INIT && threadIdx.x == 0) {  // scalars once per CTA (an FP64 division per thread is slow here)
    const double mq = f.mean_zero ? red_mv->out[1] / (double)f.n : 0.0;
    const double pq = red_mv->out[0] - mq * red_mv->out[2];
    s_sc[0] = (V)(st->rz[par] / pq);
    s_sc[1] = (V)mq;
  }
  __syncthreads();
  const V alpha = INIT ? V(0) : s_sc[0];
  const V mu_q = INIT ? V(0) : s_sc[1];
  const int ntile = (f.ne + TB - 1) / TB;
  V a0 = V(0), a1 = V(0);
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t row = (int64_t)tile * ROWS + threadIdx.x;
    const bool act = threadIdx.x < ROWS && row < f.n;
    V rv = V(0);
    if (act) {
      if (INIT) {
        rv = b[row];
        x[row] = V(0);
      } else {
        x[row] = fma(alpha, p[row], x[row]);
        rv = r[row] - alpha * (q[row] - mu_q);
      }
      r[row] = rv;
      a0 = fma(rv, rv, a0);
      a1 += rv;
    }
    s_r[threadIdx.x] = rv;
    __syncthreads();
    if (act) x1[row] = mg_bj<NPHI, V>(f, row, s_r + (threadIdx.x / NPHI) * NPHI);
    __syncthreads();
  }
  double v[2] = {(double)a0, (double)a1};
  grid_reduce<2>(v, part, red);
}

// t1 = r - A x1 (kept for the post-smoothing) and w[t][m] = sum_k
// lambda_m(xi_k) t1_(t, k): the residual restricted to each triangle's
// vertices.
template <int NPHI, typename T, typename V>
__global__ void __launch_bounds__(kMGThreads) k_mg_resid_restrict(MGFine f, const V* __restrict__ r,
                                                                 const V* __restrict__ x1, V* __restrict__ w,
                                                                 V* __restrict__ t1, const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  constexpr int TB = kMGThreads / NPHI, ROWS = TB * NPHI;
  __shared__ V s_t[kMGThreads];
  const int ntile = (f.ne + TB - 1) / TB;
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t row = (int64_t)tile * ROWS + threadIdx.x;
    V tv = V(0);
    if (threadIdx.x < ROWS && row < f.n) {
      tv = r[row] - mg_row<NPHI, T, V>(f.svals, f, row, x1);
      t1[row] = tv;
    }
    s_t[threadIdx.x] = tv;
    __syncthreads();
    if (threadIdx.x < 3 * TB) {
      const int lt = threadIdx.x / 3, m = threadIdx.x % 3;
      const int tri = tile * TB + lt;
      if (tri < f.ne) {
        V acc = V(0);
#pragma unroll
        for (int k = 0; k < NPHI; ++k) {
          V l[3];
          node_lam<NPHI, V>(k, l);
          acc = fma(l[m], s_t[lt * NPHI + k], acc);
        }
        w[(size_t)tri * 3 + m] = acc;
      }
    }
    __syncthreads();
  }
}

// b0[v] = sum of w over the (triangle, vertex) incidences of vertex v (Pc^T t).
template <typename V>
__global__ void k_mg_vgather(int nv, const int32_t* __restrict__ ptr, const int32_t* __restrict__ inc,
                             const V* __restrict__ w, V* __restrict__ b0, const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  V acc = V(0);
  for (int k = ptr[v]; k < ptr[v + 1]; ++k) acc += w[inc[k]];
  b0[v] = acc;
}

// ---- coarse levels (CSR, one thread per row)
// init + sum_k av[k] (s[ci[k]] x[ci[k]]) (SCALE) or init + sum_k av[k] x[ci[k]]
// over k in [k0, k1), accumulated in k order.  The loads of four entries are issued
// before their products, so a row costs one dependent load chain per four
// entries instead of one per entry (the coarse levels are latency-bound).
template <typename V, bool SCALE>
__device__ __forceinline__ V csr_dot(const int32_t* __restrict__ ci, const V* __restrict__ av,
                                     const V* __restrict__ s, const V* x, int k0, int k1, V init = V(0)) {
  V acc = init;
  int k = k0;
  for (; k + 4 <= k1; k += 4) {
    int j[4];
    V a[4], v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) j[u] = ci[k + u];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = av[k + u];
      v[u] = SCALE ? s[j[u]] * x[j[u]] : x[j[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc = fma(a[u], v[u], acc);
  }
  for (; k < k1; ++k) {
    const int jj = ci[k];
    acc = fma(av[k], SCALE ? s[jj] * x[jj] : x[jj], acc);
  }
  return acc;
}

// x = wd b;  t = b - A (wd b)
template <typename V>
__global__ void k_csr_smooth0(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const V* __restrict__ av, const V* __restrict__ wd, const V* __restrict__ b,
                              V* __restrict__ x, V* __restrict__ t, const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V acc = csr_dot<V, true>(ci, av, wd, b, rp[i], rp[i + 1]);
  x[i] = wd[i] * b[i];
  t[i] = b[i] - acc;
}
// sum_k mv[k] x[ci[k]] over k in [k0, k1) by one warp (lane-strided partial
// sums, then a fixed shuffle tree: a deterministic order); lane 0 holds it.
template <typename V>
__device__ __forceinline__ V warp_dot(const int32_t* __restrict__ ci, const V* __restrict__ mv, const V* x, int k0,
                                      int k1, int lane) {
  V acc = V(0);
  for (int k = k0 + lane; k < k1; k += 32) acc = fma(mv[k], ci ? x[ci[k]] : x[k - k0], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  return acc;
}

// y = M x with one warp per row (the restriction's rows are long: an
// aggregate's DOFs and their neighbours)
template <typename V>
__global__ void k_csr_spmv_warp(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const V* __restrict__ mv, const V* __restrict__ x, V* __restrict__ y,
                                const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  const V acc = warp_dot<V>(ci, mv, x, rp[i], rp[i + 1], lane);
  if (lane == 0) y[i] = acc;
}

// x += P e
template <typename V>
__global__ void k_csr_prolong_add(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                  const V* __restrict__ pv, const V* __restrict__ e, V* __restrict__ x,
                                  const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = csr_dot<V, false>(ci, pv, nullptr, e, rp[i], rp[i + 1], x[i]);
}
// y = x + wd (b - A x)
template <typename V>
__global__ void k_csr_smooth1(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const V* __restrict__ av, const V* __restrict__ wd, const V* __restrict__ b,
                              const V* __restrict__ x, V* __restrict__ y, const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V acc = csr_dot<V, false>(ci, av, nullptr, x, rp[i], rp[i + 1]);
  y[i] = fma(wd[i], b[i] - acc, x[i]);
}
// x = C b (dense coarsest inverse, row-major nc x nc; one CTA)
// Device view of one coarse level (pointers into MGSys's arrays).
template <typename V>
struct MGLevelView {
  int n, nnext;
  const int32_t *Arp, *Aci, *Prp, *Pci, *Rrp, *Rci;
  const V *Av, *wd, *Pv, *Rv;
  V *b, *x, *t, *y;
};

// Levels this small run inside one CTA (always the dense coarsest level).  The
// CSR gathers of a level go through one SM's L1/L2 path there: a level of
// 7,637 rows (256^2 mesh, level 1) took ~220 us against ~15 us in the grid
// kernels, and one of 904 rows (level 2) still ~45 us against ~25 us.
constexpr int kTailRows = 256;
constexpr int kTailThreads = 1024;

// The V-cycle from level l0 (right-hand side in its b) down to the dense
// coarsest level and back, in ONE CTA (__syncthreads between the steps): the
// same steps as the per-level kernels, for the levels too small to fill the
// GPU, where a launch per step would cost more than its work.  The solution
// of level l0 ends in its y (in x when l0 is the coarsest).
template <typename V>
__global__ void __launch_bounds__(kTailThreads) k_coarse_tail(const MGLevelView<V>* __restrict__ lv, int l0, int L,
                                                             const V* __restrict__ C, const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31), nwarp = (int)(blockDim.x >> 5);
  for (int l = l0; l + 1 < L; ++l) {
    const MGLevelView<V> D = lv[l];
    for (int i = threadIdx.x; i < D.n; i += blockDim.x) {
      const V acc = csr_dot<V, true>(D.Aci, D.Av, D.wd, D.b, D.Arp[i], D.Arp[i + 1]);
      D.x[i] = D.wd[i] * D.b[i];
      D.t[i] = D.b[i] - acc;
    }
    __syncthreads();
    // the restriction's rows are long (an aggregate's DOFs and their
    // neighbours): one warp per row, as k_csr_spmv_warp
    V* bn = lv[l + 1].b;
    for (int i = warp; i < D.nnext; i += nwarp) {
      const V acc = warp_dot<V>(D.Rci, D.Rv, D.t, D.Rrp[i], D.Rrp[i + 1], lane);
      if (lane == 0) bn[i] = acc;
    }
    __syncthreads();
  }
  {
    // dense coarsest solve, one warp per row of C (exactly symmetric: row i
    // holds column i, read contiguously)
    const MGLevelView<V> Z = lv[L - 1];
    for (int i = warp; i < Z.n; i += nwarp) {
      const V acc = warp_dot<V>(nullptr, C + (size_t)i * Z.n, Z.b, 0, Z.n, lane);
      if (lane == 0) Z.x[i] = acc;
    }
    __syncthreads();
  }
  for (int l = L - 2; l >= l0; --l) {
    const MGLevelView<V> D = lv[l];
    const V* sol = l + 1 == L - 1 ? lv[l + 1].x : lv[l + 1].y;
    for (int i = threadIdx.x; i < D.n; i += blockDim.x)
      D.x[i] = csr_dot<V, false>(D.Pci, D.Pv, nullptr, sol, D.Prp[i], D.Prp[i + 1], D.x[i]);
    __syncthreads();
    for (int i = threadIdx.x; i < D.n; i += blockDim.x) {
      const V acc = csr_dot<V, false>(D.Aci, D.Av, nullptr, D.x, D.Arp[i], D.Arp[i + 1]);
      D.y[i] = fma(D.wd[i], D.b[i] - acc, D.x[i]);
    }
    __syncthreads();
  }
}

// One coupling of the smoother's operator as FP64: row `row`, slot c (block
// c / N_phi, node c % N_phi) of the interleaved layout.
template <typename T>
__device__ __forceinline__ double coupling_at(const T* vals, int64_t n, int64_t row, int c) {
  constexpr int VEC = 16 / (int)sizeof(T);
  const T v = vals[((int64_t)(c / VEC) * n + row) * VEC + c % VEC];
  if constexpr (sizeof(T) == 2)
    return (double)__uint_as_float((unsigned)v << 16);
  else
    return (double)v;
}

// beta[row][b][m] = coefK sum_kk K_eff[row][(b, kk)] lambda_m(xi_kk): the
// stiffness part of A Pc, row by row (b = 0 the own triangle, 1..3 the
// neighbours, m their vertices).  K_eff is the difference form of the
// smoother's couplings (off-diagonal a_c, diagonal -sum a_c), so each row of
// beta sums to zero and is applied as sum beta (e0_v - (Pc e0)_row).  Layout
// [12 / VP][n][VP] with VP values of V per 16 bytes.  FP64 arithmetic.
template <int NPHI, typename TS, typename V>
__global__ void k_mg_beta(const TS* __restrict__ vals, int64_t n, double coefK, V* __restrict__ beta) {
  constexpr int VP = 16 / (int)sizeof(V);
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int k = (int)(row % NPHI);
  double bt[12] = {};
  double rs = 0.0;
  for (int c = 0; c < 4 * NPHI; ++c) {
    const int b = c / NPHI, kk = c % NPHI;
    if (b == 0 && kk == k) continue;  // the self slot: (x_row - x_row) in the difference form
    const double a = coupling_at<TS>(vals, n, row, c);
    double l[3];
    node_lam<NPHI, double>(kk, l);
    for (int m = 0; m < 3; ++m) bt[b * 3 + m] += a * l[m];
    rs += a;
  }
  double lk[3];
  node_lam<NPHI, double>(k, lk);
  for (int m = 0; m < 3; ++m) bt[m] -= rs * lk[m];
  for (int q = 0; q < 12; ++q) beta[((int64_t)(q / VP) * n + row) * VP + q % VP] = (V)(coefK * bt[q]);
}

// Post-smoothing from the pre-smoothing residual: with x2 = x1 + Pc e0,
// r - A x2 = t1 - (A Pc) e0, and (A Pc) e0 = sum_(b, m) beta (e0_v - pe)
// (+ coefM A_t sum_kk Mref[k][kk] (Pc e0)_kk for the Helmholtz mass term),
// pe = (Pc e0)_row.  Then z = x2 + omega_f D^-1 (r - A x2); reduction (r.z,
// sum z).  This reads 12 coefficients per row instead of the row's 4 N_phi
// couplings and needs no x2 vector.
template <int NPHI, typename V>
__global__ void __launch_bounds__(kMGThreads) k_mg_post(MGFine f, const V* __restrict__ r, const V* __restrict__ x1,
                                                       const V* __restrict__ t1, const V* __restrict__ e0,
                                                       const V* __restrict__ beta, V* __restrict__ z, double* part,
                                                       MGRed* red, const MGState* st) {
  if (*((volatile const int*)&st->done)) return;
  constexpr int TB = kMGThreads / NPHI, ROWS = TB * NPHI;
  constexpr int VP = 16 / (int)sizeof(V);
  __shared__ V s_t[kMGThreads];
  const int ntile = (f.ne + TB - 1) / TB;
  V a0 = V(0), a1 = V(0);
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t row = (int64_t)tile * ROWS + threadIdx.x;
    const bool act = threadIdx.x < ROWS && row < f.n;
    V rv = V(0), tv = V(0), x2v = V(0);
    if (act) {
      const int tri = (int)(row / NPHI), k = (int)(row - (int64_t)tri * NPHI);
      V lk[3];
      node_lam<NPHI, V>(k, lk);
      V ev[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) ev[m] = e0[__ldg(f.cvid + (size_t)tri * 3 + m)];
      V pe = V(0);
#pragma unroll
      for (int m = 0; m < 3; ++m) pe = fma(lk[m], ev[m], pe);
      x2v = x1[row] + pe;
      V bt[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) bt[q] = __ldg(beta + ((int64_t)(q / VP) * f.n + row) * VP + q % VP);
      V apc = V(0);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int cb = b == 0 ? tri : __ldg(f.cols + (size_t)b * f.ne_pad + tri);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const V e = b == 0 ? ev[m] : e0[__ldg(f.cvid + (size_t)cb * 3 + m)];
          apc = fma(bt[b * 3 + m], e - pe, apc);
        }
      }
      if (f.coefM != 0.0) {
        V ml[3] = {V(0), V(0), V(0)};
#pragma unroll
        for (int kk = 0; kk < NPHI; ++kk) {
          V l[3];
          node_lam<NPHI, V>(kk, l);
          const V mr = (V)__ldg(f.Mref + k * NPHI + kk);
#pragma unroll
          for (int m = 0; m < 3; ++m) ml[m] = fma(mr, l[m], ml[m]);
        }
        V mp = V(0);
#pragma unroll
        for (int m = 0; m < 3; ++m) mp = fma(ml[m], ev[m], mp);
        apc = fma((V)(f.coefM * __ldg(f.area + tri)), mp, apc);
      }
      rv = r[row];
      tv = t1[row] - apc;
    }
    s_t[threadIdx.x] = tv;
    __syncthreads();
    if (act) {
      const V zv = x2v + mg_bj<NPHI, V>(f, row, s_t + (threadIdx.x / NPHI) * NPHI);
      z[row] = zv;
      a0 = fma(rv, zv, a0);
      a1 += zv;
    }
    __syncthreads();
  }
  double v[2] = {(double)a0, (double)a1};
  grid_reduce<2>(v, part, red);
}

// p = (z - mean z) + beta p with beta = (r, z)_new / (r, z)_old (FIRST: beta
// = 0); the convergence test; state by CTA 0.
template <typename V, bool FIRST>
__global__ void k_mg_dir(int64_t n, int mean_zero, const V* __restrict__ z, V* __restrict__ p, const MGRed* red_up,
                         const MGRed* red_post, MGState* st, int par) {
  if (*((volatile const int*)&st->done)) return;
  __shared__ double s_sc[4];
  if (threadIdx.x == 0) {  // scalars once per CTA (an FP64 division per thread is slow here)
    const double rr = red_up->out[0], sr = red_up->out[1];
    const double mz = mean_zero ? red_post->out[1] / (double)n : 0.0;
    const double rz = red_post->out[0] - mz * sr;
    s_sc[0] = rr;
    s_sc[1] = mz;
    s_sc[2] = rz;
    s_sc[3] = FIRST ? 0.0 : rz / st->rz[par];
  }
  __syncthreads();
  const double rr = s_sc[0], rz = s_sc[2];
  const V mzv = (V)s_sc[1], bv = (V)s_sc[3];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = FIRST ? z[i] - mzv : fma(bv, p[i], z[i] - mzv);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int it = st->it;
    double rr0 = st->rr0;
    if (FIRST) {
      rr0 = rr;
      st->rr0 = rr;
    } else {
      st->it = ++it;
    }
    st->rr = rr;
    st->rz[par ^ 1] = rz;
    const bool bad = !(rz > 0.0) || !isfinite(rz);
    if (bad && rr > 0.0) st->status = 1;
    if (rr <= st->stop2 * rr0 || it >= st->max_iters || bad) st->done = 1;
  }
}

// ---- topology: reduced couplings of every triangle block (FP64)
// Kr[t][b][m][m'] = sum_k,l lambda_m(k) K_(t, b)[k][l] lambda_m'(l); b = 0 also
// Mr[t][m][m'] = A_t sum_k,l lambda_m(k) Mref[k][l] lambda_m'(l).
template <int NPHI>
__global__ void k_mg_reduce(const double* __restrict__ K64, const double* __restrict__ area,
                            const double* __restrict__ Mref, int ne, int64_t n, double* __restrict__ Kr,
                            double* __restrict__ Mr) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 4 * (int64_t)ne) return;
  const int t = (int)(id / 4), b = (int)(id % 4);
  double acc[3][3] = {}, macc[3][3] = {};
  for (int k = 0; k < NPHI; ++k) {
    double lk[3];
    node_lam<NPHI, double>(k, lk);
    const int64_t row = (int64_t)t * NPHI + k;
    for (int l = 0; l < NPHI; ++l) {
      double ll[3];
      node_lam<NPHI, double>(l, ll);
      const int c = b * NPHI + l;
      const double kv = K64[((int64_t)(c / 2) * n + row) * 2 + c % 2];
      const double mv = b == 0 ? Mref[k * NPHI + l] : 0.0;
      for (int m = 0; m < 3; ++m)
        for (int q = 0; q < 3; ++q) {
          acc[m][q] += lk[m] * kv * ll[q];
          macc[m][q] += lk[m] * mv * ll[q];
        }
    }
  }
  for (int m = 0; m < 3; ++m)
    for (int q = 0; q < 3; ++q) Kr[(size_t)id * 9 + m * 3 + q] = acc[m][q];
  if (b == 0)
    for (int m = 0; m < 3; ++m)
      for (int q = 0; q < 3; ++q) Mr[(size_t)t * 9 + m * 3 + q] = area[t] * macc[m][q];
}

// ------------------------------------------------------------ host side
namespace {

template <class X>
X* mg_alloc(std::vector<void*>& allocs, int64_t& bytes, size_t count) {
  void* p = nullptr;
  const size_t b = std::max<size_t>(count * sizeof(X), 16);
  cudaError_t e = cudaMalloc(&p, b);
  if (e != cudaSuccess) throw Error(DGSL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  allocs.push_back(p);
  bytes += (int64_t)b;
  return static_cast<X*>(p);
}

void check(cudaError_t e) {
  if (e != cudaSuccess) throw Error(DGSL_ECUDA, cudaGetErrorString(e));
}

// CTAs per SM of the fine-level kernels: as many as all four stay resident
// with (the occupancy of the kernels themselves, by degree and type).  The
// kernels are latency-bound (long-scoreboard stalls on the coupled blocks), so
// resident warps are what they need: at 1024^2, p = 4, 12 CTAs per SM ran an
// iteration in 6.38 ms against 7.92 ms at 8 (256^2, p = 3: 384 against 388
// us).  The number depends on the device and the system only, so the order of
// the deterministic reductions, and the bits, are the same in every run.
// DGSL_MG_CTAS_PER_SM (1..16) overrides it, for sweeps.
template <int NPHI, typename TK, typename TS, typename V>
int fine_occupancy() {
  int o[4] = {0, 0, 0, 0};
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], k_mg_matvec<NPHI, TK, V>, kMGThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], k_mg_update<NPHI, V, false>, kMGThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[2], k_mg_resid_restrict<NPHI, TS, V>, kMGThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[3], k_mg_post<NPHI, V>, kMGThreads, 0);
  return std::max(1, std::min(std::min(o[0], o[1]), std::min(o[2], o[3])));
}

template <typename TK, typename TS, typename V>
int fine_occupancy(int nphi) {
  switch (nphi) {
    case 3: return fine_occupancy<3, TK, TS, V>();
    case 6: return fine_occupancy<6, TK, TS, V>();
    case 10: return fine_occupancy<10, TK, TS, V>();
    default: return fine_occupancy<15, TK, TS, V>();
  }
}

template <typename TS, typename V>
cudaError_t launch_beta_t(const DevOp& d, const void* vals, double coefK, void* beta, cudaStream_t s) {
  const unsigned g = (unsigned)((d.n + 255) / 256);
  const TS* tv = static_cast<const TS*>(vals);
  V* bv = static_cast<V*>(beta);
  switch (d.nphi) {
    case 3: k_mg_beta<3, TS, V><<<g, 256, 0, s>>>(tv, d.n, coefK, bv); break;
    case 6: k_mg_beta<6, TS, V><<<g, 256, 0, s>>>(tv, d.n, coefK, bv); break;
    case 10: k_mg_beta<10, TS, V><<<g, 256, 0, s>>>(tv, d.n, coefK, bv); break;
    default: k_mg_beta<15, TS, V><<<g, 256, 0, s>>>(tv, d.n, coefK, bv); break;
  }
  count_launch();
  return cudaGetLastError();
}

// beta from the couplings the smoother applies (BF16 for type 2, FP32 for
// type 0, FP64 for type 1), so the pre- and post-smoothing use one operator
cudaError_t launch_beta(const DevOp& d, int type, double coefK, void* beta, cudaStream_t s) {
  if (type == 1) return launch_beta_t<double, double>(d, d.K64, coefK, beta, s);
  if (type == 2) return launch_beta_t<uint16_t, float>(d, d.K16, coefK, beta, s);
  return launch_beta_t<float, float>(d, d.K32, coefK, beta, s);
}

int mg_ctas_per_sm(int nphi, int type) {
  if (const char* e = std::getenv("DGSL_MG_CTAS_PER_SM")) {
    const int v = std::atoi(e);
    if (v >= 1 && v <= 16) return v;
  }
  if (type == 1) return fine_occupancy<double, double, double>(nphi);
  if (type == 2) return fine_occupancy<float, uint16_t, float>(nphi);
  return fine_occupancy<float, float, float>(nphi);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

}  // namespace

MGTopo::~MGTopo() {
  cudaFree(d_cvid);
  cudaFree(d_v2t_ptr);
  cudaFree(d_v2t);
}

std::unique_ptr<MGTopo> mg_topo_build(const HostMesh& hm, const DevOp& d, cudaStream_t s) {
  auto tp = std::make_unique<MGTopo>();
  MGTopo& t = *tp;
  mg_vertex_numbering(hm, t.mg);
  // internal neighbours from the device column table
  std::vector<int32_t> cols((size_t)4 * d.ne_pad);
  check(cudaMemcpyAsync(cols.data(), d.cols, cols.size() * 4, cudaMemcpyDeviceToHost, s));
  double* kr = nullptr;
  double* mr = nullptr;
  check(cudaMalloc(&kr, (size_t)d.ne * 36 * sizeof(double)));
  check(cudaMalloc(&mr, (size_t)d.ne * 9 * sizeof(double)));
  const int g = (int)((4 * (int64_t)d.ne + 127) / 128);
  switch (d.nphi) {
    case 3: k_mg_reduce<3><<<g, 128, 0, s>>>(d.K64, d.area, d.Mref, d.ne, d.n, kr, mr); break;
    case 6: k_mg_reduce<6><<<g, 128, 0, s>>>(d.K64, d.area, d.Mref, d.ne, d.n, kr, mr); break;
    case 10: k_mg_reduce<10><<<g, 128, 0, s>>>(d.K64, d.area, d.Mref, d.ne, d.n, kr, mr); break;
    case 15: k_mg_reduce<15><<<g, 128, 0, s>>>(d.K64, d.area, d.Mref, d.ne, d.n, kr, mr); break;
    default: throw Error(DGSL_EINVAL, "multigrid: bad degree");
  }
  count_launch();
  t.Kr.resize((size_t)d.ne * 36);
  t.Mr.resize((size_t)d.ne * 9);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(t.Kr.data(), kr, t.Kr.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t.Mr.data(), mr, t.Mr.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(kr);
  cudaFree(mr);
  check(e);
  t.nbr.resize((size_t)d.ne * 3);
  for (int i = 0; i < d.ne; ++i)
    for (int b = 1; b < 4; ++b) t.nbr[(size_t)i * 3 + b - 1] = cols[(size_t)b * d.ne_pad + i];
  t.pattern = mg_coarse_pattern(t.mg, d.ne, t.nbr);
  t.graph = mg_vertex_graph(t.mg, d.ne);
  std::vector<void*> tmp;
  t.d_cvid = mg_alloc<int32_t>(tmp, t.device_bytes, t.mg.cvid.size());
  t.d_v2t_ptr = mg_alloc<int32_t>(tmp, t.device_bytes, t.mg.v2t_ptr.size());
  t.d_v2t = mg_alloc<int32_t>(tmp, t.device_bytes, t.mg.v2t.size());
  check(cudaMemcpyAsync(t.d_cvid, t.mg.cvid.data(), t.mg.cvid.size() * 4, cudaMemcpyHostToDevice, s));
  check(cudaMemcpyAsync(t.d_v2t_ptr, t.mg.v2t_ptr.data(), t.mg.v2t_ptr.size() * 4, cudaMemcpyHostToDevice, s));
  check(cudaMemcpyAsync(t.d_v2t, t.mg.v2t.data(), t.mg.v2t.size() * 4, cudaMemcpyHostToDevice, s));
  check(cudaStreamSynchronize(s));
  return tp;
}

// Device data of one level below the vertex level's solve.
template <typename V>
struct MGLevelD {
  int n = 0, nnext = 0;
  int32_t *Arp = nullptr, *Aci = nullptr, *Prp = nullptr, *Pci = nullptr, *Rrp = nullptr, *Rci = nullptr;
  V *Av = nullptr, *wd = nullptr, *Pv = nullptr, *Rv = nullptr;
  V *b = nullptr, *x = nullptr, *t = nullptr, *y = nullptr;
};

struct MGSys {
  int type = 0;
  bool singular = false;
  double coefK = 0.0, coefM = 0.0;
  MGHost host;                 // levels (FP64) and numbering
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int grid = 0;                // CTAs of the fine-level kernels
  // fine level (vector type V: float for types 0 and 2, double for 1)
  void* dinv = nullptr;
  void *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x1 = nullptr, *t1 = nullptr, *w = nullptr;
  void* beta = nullptr;        // [12 / VP][n][VP]: the stiffness part of A Pc (k_mg_beta)
  double* part = nullptr;      // [grid][3]
  MGRed* red = nullptr;        // [3]: matvec, update, post
  MGState* st = nullptr;
  MGState* h_st = nullptr;     // pinned
  const int32_t* cvid = nullptr;
  const int32_t* v2t_ptr = nullptr;
  const int32_t* v2t = nullptr;
  std::vector<MGLevelD<float>> lf;
  std::vector<MGLevelD<double>> ld;
  void* C = nullptr;
  void* views = nullptr;       // MGLevelView<V>[levels] on the device
  int tail = 0;                // first level run by k_coarse_tail
  // kMGBatch PCG iterations captured once as a CUDA graph (on a private
  // stream: the caller's may be the legacy stream, which cannot capture) and
  // replayed on the caller's stream; it writes the solution vector exec_x
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* exec_x = nullptr;
  int exec_kernels = 0;
  ~MGSys() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    for (void* a : allocs) cudaFree(a);
    if (h_st) cudaFreeHost(h_st);
  }
};

void MGSysDeleter::operator()(MGSys* p) const { delete p; }
int64_t mg_sys_bytes(const MGSys* m) { return m ? m->bytes : 0; }
const MGHost& mg_sys_host(const MGSys* m) { return m->host; }
int mg_sys_levels(const MGSys* m, std::vector<int>* sizes) {
  if (sizes) {
    sizes->clear();
    for (const auto& L : m->host.lv) sizes->push_back(L.A.n);
  }
  return (int)m->host.lv.size();
}

namespace {

template <typename V>
std::vector<V> cast(const std::vector<double>& a) {
  return std::vector<V>(a.begin(), a.end());
}

template <typename X>
X* upload(MGSys& m, const std::vector<X>& v, cudaStream_t s) {
  X* p = mg_alloc<X>(m.allocs, m.bytes, v.size());
  if (!v.empty()) check(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, s));
  return p;
}

template <typename V>
void upload_levels(MGSys& m, std::vector<MGLevelD<V>>& out, cudaStream_t s) {
  const auto& lv = m.host.lv;
  out.resize(lv.size());
  for (size_t l = 0; l < lv.size(); ++l) {
    const MGLevelH& H = lv[l];
    MGLevelD<V>& D = out[l];
    D.n = H.A.n;
    D.b = mg_alloc<V>(m.allocs, m.bytes, D.n);
    D.x = mg_alloc<V>(m.allocs, m.bytes, D.n);
    if (l + 1 == lv.size()) continue;  // the coarsest: dense solve only
    D.nnext = lv[l + 1].A.n;
    D.Arp = upload(m, H.A.rp, s);
    D.Aci = upload(m, H.A.ci, s);
    D.Av = upload(m, cast<V>(H.A.v), s);
    D.wd = upload(m, cast<V>(H.wd), s);
    D.Prp = upload(m, H.P.rp, s);
    D.Pci = upload(m, H.P.ci, s);
    D.Pv = upload(m, cast<V>(H.P.v), s);
    D.Rrp = upload(m, H.R.rp, s);
    D.Rci = upload(m, H.R.ci, s);
    D.Rv = upload(m, cast<V>(H.R.v), s);
    D.t = mg_alloc<V>(m.allocs, m.bytes, D.n);
    D.y = mg_alloc<V>(m.allocs, m.bytes, D.n);
  }
  m.C = upload(m, cast<V>(m.host.C), s);
  std::vector<MGLevelView<V>> views(lv.size());
  m.tail = (int)lv.size() - 1;
  for (size_t l = 0; l < lv.size(); ++l) {
    const MGLevelD<V>& D = out[l];
    views[l] = MGLevelView<V>{D.n, D.nnext, D.Arp, D.Aci, D.Prp, D.Pci, D.Rrp, D.Rci, D.Av, D.wd, D.Pv, D.Rv,
                              D.b, D.x, D.t, D.y};
  }
  for (int l = (int)lv.size() - 1; l >= 0 && out[l].n <= kTailRows; --l) m.tail = l;
  m.views = upload(m, views, s);
}

}  // namespace

cudaError_t launch_block_jacobi_vec(const DevOp& op, double coefK, double coefM, int vec_double, void* out, int* bad,
                                    cudaStream_t s);

MGSysPtr mg_sys_build(const MGTopo& topo, const DevOp& d, double coefK, double coefM, int type, bool singular,
                      cudaStream_t s) {
  MGSysPtr mp(new MGSys);
  MGSys& m = *mp;
  m.type = type;
  m.singular = singular;
  m.coefK = coefK;
  m.coefM = coefM;
  m.host.nv = topo.mg.nv;
  m.host.cvid = topo.mg.cvid;
  // A_0 = Pc^T A Pc on the combinatorial pattern, summed triangle by triangle
  CsrD A0 = topo.pattern;
  std::fill(A0.v.begin(), A0.v.end(), 0.0);
  const auto& cv = topo.mg.cvid;
  for (int t = 0; t < d.ne; ++t)
    for (int b = 0; b < 4; ++b) {
      const int u = b == 0 ? t : topo.nbr[(size_t)t * 3 + b - 1];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          double v = coefK * topo.Kr[((size_t)t * 4 + b) * 9 + a * 3 + c];
          if (b == 0 && coefM != 0.0) v += coefM * topo.Mr[(size_t)t * 9 + a * 3 + c];
          const int64_t k = csr_find(A0, cv[(size_t)t * 3 + a], cv[(size_t)u * 3 + c]);
          if (k < 0) throw Error(DGSL_EINVAL, "multigrid: coarse pattern is missing an entry");
          A0.v[k] += v;
        }
    }
  mg_build_levels(m.host, A0, topo.graph, singular);
  const size_t vb = type == 1 ? 8 : 4;
  const int sms = sm_count();
  const int tb = kMGThreads / d.nphi;
  const int ntile = (d.ne + tb - 1) / tb;
  m.grid = std::max(1, std::min(ntile, sms * mg_ctas_per_sm(d.nphi, type)));
  m.cvid = topo.d_cvid;
  m.v2t_ptr = topo.d_v2t_ptr;
  m.v2t = topo.d_v2t;
  // block-Jacobi blocks in the vector type
  const int vp = 16 / (int)vb;
  const size_t dinv_bytes = (size_t)((d.nphi + vp - 1) / vp) * (size_t)d.n * 16;
  m.dinv = mg_alloc<unsigned char>(m.allocs, m.bytes, dinv_bytes);
  int* bad = mg_alloc<int>(m.allocs, m.bytes, 1);
  check(cudaMemsetAsync(bad, 0, sizeof(int), s));
  check(launch_block_jacobi_vec(d, coefK, coefM, type == 1, m.dinv, bad, s));
  auto vec = [&](size_t n) { return mg_alloc<unsigned char>(m.allocs, m.bytes, n * vb); };
  m.r = vec(d.n);
  m.z = vec(d.n);
  m.p = vec(d.n);
  m.q = vec(d.n);
  m.x1 = vec(d.n);
  m.t1 = vec(d.n);
  m.beta = vec((size_t)12 * d.n);
  check(launch_beta(d, type, coefK, m.beta, s));
  m.w = vec((size_t)3 * d.ne);
  m.part = mg_alloc<double>(m.allocs, m.bytes, (size_t)m.grid * 3);
  m.red = mg_alloc<MGRed>(m.allocs, m.bytes, 3);
  m.st = mg_alloc<MGState>(m.allocs, m.bytes, 1);
  check(cudaMemsetAsync(m.red, 0, 3 * sizeof(MGRed), s));
  check(cudaMallocHost(&m.h_st, sizeof(MGState)));
  if (type == 1) upload_levels<double>(m, m.ld, s);
  else upload_levels<float>(m, m.lf, s);
  int h_bad = 0;
  check(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  check(cudaStreamSynchronize(s));
  if (h_bad) throw Error(DGSL_EINVAL, "multigrid: a diagonal block of A is not positive definite");
  return mp;
}

namespace {

template <int NPHI, typename TK, typename TS, typename V>
struct MGRun {
  MGSys& m;
  const DevOp& d;
  cudaStream_t s;
  MGFine f;
  std::vector<MGLevelD<V>>& lv;
  int launches = 0;

  MGRun(MGSys& m_, const DevOp& d_, cudaStream_t s_, std::vector<MGLevelD<V>>& lv_) : m(m_), d(d_), s(s_), lv(lv_) {
    // type 2 (BF16): BF16 couplings in the smoother only; the PCG matvec, which
    // defines the system solved, keeps the FP32 couplings
    f.vals = m.type == 1 ? (const void*)d.K64 : (const void*)d.K32;
    f.svals = m.type == 1 ? (const void*)d.K64 : m.type == 2 ? (const void*)d.K16 : (const void*)d.K32;
    f.cols = d.cols;
    f.ne_pad = d.ne_pad;
    f.ne = d.ne;
    f.n = d.n;
    f.area = d.area;
    f.Mref = d.Mref;
    f.coefK = m.coefK;
    f.coefM = m.coefM;
    f.mean_zero = m.singular ? 1 : 0;
    f.dinv = m.dinv;
    f.cvid = m.cvid;
  }
  V* v(void* p) { return static_cast<V*>(p); }
  int g1(int64_t n) { return (int)std::max<int64_t>(1, (n + 255) / 256); }

  // z = M r for r in m.r (x1, t1 and the level vectors as scratch)
  void precond(V* z, MGRed* red_post) {
    k_mg_resid_restrict<NPHI, TS, V><<<m.grid, kMGThreads, 0, s>>>(f, v(m.r), v(m.x1), v(m.w), v(m.t1), m.st);
    k_mg_vgather<V><<<g1(m.host.nv), 256, 0, s>>>(m.host.nv, m.v2t_ptr, m.v2t, v(m.w), lv[0].b, m.st);
    launches += 2;
    const int L = (int)lv.size(), T = m.tail;
    for (int l = 0; l < T; ++l) {
      auto& D = lv[l];
      k_csr_smooth0<V><<<g1(D.n), 256, 0, s>>>(D.n, D.Arp, D.Aci, D.Av, D.wd, D.b, D.x, D.t, m.st);
      k_csr_spmv_warp<V><<<g1(32 * (int64_t)D.nnext), 256, 0, s>>>(D.nnext, D.Rrp, D.Rci, D.Rv, D.t, lv[l + 1].b,
                                                                   m.st);
      launches += 2;
    }
    k_coarse_tail<V><<<1, kTailThreads, 0, s>>>(static_cast<const MGLevelView<V>*>(m.views), T, L, v(m.C), m.st);
    ++launches;
    V* sol = T == L - 1 ? lv[T].x : lv[T].y;
    for (int l = T - 1; l >= 0; --l) {
      auto& D = lv[l];
      k_csr_prolong_add<V><<<g1(D.n), 256, 0, s>>>(D.n, D.Prp, D.Pci, D.Pv, sol, D.x, m.st);
      k_csr_smooth1<V><<<g1(D.n), 256, 0, s>>>(D.n, D.Arp, D.Aci, D.Av, D.wd, D.b, D.x, D.y, m.st);
      launches += 2;
      sol = D.y;
    }
    k_mg_post<NPHI, V><<<m.grid, kMGThreads, 0, s>>>(f, v(m.r), v(m.x1), v(m.t1), sol, v(m.beta), z, m.part,
                                                     red_post, m.st);
    ++launches;
  }

  int gdir() { return (int)std::max<int64_t>(1, std::min<int64_t>((d.n + 255) / 256, (int64_t)sm_count() * 8)); }

  void prologue(const V* b, V* x) {
    k_mg_update<NPHI, V, true><<<m.grid, kMGThreads, 0, s>>>(f, b, nullptr, nullptr, x, v(m.r), v(m.x1), &m.red[0],
                                                             m.st, 1, m.part, &m.red[1]);
    ++launches;
    precond(v(m.z), &m.red[2]);
    k_mg_dir<V, true><<<gdir(), 256, 0, s>>>(d.n, f.mean_zero, v(m.z), v(m.p), &m.red[1], &m.red[2], m.st, 1);
    ++launches;
  }

  void iteration(V* x, int par) {
    k_mg_matvec<NPHI, TK, V><<<m.grid, kMGThreads, 0, s>>>(f, v(m.p), v(m.q), m.part, &m.red[0], m.st);
    k_mg_update<NPHI, V, false><<<m.grid, kMGThreads, 0, s>>>(f, nullptr, v(m.p), v(m.q), x, v(m.r), v(m.x1),
                                                              &m.red[0], m.st, par, m.part, &m.red[1]);
    launches += 2;
    precond(v(m.z), &m.red[2]);
    k_mg_dir<V, false><<<gdir(), 256, 0, s>>>(d.n, f.mean_zero, v(m.z), v(m.p), &m.red[1], &m.red[2], m.st, par);
    ++launches;
  }

  // The graph of kMGBatch iterations writing x (captured on first use).
  cudaError_t capture(V* x) {
    if (m.exec && m.exec_x == x) return cudaSuccess;
    if (m.exec) {
      cudaGraphExecDestroy(m.exec);
      m.exec = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!m.cap) e = cudaStreamCreateWithFlags(&m.cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    const cudaStream_t s0 = s;
    const int l0 = launches;
    s = m.cap;
    e = cudaStreamBeginCapture(m.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int k = 0; k < kMGBatch; ++k) iteration(x, k & 1);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(m.cap, &g);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&m.exec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    s = s0;
    m.exec_kernels = launches - l0;
    launches = l0;
    m.exec_x = e == cudaSuccess ? x : nullptr;
    return e;
  }

  cudaError_t solve(const V* b, V* x, double stop_rel, int max_iters, MGResult* res) {
    MGState init{};
    init.stop2 = stop_rel * stop_rel;
    init.max_iters = max_iters;
    cudaError_t e = capture(x);
    if (e != cudaSuccess) return e;
    *m.h_st = init;
    e = cudaMemcpyAsync(m.st, m.h_st, sizeof(MGState), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    prologue(b, x);
    int launched = 0;
    for (;;) {
      e = cudaGraphLaunch(m.exec, s);
      if (e != cudaSuccess) return e;
      launches += m.exec_kernels;
      launched += kMGBatch;
      e = cudaMemcpyAsync(m.h_st, m.st, sizeof(MGState), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      if (m.h_st->done || launched > max_iters + kMGBatch) break;
    }
    res->iters = m.h_st->it;
    res->status = m.h_st->status;
    res->rr0 = m.h_st->rr0;
    res->rr = m.h_st->rr;
    res->launches = launches;
    return cudaGetLastError();
  }

  cudaError_t apply(const V* r, V* z) {
    MGState init{};
    *m.h_st = init;
    cudaError_t e = cudaMemcpyAsync(m.st, m.h_st, sizeof(MGState), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // r -> m.r, x1 = omega D^-1 r (the x written is scratch: m.q)
    k_mg_update<NPHI, V, true><<<m.grid, kMGThreads, 0, s>>>(f, r, nullptr, nullptr, v(m.q), v(m.r), v(m.x1),
                                                             &m.red[0], m.st, 1, m.part, &m.red[1]);
    ++launches;
    precond(z, &m.red[2]);
    e = cudaStreamSynchronize(s);  // h_st is reused by the next call
    return e == cudaSuccess ? cudaGetLastError() : e;
  }
};

template <typename TK, typename TS, typename V, class F>
cudaError_t dispatch(MGSys* m, const DevOp& d, cudaStream_t s, std::vector<MGLevelD<V>>& lv, F&& fn) {
  switch (d.nphi) {
    case 3: { MGRun<3, TK, TS, V> r(*m, d, s, lv); cudaError_t e = fn(r); for (int i = 0; i < r.launches; ++i) count_launch(); return e; }
    case 6: { MGRun<6, TK, TS, V> r(*m, d, s, lv); cudaError_t e = fn(r); for (int i = 0; i < r.launches; ++i) count_launch(); return e; }
    case 10: { MGRun<10, TK, TS, V> r(*m, d, s, lv); cudaError_t e = fn(r); for (int i = 0; i < r.launches; ++i) count_launch(); return e; }
    case 15: { MGRun<15, TK, TS, V> r(*m, d, s, lv); cudaError_t e = fn(r); for (int i = 0; i < r.launches; ++i) count_launch(); return e; }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t mg_pcg(MGSys* m, const DevOp& d, const void* b, void* x, double stop_rel, int max_iters, cudaStream_t s,
                   MGResult* res) {
  if (!m || !res) return cudaErrorInvalidValue;
  if (m->type == 1)
    return dispatch<double, double, double>(m, d, s, m->ld, [&](auto& r) {
      return r.solve(static_cast<const double*>(b), static_cast<double*>(x), stop_rel, max_iters, res);
    });
  if (m->type == 2)
    return dispatch<float, uint16_t, float>(m, d, s, m->lf, [&](auto& r) {
      return r.solve(static_cast<const float*>(b), static_cast<float*>(x), stop_rel, max_iters, res);
    });
  return dispatch<float, float, float>(m, d, s, m->lf, [&](auto& r) {
    return r.solve(static_cast<const float*>(b), static_cast<float*>(x), stop_rel, max_iters, res);
  });
}

cudaError_t mg_apply(MGSys* m, const DevOp& d, const void* r, void* z, cudaStream_t s) {
  if (!m) return cudaErrorInvalidValue;
  if (m->type == 1)
    return dispatch<double, double, double>(m, d, s, m->ld, [&](auto& run) {
      return run.apply(static_cast<const double*>(r), static_cast<double*>(z));
    });
  if (m->type == 2)
    return dispatch<float, uint16_t, float>(m, d, s, m->lf, [&](auto& run) {
      return run.apply(static_cast<const float*>(r), static_cast<float*>(z));
    });
  return dispatch<float, float, float>(m, d, s, m->lf, [&](auto& run) {
    return run.apply(static_cast<const float*>(r), static_cast<float*>(z));
  });
}

}  // namespace dgsl
