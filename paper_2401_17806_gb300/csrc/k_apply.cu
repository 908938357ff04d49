// Operator applies of dgsl on sm_103a.
//
//  * assembled form: y = coefM Mbar x + coefK K x with K = G^T Mhat^{-1} G
//    stored as 4 N_phi x N_phi blocks per triangle row (diagonal + the three
//    neighbours, RCM order).  One thread per matrix row; the row's 4 N_phi
//    coefficients are read as 16-byte vectors from a layout in which a warp's
//    32 consecutive rows are contiguous (coalesced 128-bit loads).
//  * factored form (eq. pressure_final as written): per edge,
//    t = G_l x_l + G_r x_r, g = Mhat_j^{-1} t, y_l += G_l^T g, y_r += G_r^T g,
//    one warp per edge, one launch per edge colour so that no two edges of a
//    launch touch the same triangle (deterministic, no atomics).
//  * projections of eqs. d2m / m2d and the divergence G^T (eq. ins.1).
#include <cuda_bf16.h>

#include <atomic>

#include "kassembled.cuh"
#include "kernels.h"

namespace dgsl {

namespace {
std::atomic<uint64_t> g_launches{0};
}
void count_launch(int n) { g_launches.fetch_add((uint64_t)n); }
uint64_t launch_count() { return g_launches.load(); }

// dual-index tables, see kernels.h
__constant__ int c_lmap[5][15];
__constant__ int c_rmap[5][15];
__constant__ int c_dl[5][25];
__constant__ int c_dr[5][25];

void upload_dual_tables(int device) {
  static bool done[64] = {false};
  if (device >= 0 && device < 64 && done[device]) return;
  int lm[5][15] = {}, rm[5][15] = {}, dl[5][25], dr[5][25];
  for (int p = 0; p < 5; ++p)
    for (int l = 0; l < 25; ++l) dl[p][l] = dr[p][l] = -1;
  for (int p = 1; p <= 4; ++p) {
    int n = (p + 1) * (p + 2) / 2;
    int a_of[15], b_of[15], idx = 0;
    for (int b = 0; b <= p; ++b)
      for (int a = 0; a <= p - b; ++a) {
        a_of[idx] = a;
        b_of[idx] = b;
        ++idx;
      }
    int next = n;
    for (int m = 0; m < n; ++m) lm[p][m] = m;
    for (int m = 0; m < n; ++m) {
      if (a_of[m] + b_of[m] < p) {
        rm[p][m] = next++;
      } else {
        for (int u = 0; u < n; ++u)
          if (a_of[u] == b_of[m] && b_of[u] == a_of[m]) rm[p][m] = lm[p][u];
      }
    }
    for (int m = 0; m < n; ++m) {
      dl[p][lm[p][m]] = m;
      dr[p][rm[p][m]] = m;
    }
  }
  cudaMemcpyToSymbol(c_lmap, lm, sizeof(lm));
  cudaMemcpyToSymbol(c_rmap, rm, sizeof(rm));
  cudaMemcpyToSymbol(c_dl, dl, sizeof(dl));
  cudaMemcpyToSymbol(c_dr, dr, sizeof(dr));
  if (device >= 0 && device < 64) done[device] = true;
}

// ------------------------------------------------------------ assembled form

template <int NPHI>
__global__ void __launch_bounds__(256) k_assembled_f64(const double* __restrict__ vals, const int32_t* __restrict__ cols,
                                                       int ne, int64_t n, const double* __restrict__ area,
                                                       const double* __restrict__ Mref, double coefK, double coefM,
                                                       const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    double v = coefK * assembled_row<NPHI, double, double, false>(vals, cols, ne, n, row, x);
    if (coefM != 0.0) v += coefM * mass_row<NPHI, double, false>(area, Mref, row, x);
    y[row] = v;
  }
}

template <int NPHI>
__global__ void __launch_bounds__(256) k_assembled_f32(const float* __restrict__ vals, const int32_t* __restrict__ cols,
                                                       int ne, int64_t n, float coefK, const float* __restrict__ x,
                                                       float* __restrict__ y) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x)
    y[row] = coefK * assembled_row<NPHI, float, float, false>(vals, cols, ne, n, row, x);
}

static int grid_for(int64_t n, int threads = 256) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 16;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

#define DGSL_DISPATCH_P(P, ...)                                        \
  switch (P) {                                                         \
    case 1: { constexpr int NPHI = 3, NPSI = 4; __VA_ARGS__; break; }   \
    case 2: { constexpr int NPHI = 6, NPSI = 9; __VA_ARGS__; break; }   \
    case 3: { constexpr int NPHI = 10, NPSI = 16; __VA_ARGS__; break; } \
    case 4: { constexpr int NPHI = 15, NPSI = 25; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                             \
  }

cudaError_t launch_apply_assembled_f64(const DevOp& op, double coefK, double coefM, const double* x, double* y,
                                       cudaStream_t s) {
  if (!op.K64) return cudaErrorInvalidValue;
  const int g = grid_for(op.n);
  DGSL_DISPATCH_P(op.p, (void)NPSI; k_assembled_f64<NPHI><<<g, 256, 0, s>>>(op.K64, op.cols, op.ne_pad, op.n, op.area,
                                                                             op.Mref, coefK, coefM, x, y));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_apply_assembled_f32(const DevOp& op, float coefK, const float* x, float* y, cudaStream_t s) {
  if (!op.K32) return cudaErrorInvalidValue;
  const int g = grid_for(op.n);
  DGSL_DISPATCH_P(op.p, (void)NPSI; k_assembled_f32<NPHI><<<g, 256, 0, s>>>(op.K32, op.cols, op.ne_pad, op.n, coefK, x, y));
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------ factored form

template <int NPHI>
__global__ void __launch_bounds__(256) k_mass_init(const double* __restrict__ area, const double* __restrict__ Mref,
                                                   int64_t n, double coefM, const double* __restrict__ x,
                                                   double* __restrict__ y) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x)
    y[row] = coefM != 0.0 ? coefM * mass_row<NPHI, double, false>(area, Mref, row, x) : 0.0;
}

// doubles of shared memory per warp in k_factored_colour, rounded to even
__host__ __device__ constexpr int factored_slice(int nphi, int npsi) {
  return (4 * nphi * nphi + npsi * npsi + 2 * nphi + 4 * npsi + 1) / 2 * 2;
}

// One warp per edge of one colour.  The edge's G_l, G_r and Mhat^{-1} are
// staged in the warp's shared-memory slice with coalesced 16-byte loads.
template <int P, int NPHI, int NPSI>
__global__ void __launch_bounds__(128) k_factored_colour(const double* __restrict__ G, const double* __restrict__ Minv,
                                                         const int32_t* __restrict__ elr, int e0, int e1,
                                                         double coefK, const double* __restrict__ x,
                                                         double* __restrict__ y) {
  constexpr int GN = 4 * NPHI * NPHI;
  constexpr int MN = NPSI * NPSI;
  constexpr int SLICE = factored_slice(NPHI, NPSI);  // even: 16-byte aligned slices
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  double* g_s = smem + (size_t)w * SLICE;
  double* m_s = g_s + GN;
  double* x_s = m_s + MN;
  double* t_s = x_s + 2 * NPHI;
  double* r_s = t_s + 2 * NPSI;
  for (int e = e0 + blockIdx.x * wpb + w; e < e1; e += gridDim.x * wpb) {
    const double2* gsrc = reinterpret_cast<const double2*>(G + (size_t)e * GN);
    for (int i = lane; i < GN / 2; i += 32) reinterpret_cast<double2*>(g_s)[i] = __ldg(gsrc + i);
    const double* msrc = Minv + (size_t)e * MN;
    for (int i = lane; i < MN; i += 32) m_s[i] = __ldg(msrc + i);
    const int tl = __ldg(elr + 2 * e), tr = __ldg(elr + 2 * e + 1);
    for (int i = lane; i < 2 * NPHI; i += 32)
      x_s[i] = i < NPHI ? x[(size_t)tl * NPHI + i] : x[(size_t)tr * NPHI + i - NPHI];
    __syncwarp();
    // t[c][l] = sum_k G_l[c][dl(l)][k] x_l[k] + G_r[c][dr(l)][k] x_r[k]
    for (int o = lane; o < 2 * NPSI; o += 32) {
      const int c = o / NPSI, l = o % NPSI;
      const int ml = c_dl[P][l], mr = c_dr[P][l];
      double acc = 0.0;
      if (ml >= 0) {
        const double* row = g_s + ((0 * 2 + c) * NPHI + ml) * NPHI;
#pragma unroll
        for (int k = 0; k < NPHI; ++k) acc = fma(row[k], x_s[k], acc);
      }
      if (mr >= 0) {
        const double* row = g_s + ((1 * 2 + c) * NPHI + mr) * NPHI;
#pragma unroll
        for (int k = 0; k < NPHI; ++k) acc = fma(row[k], x_s[NPHI + k], acc);
      }
      t_s[o] = acc;
    }
    __syncwarp();
    // g = Mhat^{-1} t, per component
    for (int o = lane; o < 2 * NPSI; o += 32) {
      const int c = o / NPSI, l = o % NPSI;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NPSI; ++q) acc = fma(m_s[l * NPSI + q], t_s[c * NPSI + q], acc);
      r_s[o] = acc;
    }
    __syncwarp();
    // y_s[k] += coefK sum_c sum_m G_s[c][m][k] g[c][map_s(m)]
    for (int o = lane; o < 2 * NPHI; o += 32) {
      const int s = o / NPHI, k = o % NPHI;
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 0; m < NPHI; ++m) {
          const int l = s == 0 ? c_lmap[P][m] : c_rmap[P][m];
          acc = fma(g_s[((s * 2 + c) * NPHI + m) * NPHI + k], r_s[c * NPSI + l], acc);
        }
      const int t = s == 0 ? tl : tr;
      y[(size_t)t * NPHI + k] += coefK * acc;
    }
    __syncwarp();
  }
}

cudaError_t launch_apply_factored_f64(const DevOp& op, double coefK, double coefM, const double* x, double* y,
                                      cudaStream_t s) {
  if (!op.G || !op.Minv) return cudaErrorInvalidValue;
  const int g = grid_for(op.n);
  DGSL_DISPATCH_P(op.p, (void)NPSI; k_mass_init<NPHI><<<g, 256, 0, s>>>(op.area, op.Mref, op.n, coefM, x, y));
  count_launch();
  for (int c = 0; c < op.ncol; ++c) {
    const int e0 = op.colour_offsets[c], e1 = op.colour_offsets[c + 1];
    if (e1 <= e0) continue;
    const int wpb = 4;
    const int blocks = std::min((e1 - e0 + wpb - 1) / wpb, 152 * 16);
    switch (op.p) {
      case 1: { constexpr int N = 3, NP = 4; size_t sm = (size_t)wpb * factored_slice(N, NP) * 8;
        k_factored_colour<1, N, NP><<<blocks, 32 * wpb, sm, s>>>(op.G, op.Minv, op.elr, e0, e1, coefK, x, y); break; }
      case 2: { constexpr int N = 6, NP = 9; size_t sm = (size_t)wpb * factored_slice(N, NP) * 8;
        k_factored_colour<2, N, NP><<<blocks, 32 * wpb, sm, s>>>(op.G, op.Minv, op.elr, e0, e1, coefK, x, y); break; }
      case 3: { constexpr int N = 10, NP = 16; size_t sm = (size_t)wpb * factored_slice(N, NP) * 8;
        k_factored_colour<3, N, NP><<<blocks, 32 * wpb, sm, s>>>(op.G, op.Minv, op.elr, e0, e1, coefK, x, y); break; }
      case 4: { constexpr int N = 15, NP = 25; size_t sm = (size_t)wpb * factored_slice(N, NP) * 8;
        cudaFuncSetAttribute(k_factored_colour<4, N, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_factored_colour<4, N, NP><<<blocks, 32 * wpb, sm, s>>>(op.G, op.Minv, op.elr, e0, e1, coefK, x, y); break; }
      default: return cudaErrorInvalidValue;
    }
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------ projections

// b[i][k] = sum over the 3 edges (e, side s) of triangle i of
//           sum_m Uloc[e][s][m][k] vhat[e][map_s(m)]        (eq. d2m times Mbar)
template <int P, int NPHI, int NPSI>
__global__ void __launch_bounds__(256) k_d2m_rhs(const double* __restrict__ Uloc, const int32_t* __restrict__ tedge,
                                                 int64_t n, const double* __restrict__ vhat, double* __restrict__ b) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(row / NPHI), k = (int)(row % NPHI);
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int es = __ldg(tedge + 3 * i + a), e = es >> 1, s = es & 1;
      const double* U = Uloc + ((size_t)e * 2 + s) * NPHI * NPHI;
#pragma unroll
      for (int m = 0; m < NPHI; ++m) {
        const int l = s == 0 ? c_lmap[P][m] : c_rmap[P][m];
        acc = fma(__ldg(U + m * NPHI + k), __ldg(vhat + (size_t)e * NPSI + l), acc);
      }
    }
    b[row] = acc;
  }
}

// vhat_j = Mhat_j^{-1} (U_lj vbar_l + U_rj vbar_r), one warp per edge  (eq. m2d)
template <int P, int NPHI, int NPSI>
__global__ void __launch_bounds__(128) k_m2d(const double* __restrict__ Uloc, const double* __restrict__ Minv,
                                             const int32_t* __restrict__ elr, int nd, const double* __restrict__ vbar,
                                             double* __restrict__ vhat) {
  __shared__ double t_s[4][NPSI];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + w; e < nd; e += gridDim.x * wpb) {
    const int tri[2] = {__ldg(elr + 2 * e), __ldg(elr + 2 * e + 1)};
    for (int l = lane; l < NPSI; l += 32) {
      double acc = 0.0;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int m = s == 0 ? c_dl[P][l] : c_dr[P][l];
        if (m < 0) continue;
        const double* U = Uloc + ((size_t)e * 2 + s) * NPHI * NPHI + m * NPHI;
        const double* xv = vbar + (size_t)tri[s] * NPHI;
#pragma unroll
        for (int k = 0; k < NPHI; ++k) acc = fma(__ldg(U + k), __ldg(xv + k), acc);
      }
      t_s[w][l] = acc;
    }
    __syncwarp();
    for (int l = lane; l < NPSI; l += 32) {
      const double* Mi = Minv + (size_t)e * NPSI * NPSI + l * NPSI;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NPSI; ++q) acc = fma(__ldg(Mi + q), t_s[w][q], acc);
      vhat[(size_t)e * NPSI + l] = acc;
    }
    __syncwarp();
  }
}

// y[i][k] = sum over edges (e, s) of triangle i of
//           sum_c sum_m G[e][s][c][m][k] vhat[c][e][map_s(m)]   (y = G^T vhat = -D vhat)
template <int P, int NPHI, int NPSI>
__global__ void __launch_bounds__(256) k_div(const double* __restrict__ G, const int32_t* __restrict__ tedge, int nd,
                                             int64_t n, const double* __restrict__ vhat, double* __restrict__ y) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(row / NPHI), k = (int)(row % NPHI);
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int es = __ldg(tedge + 3 * i + a), e = es >> 1, s = es & 1;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const double* Gb = G + (((size_t)e * 2 + s) * 2 + c) * NPHI * NPHI;
        const double* v = vhat + ((size_t)c * nd + e) * NPSI;
#pragma unroll
        for (int m = 0; m < NPHI; ++m) {
          const int l = s == 0 ? c_lmap[P][m] : c_rmap[P][m];
          acc = fma(__ldg(Gb + m * NPHI + k), __ldg(v + l), acc);
        }
      }
    }
    y[row] = acc;
  }
}

cudaError_t launch_d2m_rhs(const DevOp& op, const double* vhat, double* b, cudaStream_t s) {
  if (!op.Uloc) return cudaErrorInvalidValue;
  const int g = grid_for(op.n);
  switch (op.p) {
    case 1: k_d2m_rhs<1, 3, 4><<<g, 256, 0, s>>>(op.Uloc, op.tedge, op.n, vhat, b); break;
    case 2: k_d2m_rhs<2, 6, 9><<<g, 256, 0, s>>>(op.Uloc, op.tedge, op.n, vhat, b); break;
    case 3: k_d2m_rhs<3, 10, 16><<<g, 256, 0, s>>>(op.Uloc, op.tedge, op.n, vhat, b); break;
    case 4: k_d2m_rhs<4, 15, 25><<<g, 256, 0, s>>>(op.Uloc, op.tedge, op.n, vhat, b); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

// Velocity update of eq. nc.2 (source terms left to the caller), one warp per
// edge:  vhat[c][e] = F[c][e] - coef Mhat_e^{-1} (G_l[c] p_l + G_r[c] p_r).
// Every element is read and written by one thread, so v may be F.
template <int P, int NPHI, int NPSI>
__global__ void __launch_bounds__(128) k_vel_update(const double* __restrict__ G, const double* __restrict__ Minv,
                                                    const int32_t* __restrict__ elr, int nd, double coef,
                                                    const double* F, const double* __restrict__ pr, double* v) {
  __shared__ double t_s[4][2 * NPSI];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + w; e < nd; e += gridDim.x * wpb) {
    const int tl = __ldg(elr + 2 * e), tr = __ldg(elr + 2 * e + 1);
    for (int o = lane; o < 2 * NPSI; o += 32) {
      const int c = o / NPSI, l = o % NPSI;
      const int ml = c_dl[P][l], mr = c_dr[P][l];
      double acc = 0.0;
      if (ml >= 0) {
        const double* row = G + (((size_t)e * 2 + 0) * 2 + c) * NPHI * NPHI + ml * NPHI;
#pragma unroll
        for (int k = 0; k < NPHI; ++k) acc = fma(__ldg(row + k), __ldg(pr + (size_t)tl * NPHI + k), acc);
      }
      if (mr >= 0) {
        const double* row = G + (((size_t)e * 2 + 1) * 2 + c) * NPHI * NPHI + mr * NPHI;
#pragma unroll
        for (int k = 0; k < NPHI; ++k) acc = fma(__ldg(row + k), __ldg(pr + (size_t)tr * NPHI + k), acc);
      }
      t_s[w][o] = acc;
    }
    __syncwarp();
    for (int o = lane; o < 2 * NPSI; o += 32) {
      const int c = o / NPSI, l = o % NPSI;
      const double* Mi = Minv + (size_t)e * NPSI * NPSI + l * NPSI;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NPSI; ++q) acc = fma(__ldg(Mi + q), t_s[w][c * NPSI + q], acc);
      const size_t idx = ((size_t)c * nd + e) * NPSI + l;
      v[idx] = F[idx] - coef * acc;
    }
    __syncwarp();
  }
}

cudaError_t launch_velocity_update(const DevOp& op, double coef, const double* F, const double* pr, double* v,
                                   cudaStream_t s) {
  if (!op.G || !op.Minv) return cudaErrorInvalidValue;
  const int wpb = 4;
  const int blocks = std::max(1, std::min((op.nd + wpb - 1) / wpb, 152 * 16));
  switch (op.p) {
    case 1: k_vel_update<1, 3, 4><<<blocks, 32 * wpb, 0, s>>>(op.G, op.Minv, op.elr, op.nd, coef, F, pr, v); break;
    case 2: k_vel_update<2, 6, 9><<<blocks, 32 * wpb, 0, s>>>(op.G, op.Minv, op.elr, op.nd, coef, F, pr, v); break;
    case 3: k_vel_update<3, 10, 16><<<blocks, 32 * wpb, 0, s>>>(op.G, op.Minv, op.elr, op.nd, coef, F, pr, v); break;
    case 4: k_vel_update<4, 15, 25><<<blocks, 32 * wpb, 0, s>>>(op.G, op.Minv, op.elr, op.nd, coef, F, pr, v); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_m2d(const DevOp& op, const double* vbar, double* vhat, cudaStream_t s) {
  if (!op.Uloc || !op.Minv) return cudaErrorInvalidValue;
  const int g = std::max(1, std::min((op.nd + 3) / 4, 152 * 16));
  switch (op.p) {
    case 1: k_m2d<1, 3, 4><<<g, 128, 0, s>>>(op.Uloc, op.Minv, op.elr, op.nd, vbar, vhat); break;
    case 2: k_m2d<2, 6, 9><<<g, 128, 0, s>>>(op.Uloc, op.Minv, op.elr, op.nd, vbar, vhat); break;
    case 3: k_m2d<3, 10, 16><<<g, 128, 0, s>>>(op.Uloc, op.Minv, op.elr, op.nd, vbar, vhat); break;
    case 4: k_m2d<4, 15, 25><<<g, 128, 0, s>>>(op.Uloc, op.Minv, op.elr, op.nd, vbar, vhat); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_div(const DevOp& op, const double* vhat, double* y, cudaStream_t s) {
  if (!op.G) return cudaErrorInvalidValue;
  const int g = grid_for(op.n);
  switch (op.p) {
    case 1: k_div<1, 3, 4><<<g, 256, 0, s>>>(op.G, op.tedge, op.nd, op.n, vhat, y); break;
    case 2: k_div<2, 6, 9><<<g, 256, 0, s>>>(op.G, op.tedge, op.nd, op.n, vhat, y); break;
    case 3: k_div<3, 10, 16><<<g, 256, 0, s>>>(op.G, op.tedge, op.nd, op.n, vhat, y); break;
    case 4: k_div<4, 15, 25><<<g, 256, 0, s>>>(op.G, op.tedge, op.nd, op.n, vhat, y); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------ refinement helpers

template <int NPHI>
__global__ void __launch_bounds__(256) k_residual_f64(const double* __restrict__ vals, const int32_t* __restrict__ cols,
                                                      int ne, int64_t n, const double* __restrict__ area,
                                                      const double* __restrict__ Mref, double coefK, double coefM,
                                                      const double* __restrict__ b, double b_shift,
                                                      const double* __restrict__ x, double* __restrict__ r,
                                                      double* __restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    double ax = coefK * assembled_row<NPHI, double, double, false>(vals, cols, ne, n, row, x);
    if (coefM != 0.0) ax += coefM * mass_row<NPHI, double, false>(area, Mref, row, x);
    const double v = (b[row] - b_shift) - ax;
    r[row] = v;
    acc[0] += v;
    acc[1] = fma(v, v, acc[1]);
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc[0];
    part[2 * blockIdx.x + 1] = acc[1];
  }
}

// sum over rows of sum_c (a_c x_c)^2, a_c the row's FP64 couplings of
// coefK K + coefM Mbar (the self coupling included): with each x_c rounded to
// FP64 (a relative error uniform in +-2^-53, independent between values) the
// residual moves by a vector of expected squared norm 2^-106 / 3 times this
// sum.  That is the residual the exactly rounded solution would show: the
// floor under which no FP64 iterate's residual can be driven.
template <int NPHI>
__global__ void __launch_bounds__(256) k_residual_floor_f64(const double* __restrict__ vals,
                                                            const int32_t* __restrict__ cols, int ne, int64_t n,
                                                            const double* __restrict__ area,
                                                            const double* __restrict__ Mref, double coefK,
                                                            double coefM, const double* __restrict__ x,
                                                            double* __restrict__ part) {
  constexpr int NC = 4 * NPHI;
  double acc[2] = {0.0, 0.0};
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(row / NPHI), k = (int)(row - (int64_t)i * NPHI);
    int col[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) col[b] = __ldg(cols + (size_t)b * ne + i);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int b = c / NPHI, kk = c % NPHI;
      double a = coefK * __ldg(vals + ((size_t)(c / 2) * n + row) * 2 + c % 2);
      if (b == 0 && coefM != 0.0) a += coefM * __ldg(area + i) * __ldg(Mref + k * NPHI + kk);
      const double t = a * __ldg(x + (size_t)col[b] * NPHI + kk);
      acc[0] = fma(t, t, acc[0]);
    }
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc[0];
    part[2 * blockIdx.x + 1] = acc[1];
  }
}

cudaError_t launch_residual_floor_f64(const DevOp& op, double coefK, double coefM, const double* x, double* part,
                                      int max_parts, int* nparts, cudaStream_t s) {
  const int g = std::min(grid_for(op.n), max_parts);
  *nparts = g;
  DGSL_DISPATCH_P(op.p, (void)NPSI; k_residual_floor_f64<NPHI><<<g, 256, 0, s>>>(
                            op.K64, op.cols, op.ne_pad, op.n, op.area, op.Mref, coefK, coefM, x, part));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_residual_f64(const DevOp& op, double coefK, double coefM, int mean_zero, const double* b,
                                const double* x, double b_mean, double* r, double* part, int max_parts, int* nparts,
                                cudaStream_t s) {
  const int g = std::min(grid_for(op.n), max_parts);
  *nparts = g;
  const double shift = mean_zero ? b_mean : 0.0;
  DGSL_DISPATCH_P(op.p, (void)NPSI; k_residual_f64<NPHI><<<g, 256, 0, s>>>(op.K64, op.cols, op.ne_pad, op.n, op.area,
                                                                            op.Mref, coefK, coefM, b, shift, x, r, part));
  count_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_sum2(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[i];
    acc[0] += x;
    acc[1] = fma(x, x, acc[1]);
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc[0];
    part[2 * blockIdx.x + 1] = acc[1];
  }
}

cudaError_t launch_sum2(const double* v, int64_t n, double* part, int max_parts, int* nparts, cudaStream_t s) {
  const int g = std::min(grid_for(n), max_parts);
  *nparts = g;
  k_sum2<<<g, 256, 0, s>>>(v, n, part);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_scale_to_f32(const double* __restrict__ v, double scale, float* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(v[i] * scale);
}
cudaError_t launch_scale_to_f32(const double* v, double scale, float* out, int64_t n, cudaStream_t s) {
  k_scale_to_f32<<<grid_for(n), 256, 0, s>>>(v, scale, out, n);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_axpy_f32_to_f64(double a, const float* __restrict__ d, double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, (double)d[i], x[i]);
}
cudaError_t launch_axpy_f32_to_f64(double a, const float* d, double* x, int64_t n, cudaStream_t s) {
  k_axpy_f32_to_f64<<<grid_for(n), 256, 0, s>>>(a, d, x, n);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_remove_mean(double* __restrict__ x, const double* __restrict__ sum, int64_t n) {
  const double mu = *sum / (double)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] -= mu;
}
cudaError_t launch_remove_mean_f64(double* x, const double* sum_dev, int64_t n, cudaStream_t s) {
  k_remove_mean<<<grid_for(n), 256, 0, s>>>(x, sum_dev, n);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_axpy_f64(double a, const double* __restrict__ d, double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, d[i], x[i]);
}
cudaError_t launch_axpy_f64(double a, const double* d, double* x, int64_t n, cudaStream_t s) {
  k_axpy_f64<<<grid_for(n), 256, 0, s>>>(a, d, x, n);
  count_launch();
  return cudaGetLastError();
}

// ---- inverse main-grid mass matrix: y_i = Mref^-1 x_i / A_i (eq. MassMatrixM), thread per row
template <int NPHI>
__global__ void __launch_bounds__(256) k_mass_inv(const double* __restrict__ area, const double* __restrict__ Minv,
                                                  int64_t n, int ncomp, const double* __restrict__ x,
                                                  double* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ncomp) return;
  const int64_t c = t / n, row = t - c * n;
  const int64_t i = row / NPHI;
  const int k = (int)(row - i * NPHI);
  const double* xi = x + c * n + i * NPHI;
  double acc = 0.0;
#pragma unroll
  for (int l = 0; l < NPHI; ++l) acc = fma(__ldg(Minv + k * NPHI + l), __ldg(xi + l), acc);
  y[t] = acc / __ldg(area + i);
}

cudaError_t launch_mass_inv(const DevOp& op, const double* x, double* y, int ncomp, cudaStream_t s) {
  if (!op.Mrefinv || ncomp < 1) return cudaErrorInvalidValue;
  const int g = (int)((op.n * ncomp + 255) / 256);
  switch (op.p) {
    case 1: k_mass_inv<3><<<g, 256, 0, s>>>(op.area, op.Mrefinv, op.n, ncomp, x, y); break;
    case 2: k_mass_inv<6><<<g, 256, 0, s>>>(op.area, op.Mrefinv, op.n, ncomp, x, y); break;
    case 3: k_mass_inv<10><<<g, 256, 0, s>>>(op.area, op.Mrefinv, op.n, ncomp, x, y); break;
    case 4: k_mass_inv<15><<<g, 256, 0, s>>>(op.area, op.Mrefinv, op.n, ncomp, x, y); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

// ---- block-Jacobi preconditioner (an extension): P_i = D_i^-1 for the diagonal blocks
// D_i = coefK K_0(i) + coefM A_i Mref of A (symmetrised), one triangle per
// thread in FP64: Cholesky D = L L^T, W = L^-1 by forward substitution, then
// P = W^T W, written symmetric into the interleaved layout of the couplings.
template <int NPHI, typename V>
__global__ void __launch_bounds__(64) k_block_jacobi(const double* __restrict__ K64, const double* __restrict__ area,
                                                     const double* __restrict__ Mref, int ne, int64_t n,
                                                     double coefK, double coefM, V* __restrict__ out, int* bad) {
  constexpr int VP = 16 / (int)sizeof(V);
  constexpr int NGP = (NPHI + VP - 1) / VP;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const int64_t row0 = (int64_t)i * NPHI;
  auto kd = [&](int k, int kk) { return K64[((int64_t)(kk / 2) * n + row0 + k) * 2 + kk % 2]; };
  const double am = coefM != 0.0 ? coefM * area[i] : 0.0;
  double L[NPHI][NPHI];
  for (int k = 0; k < NPHI; ++k)
    for (int kk = 0; kk < NPHI; ++kk)
      L[k][kk] = 0.5 * (coefK * (kd(k, kk) + kd(kk, k)) + am * (Mref[k * NPHI + kk] + Mref[kk * NPHI + k]));
  bool spd = true;
  for (int j = 0; j < NPHI; ++j) {
    double d = L[j][j];
    for (int m = 0; m < j; ++m) d -= L[j][m] * L[j][m];
    if (!(d > 0.0) || !isfinite(d)) {
      spd = false;
      d = 1.0;
    }
    const double ljj = sqrt(d);
    L[j][j] = ljj;
    for (int r = j + 1; r < NPHI; ++r) {
      double v = L[r][j];
      for (int m = 0; m < j; ++m) v -= L[r][m] * L[j][m];
      L[r][j] = v / ljj;
    }
  }
  if (!spd) atomicExch(bad, 1);
  double W[NPHI][NPHI];  // L^-1, lower triangular
  for (int c = 0; c < NPHI; ++c)
    for (int r = 0; r < NPHI; ++r) {
      if (r < c) {
        W[r][c] = 0.0;
        continue;
      }
      double v = r == c ? 1.0 : 0.0;
      for (int m = c; m < r; ++m) v -= L[r][m] * W[m][c];
      W[r][c] = v / L[r][r];
    }
  for (int k = 0; k < NPHI; ++k)
    for (int l = k; l < NPHI; ++l) {
      double v = 0.0;
      for (int m = l; m < NPHI; ++m) v += W[m][k] * W[m][l];
      out[((int64_t)(l / VP) * n + row0 + k) * VP + l % VP] = (V)v;
      out[((int64_t)(k / VP) * n + row0 + l) * VP + k % VP] = (V)v;
    }
  for (int k = 0; k < NPHI; ++k)
    for (int l = NPHI; l < NGP * VP; ++l) out[((int64_t)(l / VP) * n + row0 + k) * VP + l % VP] = V(0);
}

// Couplings of A P: thread (row, b) forms the row's block b, sum_m A_b(i)[k][m]
// P_j[m][l] (j the block's triangle), in FP64 from the FP64 couplings and P,
// rounded once to the coupling type.
__device__ __forceinline__ void store_cvt(double v, double* o) { *o = v; }
__device__ __forceinline__ void store_cvt(double v, float* o) { *o = (float)v; }
__device__ __forceinline__ void store_cvt(double v, uint16_t* o) {  // BF16, round to nearest even
  const float f = (float)v;
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);
  *o = (uint16_t)(u >> 16);
}

template <int NPHI, typename T>
__global__ void __launch_bounds__(128) k_fold_ap(const double* __restrict__ K64, const int32_t* __restrict__ cols,
                                                 int ne_pad, const double* __restrict__ area,
                                                 const double* __restrict__ Mref, const double* __restrict__ P64,
                                                 int64_t n, double coefK, double coefM, T* __restrict__ out) {
  constexpr int VEC = 16 / (int)sizeof(T);
  constexpr int NC = 4 * NPHI;
  constexpr int NG = (NC + VEC - 1) / VEC;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * n) return;
  const int b = (int)(t / n);
  const int64_t row = t - (int64_t)b * n;
  const int i = (int)(row / NPHI), k = (int)(row % NPHI);
  const int64_t j0 = (int64_t)cols[(size_t)b * ne_pad + i] * NPHI;
  double a[NPHI];
#pragma unroll
  for (int m = 0; m < NPHI; ++m) {
    const int c = b * NPHI + m;
    a[m] = coefK * K64[((int64_t)(c / 2) * n + row) * 2 + c % 2];
    if (b == 0 && coefM != 0.0) a[m] += coefM * area[i] * Mref[k * NPHI + m];
  }
  for (int l = 0; l < NPHI; ++l) {
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < NPHI; ++m) v += a[m] * P64[((int64_t)(l / 2) * n + j0 + m) * 2 + l % 2];
    const int c = b * NPHI + l;
    store_cvt(v, out + ((int64_t)(c / VEC) * n + row) * VEC + c % VEC);
  }
  if (b == 3)
    for (int c = NC; c < NG * VEC; ++c) store_cvt(0.0, out + ((int64_t)(c / VEC) * n + row) * VEC + c % VEC);
}

// P from the FP64 layout (2 values per 16 bytes) to the FP32 one (4).
template <int NPHI>
__global__ void k_p64_to_f32(const double* __restrict__ P64, int64_t n, float* __restrict__ out) {
  constexpr int W = (NPHI + 3) / 4 * 4;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= W * n) return;
  const int l = (int)(t / n);
  const int64_t row = t - (int64_t)l * n;
  out[((int64_t)(l / 4) * n + row) * 4 + l % 4] =
      l < NPHI ? (float)P64[((int64_t)(l / 2) * n + row) * 2 + l % 2] : 0.0f;
}

size_t precond_ap_bytes(const DevOp& op, int type) {
  const int vec = type == 1 ? 2 : type == 2 ? 8 : 4;
  const int ng = (4 * op.nphi + vec - 1) / vec;
  return (size_t)ng * (size_t)op.n * 16;
}
size_t precond_pinv_bytes(const DevOp& op, int type) {
  const int vp = type == 1 ? 2 : 4;
  return (size_t)((op.nphi + vp - 1) / vp) * (size_t)op.n * 16;
}

template <int NPHI>
static void run_build_precond(const DevOp& op, double coefK, double coefM, int type, void* ap, void* pinv,
                              double* p64, int* bad, cudaStream_t s) {
  k_block_jacobi<NPHI, double><<<(op.ne + 63) / 64, 64, 0, s>>>(op.K64, op.area, op.Mref, op.ne, op.n, coefK, coefM,
                                                                p64, bad);
  const int gf = (int)((4 * op.n + 127) / 128);
  if (type == 1)
    k_fold_ap<NPHI, double><<<gf, 128, 0, s>>>(op.K64, op.cols, op.ne_pad, op.area, op.Mref, p64, op.n, coefK,
                                               coefM, static_cast<double*>(ap));
  else if (type == 2)
    k_fold_ap<NPHI, uint16_t><<<gf, 128, 0, s>>>(op.K64, op.cols, op.ne_pad, op.area, op.Mref, p64, op.n, coefK,
                                                 coefM, static_cast<uint16_t*>(ap));
  else
    k_fold_ap<NPHI, float><<<gf, 128, 0, s>>>(op.K64, op.cols, op.ne_pad, op.area, op.Mref, p64, op.n, coefK,
                                              coefM, static_cast<float*>(ap));
  if (type == 1) {
    if (pinv != p64) cudaMemcpyAsync(pinv, p64, precond_pinv_bytes(op, 1), cudaMemcpyDeviceToDevice, s);
  } else {
    constexpr int W = (NPHI + 3) / 4 * 4;
    k_p64_to_f32<NPHI><<<(int)((W * op.n + 255) / 256), 256, 0, s>>>(p64, op.n, static_cast<float*>(pinv));
  }
}

// The inverse diagonal blocks alone (the multigrid smoother's D^-1), in the
// vector type: FP64 (vec_double) or FP32, in the interleaved layout of P.
cudaError_t launch_block_jacobi_vec(const DevOp& op, double coefK, double coefM, int vec_double, void* out, int* bad,
                                    cudaStream_t s) {
  if (!op.K64 || op.ne < 1 || !out || !bad) return cudaErrorInvalidValue;
  const int g = (op.ne + 63) / 64;
  DGSL_DISPATCH_P(op.p, (void)NPSI;
                  if (vec_double) k_block_jacobi<NPHI, double><<<g, 64, 0, s>>>(op.K64, op.area, op.Mref, op.ne, op.n,
                                                                                coefK, coefM, static_cast<double*>(out),
                                                                                bad);
                  else k_block_jacobi<NPHI, float><<<g, 64, 0, s>>>(op.K64, op.area, op.Mref, op.ne, op.n, coefK,
                                                                     coefM, static_cast<float*>(out), bad));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_build_precond(const DevOp& op, double coefK, double coefM, int type, void* ap, void* pinv,
                                 double* p64, int* bad, cudaStream_t s) {
  if (!op.K64 || op.ne < 1 || type < 0 || type > 2 || !ap || !pinv || !p64) return cudaErrorInvalidValue;
  switch (op.p) {
    case 1: run_build_precond<3>(op, coefK, coefM, type, ap, pinv, p64, bad, s); break;
    case 2: run_build_precond<6>(op, coefK, coefM, type, ap, pinv, p64, bad, s); break;
    case 3: run_build_precond<10>(op, coefK, coefM, type, ap, pinv, p64, bad, s); break;
    case 4: run_build_precond<15>(op, coefK, coefM, type, ap, pinv, p64, bad, s); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch(type == 1 ? 2 : 3);
  return cudaGetLastError();
}

__global__ void k_sum_to_first(double* part, int nparts) {
  double v[1] = {0.0};
  for (int j = threadIdx.x; j < nparts; j += blockDim.x) v[0] += part[2 * j];
  block_sum<1>(v);
  if (threadIdx.x == 0) part[0] = v[0];
}
cudaError_t launch_sum_to_first(double* part, int nparts, cudaStream_t s) {
  k_sum_to_first<<<1, 256, 0, s>>>(part, nparts);
  count_launch();
  return cudaGetLastError();
}

// y = 2 a - prev and prev = a, elementwise (y may be a): the linear
// extrapolation of a quantity from its last two values.
__global__ void k_extrapolate(const double* a, double* prev, double* y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double cur = a[i];
  y[i] = 2.0 * cur - prev[i];
  prev[i] = cur;
}

cudaError_t launch_extrapolate(const double* a, double* prev, double* y, int64_t n, cudaStream_t s) {
  k_extrapolate<<<(int)((n + 255) / 256), 256, 0, s>>>(a, prev, y, n);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace dgsl
