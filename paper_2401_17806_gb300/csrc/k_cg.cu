// Persistent conjugate-gradient kernels of dgsl (cooperative launch, one CTA
// set resident for the whole solve).
//
// CG as the paper uses it for eq. pressure_final and eq. ad5 (symmetric
// positive (semi)definite, matrix-free apply, no preconditioner).  Reading:
// x0 = 0, stop when the recursive residual satisfies ||r|| <= stop_rel ||r0||.
// For the periodic pressure operator (nullspace span{1}) the right-hand side
// is projected to mean zero and the mean of every A p is removed before it
// updates r, so r and p stay mean-free in floating point.
//
// One iteration = two grid phases:
//   A: p_new = r + beta p_old (formed on the fly for the gathered neighbours),
//      q = A p_new, partial sums of p_new.q and sum(q)            -> barrier
//   B: alpha = r.r / p_new.q; x += alpha p_new; r -= alpha (q - mean q);
//      partial sums of r.r                                          -> barrier
// Partials are summed by every CTA in the same fixed order, so all CTAs take
// identical, deterministic decisions (alpha, beta, stop) without a third
// barrier.  p is double-buffered so phase A never overwrites values other
// CTAs still gather.  Vector data written during the launch is read with
// L1-bypassing loads.  Dot products are accumulated per thread in the vector
// precision and reduced across the grid in FP64.
#include "kassembled.cuh"
#include "kernels.h"

namespace dgsl {

template <typename T, typename V>
struct CGParams {
  const T* vals;
  const int32_t* cols;
  const double* area;
  const double* Mref;
  int ne;
  int64_t n;
  V coefK, coefM;
  int mean_zero;
  V* x;
  V* r;
  V* p0;
  V* p1;
  V* q;
  double* part;
  int max_parts;
  GridBarrier* bar;
  CGResult* res;
  double stop_rel;
  int max_iters;
  uint64_t timeout_ns;
};

template <int NPHI, typename T, typename V>
__global__ void __launch_bounds__(256, 2) k_cg(CGParams<T, V> a) {
  const unsigned nb = gridDim.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = a.n;
  double* partA = a.part;
  double* partB = a.part + 2 * (size_t)a.max_parts;
  int it = 0;
  double rr = 0.0, rr0 = 0.0;
  double tot[2];
  // prologue: mean of r0, x = 0, p buffers = 0
  {
    double acc[2] = {0.0, 0.0};
    V s = V(0);
    for (int64_t row = t0; row < n; row += stride) {
      s += a.r[row];
      a.x[row] = V(0);
      a.p0[row] = V(0);
      a.p1[row] = V(0);
    }
    acc[0] = (double)s;
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
      partA[2 * blockIdx.x] = acc[0];
      partA[2 * blockIdx.x + 1] = 0.0;
    }
  }
  if (!grid_sync(a.bar, nb, a.timeout_ns)) goto done;
  sum_partials<2>(partA, nb, tot);
  {
    const V mu = a.mean_zero ? (V)(tot[0] / (double)n) : V(0);
    double acc[2] = {0.0, 0.0};
    V s = V(0);
    for (int64_t row = t0; row < n; row += stride) {
      const V v = a.r[row] - mu;
      a.r[row] = v;
      s = fma(v, v, s);
    }
    acc[0] = (double)s;
    block_sum<2>(acc);
    if (threadIdx.x == 0) {
      partB[2 * blockIdx.x] = acc[0];
      partB[2 * blockIdx.x + 1] = 0.0;
    }
  }
  if (!grid_sync(a.bar, nb, a.timeout_ns)) goto done;
  sum_partials<2>(partB, nb, tot);
  rr = rr0 = tot[0];
  {
    const double stop = a.stop_rel * a.stop_rel * rr0;
    double beta = 0.0;
    V* pold = a.p0;
    V* pnew = a.p1;
    while (rr > stop && it < a.max_iters) {
      // ---- phase A
      {
        const V vb = (V)beta;
        const V* rr_ = a.r;
        const V* po = pold;
        auto pv = [rr_, po, vb](size_t c) { return fma(vb, ldcg(po + c), ldcg(rr_ + c)); };
        V s_pq = V(0), s_q = V(0);
        for (int64_t row = t0; row < n; row += stride) {
          const V pr = pv((size_t)row);
          V qv = a.coefK * assembled_row_f<NPHI, T, V>(a.vals, a.cols, a.ne, n, row, pv);
          if (a.coefM != V(0)) qv = fma(a.coefM, mass_row_f<NPHI, V>(a.area, a.Mref, row, pv), qv);
          pnew[row] = pr;
          a.q[row] = qv;
          s_pq = fma(pr, qv, s_pq);
          s_q += qv;
        }
        double acc[2] = {(double)s_pq, (double)s_q};
        block_sum<2>(acc);
        if (threadIdx.x == 0) {
          partA[2 * blockIdx.x] = acc[0];
          partA[2 * blockIdx.x + 1] = acc[1];
        }
      }
      if (!grid_sync(a.bar, nb, a.timeout_ns)) goto done;
      sum_partials<2>(partA, nb, tot);
      {
        const double alpha = rr / tot[0];
        const V va = (V)alpha;
        const V muq = a.mean_zero ? (V)(tot[1] / (double)n) : V(0);
        V s_rr = V(0);
        for (int64_t row = t0; row < n; row += stride) {
          const V pr = ldcg(pnew + row);
          a.x[row] = fma(va, pr, a.x[row]);
          const V rv = fma(-va, ldcg(a.q + row) - muq, ldcg(a.r + row));
          a.r[row] = rv;
          s_rr = fma(rv, rv, s_rr);
        }
        double acc[2] = {(double)s_rr, 0.0};
        block_sum<2>(acc);
        if (threadIdx.x == 0) {
          partB[2 * blockIdx.x] = acc[0];
          partB[2 * blockIdx.x + 1] = 0.0;
        }
      }
      if (!grid_sync(a.bar, nb, a.timeout_ns)) goto done;
      sum_partials<2>(partB, nb, tot);
      beta = tot[0] / rr;
      rr = tot[0];
      ++it;
      V* tmp = pold;
      pold = pnew;
      pnew = tmp;
    }
  }
done:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.res->iters = it;
    a.res->rr0 = rr0;
    a.res->rr = rr;
    a.res->status = *((volatile int*)&a.bar->status);
  }
}

namespace {
template <class KernelT>
int coop_blocks(KernelT kern) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0);
  per = std::min(per, 2);
  return std::max(1, sms * per);
}

template <int NPHI, typename T, typename V>
cudaError_t run_cg(const DevOp& op, const T* vals, V coefK, V coefM, int mean_zero, V* x, V* r, double stop_rel,
                   int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s, int* grid_used) {
  auto kern = k_cg<NPHI, T, V>;
  int blocks = std::min(coop_blocks(kern), w.max_parts);
  int64_t need = (op.n + 255) / 256;
  blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, need));
  if (grid_used) *grid_used = blocks;
  CGParams<T, V> a;
  a.vals = vals;
  a.cols = op.cols;
  a.area = op.area;
  a.Mref = op.Mref;
  a.ne = op.ne;
  a.n = op.n;
  a.coefK = coefK;
  a.coefM = coefM;
  a.mean_zero = mean_zero;
  a.x = x;
  a.r = r;
  a.p0 = static_cast<V*>(w.p);
  a.p1 = static_cast<V*>(w.p) + op.n;
  a.q = static_cast<V*>(w.q);
  a.part = w.part;
  a.max_parts = w.max_parts;
  a.bar = w.bar;
  a.res = w.res;
  a.stop_rel = stop_rel;
  a.max_iters = max_iters;
  a.timeout_ns = timeout_ns;
  cudaError_t err = cudaMemsetAsync(w.bar, 0, sizeof(GridBarrier), s);
  if (err != cudaSuccess) return err;
  void* args[] = {&a};
  err = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(256), args, 0, s);
  count_launch();
  return err;
}
}  // namespace

int cg_max_blocks(const DevOp& op, int prec) {
  (void)op;
  (void)prec;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 2;
}

cudaError_t launch_cg_f64(const DevOp& op, double coefK, double coefM, int mean_zero, double* x, double* r,
                          double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s,
                          int* grid_used) {
  if (!op.K64) return cudaErrorInvalidValue;
  switch (op.p) {
    case 1: return run_cg<3, double, double>(op, op.K64, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
    case 2: return run_cg<6, double, double>(op, op.K64, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
    case 3: return run_cg<10, double, double>(op, op.K64, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
    case 4: return run_cg<15, double, double>(op, op.K64, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cg_f32(const DevOp& op, int bf16, float coefK, float coefM, int mean_zero, float* x, float* r,
                          double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s,
                          int* grid_used) {
  if (bf16) {
    if (!op.K16) return cudaErrorInvalidValue;
    switch (op.p) {
      case 1: return run_cg<3, uint16_t, float>(op, op.K16, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
      case 2: return run_cg<6, uint16_t, float>(op, op.K16, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
      case 3: return run_cg<10, uint16_t, float>(op, op.K16, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
      case 4: return run_cg<15, uint16_t, float>(op, op.K16, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
    }
    return cudaErrorInvalidValue;
  }
  if (!op.K32) return cudaErrorInvalidValue;
  switch (op.p) {
    case 1: return run_cg<3, float, float>(op, op.K32, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
    case 2: return run_cg<6, float, float>(op, op.K32, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
    case 3: return run_cg<10, float, float>(op, op.K32, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
    case 4: return run_cg<15, float, float>(op, op.K32, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dgsl
