// Persistent conjugate-gradient kernels of dgsl (cooperative launch: all CTAs
// resident for the whole solve).
//
// CG as the paper uses it for eq. pressure_final and eq. ad5 (symmetric
// positive (semi)definite, matrix-free apply, no preconditioner), in the
// Chronopoulos-Gear arrangement: with w = A r and s = A p carried by
// recurrence, both inner products of an iteration come from one grid-wide
// reduction, so an iteration costs one pass and one grid barrier:
//   p = r + beta p;  s = w' + beta s;  x += alpha p;  r <- r - alpha s;
//   w <- A r;  reduce (r.r, w.r, sum w, sum r);
//   beta' = g'/g;  alpha' = g' / (d' - beta' g' / alpha)
// where w' = w - mean(w) for the periodic pressure operator (nullspace span{1};
// r and p stay mean-free).  Reading: x0 = 0, stop when the recursive residual
// satisfies ||r|| <= stop_rel ||r0||.
//
// The pass is tiled by triangles: a CTA stages, for a tile of triangles, the
// new residual of each triangle and of its three neighbours in shared memory
// (formed on the fly as r - alpha (w' + beta s) from the previous buffers), so
// each neighbour block is gathered once per tile instead of once per matrix
// row; r, w and s are double-buffered because other CTAs still gather the
// previous values.  Each thread then owns one matrix row: it streams that row's
// 4 N_phi coupling coefficients (16-byte loads) against the staged values.
// Partial sums are reduced per CTA and summed by every CTA in the same fixed
// order, so all CTAs take identical, deterministic decisions.
#include "kassembled.cuh"
#include "kernels.h"

namespace dgsl {

// threads per CTA of the persistent CG (one matrix row per thread in a tile)
constexpr int kCgThreads = 128;

template <typename T, typename V>
struct CGParams {
  const T* vals;
  const int32_t* cols;
  const double* area;
  const double* Mref;
  int ne;
  int ne_pad;    // row stride of cols (multiple of 4)
  int64_t n;
  V coefK, coefM;
  int mean_zero;
  V* x;          // result (starts at 0)
  V* r0;         // right-hand side on entry; residual buffer 0
  V* vec;        // 6 n: p | r1 | w0 | w1 | s0 | s1
  double* part;  // [max_parts][4]
  int max_parts;
  GridBarrier* bar;
  CGResult* res;
  double stop_rel;
  int max_iters;
  uint64_t timeout_ns;
};

// Grid barrier on a monotonic 64-bit arrival counter: the k-th barrier of a
// launch completes when the counter reaches k * nblocks.  Arrival is a release
// atomic, waiting an acquire load, bounded by timeout_ns (reported through
// b->status).
__device__ __forceinline__ bool grid_sync_epoch(GridBarrier* b, unsigned nblocks, unsigned long long& epoch,
                                                uint64_t timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    const unsigned long long target = epoch * (unsigned long long)nblocks;
    unsigned long long v;
    asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(v) : "l"(&b->count) : "memory");
    int ok = 1;
    if (v + 1 < target) {
      const uint64_t t0 = globaltimer_ns();
      for (unsigned spins = 1;; ++spins) {
        asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(&b->count) : "memory");
        if (v >= target) break;
        if (*((volatile int*)&b->status) != kStatusOk) { ok = 0; break; }
        if ((spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
          atomicCAS(&b->status, kStatusOk, kStatusTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*((volatile int*)&b->status) != kStatusOk) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Grid-wide sum of acc[0..3] (deterministic): every CTA reduces its threads'
// values, publishes them in part[], and arrives; the last CTA to arrive sums
// all partials in CTA order and releases the totals, which the other CTAs
// read as four numbers (instead of every CTA re-reading every partial).
__device__ __forceinline__ bool grid_allreduce4(GridBarrier* b, double* part, unsigned nblocks,
                                                unsigned long long& epoch, uint64_t timeout_ns, double (&acc)[4],
                                                double (&tot)[4]) {
  __shared__ int s_state;  // 1: this CTA arrived last, 0: wait, -1: error
  __shared__ double s_tot[4];
  block_sum<4>(acc);
  ++epoch;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) part[4 * blockIdx.x + i] = acc[i];
    const unsigned long long target = epoch * (unsigned long long)nblocks;
    unsigned long long v;
    asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(v) : "l"(&b->count) : "memory");
    __threadfence();
    s_state = v + 1 == target ? 1 : 0;
  }
  __syncthreads();
  if (s_state == 1) {
    double t[4];
    sum_partials<4>(part, nblocks, t);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        b->total[i] = t[i];
        s_tot[i] = t[i];
      }
      __threadfence();
      asm volatile("st.release.gpu.u64 [%0], %1;" ::"l"(&b->gen), "l"(epoch) : "memory");
    }
  } else if (threadIdx.x == 0) {
    const uint64_t t0 = globaltimer_ns();
    unsigned long long g;
    int st = 0;
    for (unsigned spins = 1;; ++spins) {
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(g) : "l"(&b->gen) : "memory");
      if (g >= epoch) break;
      if (*((volatile int*)&b->status) != kStatusOk) { st = -1; break; }
      if ((spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
        atomicCAS(&b->status, kStatusOk, kStatusTimeout);
        st = -1;
        break;
      }
    }
    if (st == 0)
#pragma unroll
      for (int i = 0; i < 4; ++i) s_tot[i] = __ldcg(&b->total[i]);
    s_state = st;
  }
  __syncthreads();
  const bool ok = s_state >= 0 && *((volatile int*)&b->status) == kStatusOk;
#pragma unroll
  for (int i = 0; i < 4; ++i) tot[i] = s_tot[i];
  __syncthreads();
  return ok;
}

template <typename V>
__device__ __forceinline__ double to_d(V v) { return (double)v; }

// Tile geometry: TT triangles (a multiple of 4; TR = TT N_phi matrix rows, one
// per thread) per tile.  A stage holds the tile's coupling coefficients (NG
// chunks of TR 16-byte vectors, each contiguous in global memory) and its
// column indices (4 chunks of TT int32), all brought in by TMA bulk copies; two
// stages per CTA, at most ~96 KB each.
template <int NPHI, typename T>
struct TileCfg {
  static constexpr int VEC = Pack<T>::VEC;
  static constexpr int NC = 4 * NPHI;
  static constexpr int NG = (NC + VEC - 1) / VEC;
  static constexpr int TT0 = kCgThreads / NPHI;
  static constexpr int TTS = 98304 / (NG * NPHI * 16);
  static constexpr int TT = (TT0 < TTS ? TT0 : TTS) / 4 * 4;
  static constexpr int TR = TT * NPHI;
  static constexpr int COLS = NG * TR * 16;        // byte offset of the indices
  static constexpr int STAGE = COLS + 16 * TT;     // 4 x TT int32
};

// Issue (one thread) the bulk copies of tile `tile`'s couplings into `stage`.
template <int NPHI, typename T>
__device__ __forceinline__ void issue_tile(const T* vals, const int32_t* cols, int64_t n, int ne, int ne_pad,
                                           int tile, unsigned char* stage, uint64_t* bar) {
  using C = TileCfg<NPHI, T>;
  const int tri0 = tile * C::TT;                 // multiple of 4
  const int nt = min(C::TT, ne - tri0);
  const uint32_t bytes = (uint32_t)(nt * NPHI * 16);
  const uint32_t cbytes = (uint32_t)(((nt + 3) / 4) * 16);  // padded rows of cols
  const int64_t row0 = (int64_t)tri0 * NPHI;
  const uint64_t pol = l2_evict_first_policy();   // couplings stream; vectors stay in L2
  fence_proxy_async_smem();
  mbar_expect_tx(bar, bytes * C::NG + 4 * cbytes);
#pragma unroll 1
  for (int g = 0; g < C::NG; ++g)
    bulk_g2s_hint(stage + (size_t)g * C::TR * 16, vals + ((size_t)g * n + row0) * C::VEC, bytes, bar, pol);
#pragma unroll
  for (int b = 0; b < 4; ++b)
    bulk_g2s(stage + C::COLS + b * C::TT * 4, cols + (size_t)b * ne_pad + tri0, cbytes, bar);
}

__device__ __forceinline__ void lds16(const unsigned char* p, double (&v)[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void lds16(const unsigned char* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void lds16_bf16(const unsigned char* p, float (&v)[8]) {
  const uint4 t = *reinterpret_cast<const uint4*>(p);
  const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
template <typename T, int VEC, typename W>
__device__ __forceinline__ void lds_vals(const unsigned char* p, W (&v)[VEC]) {
  if constexpr (sizeof(T) == 2) lds16_bf16(p, v);
  else lds16(p, v);
}

// Per-CTA pipeline state (identical in every thread): tiles are processed in
// a fixed rotation over kStages shared-memory stages; `done` counts the tiles
// this CTA has consumed since launch and `issued` the tiles whose copies were
// issued, so tile g uses stage g % kStages with mbarrier parity (g / kStages) & 1.
constexpr int kStages = 3;
struct StageState {
  unsigned done;
  unsigned issued;
};

template <int NPHI, typename T, typename V>
__device__ __forceinline__ void issue_next(const CGParams<T, V>& a, int tile, unsigned char* stages, uint64_t* mbar,
                                           StageState& st) {
  using C = TileCfg<NPHI, T>;
  const int s = (int)(st.issued % kStages);
  if (threadIdx.x == 0)
    issue_tile<NPHI, T>(a.vals, a.cols, a.n, a.ne, a.ne_pad, tile, stages + (size_t)s * C::STAGE, &mbar[s]);
  ++st.issued;
}

// One fused Chronopoulos-Gear pass over this CTA's tiles.  Reads the "old"
// buffers (ro, wo, so), writes the "new" ones (rn, wn, sn), updates p and x in
// place.  acc receives (r.r, w.r, sum w, sum r) of the new vectors.
// Pipeline, for this CTA's q-th tile of the pass: its couplings and indices
// were copied two tiles ahead (the first two before the pass began, across
// the previous grid barrier); its neighbour values are gathered into
// registers while tile q-1 is computed, then combined into shared memory.
// Returns false if a stage wait timed out.
template <int NPHI, typename T, typename V>
__device__ __forceinline__ bool cg_pass(const CGParams<T, V>& a, V alpha, V beta, V muw, const V* ro, const V* wo,
                                        const V* so, V* rn, V* wn, V* sn, V* p, unsigned char* stages,
                                        uint64_t* mbar, StageState& st, double (&acc)[4]) {
  using C = TileCfg<NPHI, T>;
  constexpr int VEC = C::VEC, NC = C::NC, NG = C::NG, TT = C::TT;
  constexpr int NSV = TT * 4 * NPHI;                 // staged neighbour values per tile
  constexpr int J = (NSV + kCgThreads - 1) / kCgThreads;
  __shared__ V s_rn[2][NSV];                         // r_new of the 4 blocks per triangle
  __shared__ V s_own[2][3][TT * NPHI];               // r_old, w_old - mu, s_old of own rows
  const int64_t n = a.n;
  const int ne = a.ne;
  const int ntiles = (ne + TT - 1) / TT;
  const int nq = ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  V g_rr = V(0), g_wr = V(0), g_w = V(0), g_r = V(0);
  V gr[J], gw[J], gs[J];
  V p_nx = V(0), x_nx = V(0);
  bool ok = true;

  auto stage_of = [&](unsigned g) { return stages + (size_t)(g % kStages) * C::STAGE; };
  auto wait_stage = [&](unsigned g) {
    const bool got = mbar_wait_bounded(&mbar[g % kStages], (g / kStages) & 1u, a.timeout_ns);
    return __syncthreads_and(got) != 0;
  };
  auto load_tile = [&](unsigned g, int tile) {
    // neighbour gather (3 L2 loads per value) and own-row p, x of tile `tile`
    const int tri0 = tile * TT;
    const int nt = min(TT, ne - tri0);
    const int32_t* s_col = reinterpret_cast<const int32_t*>(stage_of(g) + C::COLS);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int i = threadIdx.x + j * kCgThreads;
      if (i < nt * 4 * NPHI) {
        const int tb = i / NPHI, kk = i - tb * NPHI;
        const size_t c = (size_t)s_col[(tb & 3) * TT + (tb >> 2)] * NPHI + kk;
        gr[j] = ldcg(ro + c);
        gw[j] = ldcg(wo + c);
        gs[j] = ldcg(so + c);
      }
    }
    if ((int)threadIdx.x < nt * NPHI) {
      const int64_t row = (int64_t)tri0 * NPHI + threadIdx.x;
      p_nx = ldcg(p + row);
      x_nx = ldcg(a.x + row);
    }
  };
  auto combine = [&](int buf, int tile) {
    const int tri0 = tile * TT;
    const int nt = min(TT, ne - tri0);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int i = threadIdx.x + j * kCgThreads;
      if (i < nt * 4 * NPHI) {
        const int tb = i / NPHI, kk = i - tb * NPHI;
        const V w1 = gw[j] - muw;
        s_rn[buf][i] = fma(-alpha, fma(beta, gs[j], w1), gr[j]);
        if ((tb & 3) == 0) {
          const int lr = (tb >> 2) * NPHI + kk;
          s_own[buf][0][lr] = gr[j];
          s_own[buf][1][lr] = w1;
          s_own[buf][2][lr] = gs[j];
        }
      }
    }
  };

  if (nq > 0) {
    // tile 0: its copy is in flight since before the pass
    if (!wait_stage(st.done)) return false;
    load_tile(st.done, (int)blockIdx.x);
    combine(0, (int)blockIdx.x);
    __syncthreads();
  }
  for (int q = 0; q < nq; ++q) {
    const int tile = (int)blockIdx.x + q * (int)gridDim.x;
    const unsigned g = st.done;  // global index of tile q
    if (q + 2 < nq) issue_next<NPHI, T, V>(a, tile + 2 * (int)gridDim.x, stages, mbar, st);
    const V p_old = p_nx, x_old = x_nx;
    const bool more = q + 1 < nq;
    if (more) {
      if (!wait_stage(g + 1)) {
        ok = false;
        break;
      }
      load_tile(g + 1, tile + (int)gridDim.x);  // in flight while tile q is computed
    }
    const int tri0 = tile * TT;
    const int nt = min(TT, ne - tri0);
    const int lt = threadIdx.x / NPHI, k = threadIdx.x - lt * NPHI;
    const int buf = q & 1;
    if ((int)threadIdx.x < nt * NPHI) {
      const int64_t row = (int64_t)tri0 * NPHI + threadIdx.x;
      const unsigned char* sv = stage_of(g) + (size_t)threadIdx.x * 16;
      const V* xs = s_rn[buf] + lt * 4 * NPHI;
      V wv = V(0);
#pragma unroll
      for (int gg = 0; gg < NG; ++gg) {
        typename ValOf<T>::type v[VEC];
        lds_vals<T, VEC>(sv + (size_t)gg * C::TR * 16, v);
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          const int c = gg * VEC + u;
          if (c < NC) wv = fma((V)v[u], xs[c], wv);
        }
      }
      wv *= a.coefK;
      if (a.coefM != V(0)) {
        V mv = V(0);
#pragma unroll
        for (int kk = 0; kk < NPHI; ++kk) mv = fma((V)__ldg(a.Mref + k * NPHI + kk), xs[kk], mv);
        wv = fma(a.coefM * (V)__ldg(a.area + tri0 + lt), mv, wv);
      }
      const V r_old = s_own[buf][0][threadIdx.x];
      const V w_old = s_own[buf][1][threadIdx.x];
      const V s_old = s_own[buf][2][threadIdx.x];
      const V p_new = fma(beta, p_old, r_old);
      const V s_new = fma(beta, s_old, w_old);
      a.x[row] = fma(alpha, p_new, x_old);
      const V r_new = xs[k];
      p[row] = p_new;
      sn[row] = s_new;
      rn[row] = r_new;
      wn[row] = wv;
      g_rr = fma(r_new, r_new, g_rr);
      g_wr = fma(wv, r_new, g_wr);
      g_w += wv;
      g_r += r_new;
    }
    if (more) combine(buf ^ 1, tile + (int)gridDim.x);
    __syncthreads();
    ++st.done;
  }
  if (ok && nq > 0) {
    // the couplings are constant: the next pass's first two tiles are copied now,
    // overlapping the grid barrier
    issue_next<NPHI, T, V>(a, (int)blockIdx.x, stages, mbar, st);
    if (nq > 1) issue_next<NPHI, T, V>(a, (int)blockIdx.x + (int)gridDim.x, stages, mbar, st);
  }
  acc[0] = to_d(g_rr);
  acc[1] = to_d(g_wr);
  acc[2] = to_d(g_w);
  acc[3] = to_d(g_r);
  return ok;
}

template <int NPHI, typename T, typename V>
__global__ void __launch_bounds__(kCgThreads, 1) k_cg(CGParams<T, V> a) {
  extern __shared__ __align__(128) unsigned char stages[];
  __shared__ __align__(8) uint64_t mbar[kStages];
  const unsigned nb = gridDim.x;
  unsigned long long epoch = 0;
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  V* p = a.vec;
  V* const r0b = a.r0;
  V* const r1b = a.vec + n;
  V* const w0b = a.vec + 2 * n;
  V* const w1b = a.vec + 3 * n;
  V* const s0b = a.vec + 4 * n;
  V* const s1b = a.vec + 5 * n;
  double* part = a.part;
  int it = 0;
  double rr = 0.0, rr0 = 0.0, tot[4];
  StageState st;
  st.done = 0u;
  st.issued = 0u;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&mbar[i], 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  {
    // the first two tiles' couplings load while the prologue runs
    using Cfg = TileCfg<NPHI, T>;
    const int ntiles = (a.ne + Cfg::TT - 1) / Cfg::TT;
    if ((int)blockIdx.x < ntiles) issue_next<NPHI, T, V>(a, (int)blockIdx.x, stages, mbar, st);
    if ((int)blockIdx.x + (int)gridDim.x < ntiles)
      issue_next<NPHI, T, V>(a, (int)blockIdx.x + (int)gridDim.x, stages, mbar, st);
  }
  // prologue: mean of r0; x = p = w = s = 0
  {
    V s = V(0);
    for (int64_t row = t0; row < n; row += stride) {
      s += r0b[row];
      a.x[row] = V(0);
      p[row] = V(0);
      w0b[row] = V(0);
      s0b[row] = V(0);
    }
    double acc[4] = {to_d(s), 0.0, 0.0, 0.0};
    if (!grid_allreduce4(a.bar, part, nb, epoch, a.timeout_ns, acc, tot)) goto done;
  }
  if (a.mean_zero) {
    const V mu = (V)(tot[0] / (double)n);
    for (int64_t row = t0; row < n; row += stride) r0b[row] -= mu;
  }
  if (!grid_sync_epoch(a.bar, nb, epoch, a.timeout_ns)) goto done;
  {
    V alpha = V(0), beta = V(0), muw = V(0);
    double g_old = 0.0, a_old = 0.0, stop = 0.0;
    int cur = 0;
    for (int pass = 0;; ++pass) {
      double acc[4];
      const bool ok = cur == 0
          ? cg_pass<NPHI, T, V>(a, alpha, beta, muw, r0b, w0b, s0b, r1b, w1b, s1b, p, stages, mbar, st, acc)
          : cg_pass<NPHI, T, V>(a, alpha, beta, muw, r1b, w1b, s1b, r0b, w0b, s0b, p, stages, mbar, st, acc);
      if (!ok) {
        if (threadIdx.x == 0) atomicCAS(&a.bar->status, kStatusOk, kStatusTimeout);
        goto done;
      }
      if (!grid_allreduce4(a.bar, part, nb, epoch, a.timeout_ns, acc, tot)) goto done;
      cur ^= 1;
      const double g = tot[0];
      const double mu = a.mean_zero ? tot[2] / (double)n : 0.0;
      const double d = tot[1] - mu * tot[3];  // (w - mu 1) . r
      rr = g;
      double an, bn;
      if (pass == 0) {
        rr0 = g;
        stop = a.stop_rel * a.stop_rel * rr0;
        bn = 0.0;
        an = g / d;
      } else {
        ++it;
        bn = g / g_old;
        an = g / (d - bn * g / a_old);
      }
      if (!(g > stop) || it >= a.max_iters || !(an > 0.0) || !isfinite(an)) break;
      g_old = g;
      a_old = an;
      alpha = (V)an;
      beta = (V)bn;
      muw = (V)mu;
    }
  }
done:
  // no CTA leaves with a bulk copy still writing its shared memory
  if (threadIdx.x == 0)
    for (unsigned g = st.done; g < st.issued; ++g)
      if (!mbar_wait_bounded(&mbar[g % kStages], (g / kStages) & 1u, a.timeout_ns))
        atomicCAS(&a.bar->status, kStatusOk, kStatusTimeout);
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.res->iters = it;
    a.res->rr0 = rr0;
    a.res->rr = rr;
    a.res->status = *((volatile int*)&a.bar->status);
  }
}

// Self-test of the bounded waits: `which` = 0 runs the grid barrier of this
// file expecting one CTA more than the launch has; 1 waits on an mbarrier no
// copy will complete.  Both waits must give up after timeout_ns, record
// kStatusTimeout in bar->status and return, leaving the context usable.
__global__ void k_selftest_wait(GridBarrier* bar, int which, uint64_t timeout_ns) {
  __shared__ __align__(8) uint64_t mb;
  if (which == 0) {
    unsigned long long epoch = 0;
    grid_sync_epoch(bar, gridDim.x + 1, epoch, timeout_ns);
  } else {
    if (threadIdx.x == 0) {
      mbar_init(&mb, 1);
      fence_proxy_async_smem();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&mb, 0u, timeout_ns)) atomicCAS(&bar->status, kStatusOk, kStatusTimeout);
    __syncthreads();
  }
}

cudaError_t launch_selftest_wait(GridBarrier* bar, int which, uint64_t timeout_ns, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  if (err != cudaSuccess) return err;
  k_selftest_wait<<<which == 0 ? 2 : 1, 64, 0, s>>>(bar, which, timeout_ns);
  count_launch();
  return cudaGetLastError();
}

namespace {
template <class KernelT>
int coop_blocks(KernelT kern, size_t dyn_smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kCgThreads, dyn_smem);
  per = std::max(1, std::min(per, 8));
  return sms * per;
}

template <int NPHI, typename T, typename V>
cudaError_t run_cg(const DevOp& op, const T* vals, V coefK, V coefM, int mean_zero, V* x, V* r, double stop_rel,
                   int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s, int* grid_used) {
  auto kern = k_cg<NPHI, T, V>;
  using Cfg = TileCfg<NPHI, T>;
  const size_t dyn = kStages * (size_t)Cfg::STAGE;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (err != cudaSuccess) return err;
  const int ntiles = (op.ne + Cfg::TT - 1) / Cfg::TT;
  int blocks = std::min(coop_blocks(kern, dyn), w.max_parts);
  blocks = std::max(1, std::min(blocks, ntiles));
  if (grid_used) *grid_used = blocks;
  CGParams<T, V> a;
  a.vals = vals;
  a.cols = op.cols;
  a.area = op.area;
  a.Mref = op.Mref;
  a.ne = op.ne;
  a.ne_pad = op.ne_pad;
  a.n = op.n;
  a.coefK = coefK;
  a.coefM = coefM;
  a.mean_zero = mean_zero;
  a.x = x;
  a.r0 = r;
  a.vec = static_cast<V*>(w.vec);
  a.part = w.part;
  a.max_parts = w.max_parts;
  a.bar = w.bar;
  a.res = w.res;
  a.stop_rel = stop_rel;
  a.max_iters = max_iters;
  a.timeout_ns = timeout_ns;
  err = cudaMemsetAsync(w.bar, 0, sizeof(GridBarrier), s);
  if (err != cudaSuccess) return err;
  void* args[] = {&a};
  err = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kCgThreads), args, dyn, s);
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
  return sms * 8;
}

#define DGSL_CG_CASES(T, V, VALS)                                                                              \
  switch (op.p) {                                                                                              \
    case 1: return run_cg<3, T, V>(op, VALS, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);  \
    case 2: return run_cg<6, T, V>(op, VALS, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used);  \
    case 3: return run_cg<10, T, V>(op, VALS, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used); \
    case 4: return run_cg<15, T, V>(op, VALS, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w, timeout_ns, s, grid_used); \
  }                                                                                                            \
  return cudaErrorInvalidValue;

cudaError_t launch_cg_f64(const DevOp& op, double coefK, double coefM, int mean_zero, double* x, double* r,
                          double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s,
                          int* grid_used) {
  if (!op.K64) return cudaErrorInvalidValue;
  DGSL_CG_CASES(double, double, op.K64)
}

cudaError_t launch_cg_f32(const DevOp& op, int bf16, float coefK, float coefM, int mean_zero, float* x, float* r,
                          double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s,
                          int* grid_used) {
  if (bf16) {
    if (!op.K16) return cudaErrorInvalidValue;
    DGSL_CG_CASES(uint16_t, float, op.K16)
  }
  if (!op.K32) return cudaErrorInvalidValue;
  DGSL_CG_CASES(float, float, op.K32)
}

}  // namespace dgsl
