// Batched persistent solver engine of dgsl: many independent Schur / Helmholtz
// solves (different meshes, degrees and sizes) iterated by one cooperative
// launch, each with its own FP64 iterative refinement around an FP32 (or BF16-
// coupling) Chronopoulos-Gear CG, as dgsl_cg_solve does for one solve.
//
// A slot is one solve.  Each grid pass processes the chunks (contiguous groups
// of triangles) of every active slot according to that slot's phase; the CTA
// that finishes a slot's last chunk of the pass sums the slot's per-chunk
// partials in chunk order (deterministic) and advances the slot's state
// machine:
//   BSUM   sum b, sum b^2; x = 0
//   RESID  r64 = (b - mean b) - A64 x  (FP64 couplings), sum r^2
//   SCALE  r = r64 / ||r64|| in FP32; CG vectors = 0; sum r
//   PROJ   r -= mean r (periodic pressure operator)
//   CG     fused Chronopoulos-Gear pass (as in k_cg.cu), sums (r.r, w.r, sum w, sum r)
//   UPDATE x += ||r64|| d  (FP64), then RESID again
//   XSUM / XFIX  final mean removal (pressure), then DONE
// One grid barrier per pass serves all slots.  At every barrier the last CTA
// to arrive rebuilds the list of active chunks and admits slots the host has
// published in a mapped inbox since the previous pass, so requests that arrive
// while the kernel runs join at the next pass (continuous batching).  Completion
// records are written to host-mapped memory.  Every wait is bounded.
#include <cuda_bf16.h>

#include "kassembled.cuh"
#include "kbatch.h"
#include "kernels.h"

namespace dgsl {

constexpr int kBThreads = 128;

// ---------------------------------------------------------------- state
enum : int { PH_BSUM = 0, PH_RESID, PH_SCALE, PH_PROJ, PH_CG, PH_UPDATE, PH_XSUM, PH_XFIX, PH_DONE };

struct BState {                    // kernel-owned, one per slot (device memory)
  unsigned long long arrivals;     // chunk completions (monotonic)
  unsigned long long target;       // arrivals that complete the current pass
  int phase, iters, refinements, inner, status, stall, cur, first;
  double bmean, bnorm, rnorm, relres, best, scale, rmean, xmean;
  double alpha, beta, muw, g_old, a_old, stop, stop_rel;
};

struct EngineShared {              // device memory, zeroed before each launch
  unsigned long long count;        // barrier arrivals
  unsigned long long gen;          // last released barrier epoch
  int status;
  int n_act;                       // active slots in the list
  int total_chunks;                // chunks of the active slots
  int admitted;                    // slots admitted so far (copied from the inbox)
  int list_dirty;
  int exit_now;
  int pad[2];
};

// Barrier whose last arriving CTA runs `hook` (whole CTA) before releasing the
// others; bounded waits as in k_cg.cu.  Returns false on timeout / error.
template <class Hook>
__device__ __forceinline__ bool grid_sync_hook(EngineShared* e, unsigned nblocks, unsigned long long& epoch,
                                               uint64_t timeout_ns, Hook hook) {
  __shared__ int s_last;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    unsigned long long v;
    asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(v) : "l"(&e->count) : "memory");
    s_last = v + 1 == epoch * (unsigned long long)nblocks ? 1 : 0;
  }
  __syncthreads();
  int ok = 1;
  if (s_last) {
    hook();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      asm volatile("st.release.gpu.u64 [%0], %1;" ::"l"(&e->gen), "l"(epoch) : "memory");
    }
  } else if (threadIdx.x == 0) {
    const uint64_t t0 = globaltimer_ns();
    for (unsigned spins = 1;; ++spins) {
      unsigned long long g;
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(g) : "l"(&e->gen) : "memory");
      if (g >= epoch) break;
      if (*((volatile int*)&e->status) != kStatusOk) break;
      if ((spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
        atomicCAS(&e->status, kStatusOk, kStatusTimeout);
        break;
      }
    }
  }
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = *((volatile int*)&e->status) == kStatusOk;
  __syncthreads();
  ok = s_ok;
  return ok != 0;
}


// ---------------------------------------------------------------- chunk work

// CG tile geometry for the engine (kBThreads rows per tile), as in k_cg.cu.
template <int NPHI, typename T>
struct BTile {
  static constexpr int VEC = Pack<T>::VEC;
  static constexpr int NC = 4 * NPHI;
  static constexpr int NG = (NC + VEC - 1) / VEC;
  static constexpr int TT = (kBThreads / NPHI) / 4 * 4;
  static constexpr int TR = TT * NPHI;
  static constexpr int COLS = NG * TR * 16;
  static constexpr int STAGE = COLS + 16 * TT;
};

// Per-slot scalars a chunk needs, read once per chunk (L2-coherent loads).
struct ChunkCtx {
  int phase, cur, mean_zero;
  double bmean, scale, rmean, rnorm, xmean, alpha, beta, muw;
};

__device__ __forceinline__ ChunkCtx load_ctx(const BSlotDesc& d, const BState* st) {
  ChunkCtx c;
  c.phase = __ldcg(&st->phase);
  c.cur = __ldcg(&st->cur);
  c.mean_zero = d.mean_zero;
  c.bmean = __ldcg(&st->bmean);
  c.scale = __ldcg(&st->scale);
  c.rmean = __ldcg(&st->rmean);
  c.rnorm = __ldcg(&st->rnorm);
  c.xmean = __ldcg(&st->xmean);
  c.alpha = __ldcg(&st->alpha);
  c.beta = __ldcg(&st->beta);
  c.muw = __ldcg(&st->muw);
  return c;
}

// Streaming phases over rows [r0, r1) of one slot.
template <int NPHI>
__device__ __forceinline__ void stream_chunk(const BSlotDesc& d, const ChunkCtx& c, int64_t r0, int64_t r1,
                                             double (&acc)[4]) {
  const int64_t n = d.n;
  float* fr0 = d.fvec;
  float* fd = d.fvec + n;
  float* fp = d.fvec + 2 * n;
  float* fw0 = d.fvec + 4 * n;
  float* fs0 = d.fvec + 6 * n;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    switch (c.phase) {
      case PH_BSUM: {
        const double v = __ldg(d.b + row);
        acc[0] += v;
        acc[1] = fma(v, v, acc[1]);
        d.x[row] = 0.0;
        break;
      }
      case PH_RESID: {
        const double* K = d.K64;
        double ax = d.coefK * assembled_row<NPHI, double, double, true>(K, d.cols, d.ne_pad, n, row, d.x);
        if (d.coefM != 0.0) ax += d.coefM * mass_row<NPHI, double, true>(d.area, d.Mref, row, d.x);
        const double v = (__ldg(d.b + row) - c.bmean) - ax;
        d.r64[row] = v;
        acc[0] = fma(v, v, acc[0]);
        acc[1] += v;
        break;
      }
      case PH_SCALE: {
        const float v = (float)(__ldcg(d.r64 + row) * c.scale);
        fr0[row] = v;
        fd[row] = 0.f;
        fp[row] = 0.f;
        fw0[row] = 0.f;
        fs0[row] = 0.f;
        acc[0] += (double)v;
        break;
      }
      case PH_PROJ:
        fr0[row] = __ldcg(fr0 + row) - (float)c.rmean;
        break;
      case PH_UPDATE:
        d.x[row] = fma(c.rnorm, (double)__ldcg(fd + row), __ldcg(d.x + row));
        break;
      case PH_XSUM:
        acc[0] += __ldcg(d.x + row);
        break;
      case PH_XFIX:
        d.x[row] = __ldcg(d.x + row) - c.xmean;
        break;
      default:
        break;
    }
  }
}

struct BStages {
  int cur;
  unsigned ph[2];
  int pend[2];
};

template <int NPHI, typename T>
__device__ __forceinline__ void b_issue(const BSlotDesc& d, int tri0, int nt, unsigned char* stage, uint64_t* bar) {
  using C = BTile<NPHI, T>;
  const uint32_t bytes = (uint32_t)(nt * NPHI * 16);
  const uint32_t cbytes = (uint32_t)(((nt + 3) / 4) * 16);
  const int64_t row0 = (int64_t)tri0 * NPHI;
  const T* vals = static_cast<const T*>(d.Kin);
  const uint64_t pol = l2_evict_first_policy();
  fence_proxy_async_smem();
  mbar_expect_tx(bar, bytes * C::NG + 4 * cbytes);
#pragma unroll 1
  for (int g = 0; g < C::NG; ++g)
    bulk_g2s_hint(stage + (size_t)g * C::TR * 16, vals + ((size_t)g * d.n + row0) * C::VEC, bytes, bar, pol);
#pragma unroll
  for (int b = 0; b < 4; ++b) bulk_g2s(stage + C::COLS + b * C::TT * 4, d.cols + (size_t)b * d.ne_pad + tri0, cbytes, bar);
}

template <typename T, int VEC>
__device__ __forceinline__ void b_lds(const unsigned char* p, float (&v)[VEC]) {
  if constexpr (sizeof(T) == 2) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      v[2 * i] = __uint_as_float(w[i] << 16);
      v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
}

// One Chronopoulos-Gear pass over triangles [t0, t1) of one slot (t0 and the
// tile size are multiples of 4), tiles double-buffered through the stages.
template <int NPHI, typename T>
__device__ __forceinline__ bool cg_chunk(const BSlotDesc& d, const ChunkCtx& c, int t0, int t1, unsigned char* stages,
                                         uint64_t* mbar, BStages& st, uint64_t timeout_ns, double (&acc)[4]) {
  using C = BTile<NPHI, T>;
  constexpr int VEC = C::VEC, NC = C::NC, NG = C::NG, TT = C::TT;
  __shared__ float s_rn[TT * 4 * NPHI];
  const int64_t n = d.n;
  float* const fb = d.fvec;
  const float* ro = fb + (c.cur ? 3 : 0) * n;
  const float* wo = fb + (c.cur ? 5 : 4) * n;
  const float* so = fb + (c.cur ? 7 : 6) * n;
  float* rn = fb + (c.cur ? 0 : 3) * n;
  float* wn = fb + (c.cur ? 4 : 5) * n;
  float* sn = fb + (c.cur ? 6 : 7) * n;
  float* p = fb + 2 * n;
  float* xd = fb + n;
  const float alpha = (float)c.alpha, beta = (float)c.beta, muw = (float)c.muw;
  const float coefK = (float)d.coefK, coefM = (float)d.coefM;
  float g_rr = 0.f, g_wr = 0.f, g_w = 0.f, g_r = 0.f;
  if (t0 < t1) {
    if (threadIdx.x == 0) b_issue<NPHI, T>(d, t0, min(TT, t1 - t0), stages + (size_t)st.cur * C::STAGE, &mbar[st.cur]);
    st.pend[st.cur] = 1;
  }
  bool ok = true;
  for (int tri0 = t0; tri0 < t1; tri0 += TT) {
    const int nt = min(TT, t1 - tri0);
    if (tri0 + TT < t1) {
      if (threadIdx.x == 0)
        b_issue<NPHI, T>(d, tri0 + TT, min(TT, t1 - tri0 - TT), stages + (size_t)(st.cur ^ 1) * C::STAGE, &mbar[st.cur ^ 1]);
      st.pend[st.cur ^ 1] = 1;
    }
    const int lt = threadIdx.x / NPHI, k = threadIdx.x - lt * NPHI;
    const bool active = threadIdx.x < nt * NPHI;
    const int64_t row = (int64_t)tri0 * NPHI + threadIdx.x;
    float r_old = 0.f, w_old = 0.f, s_old = 0.f, p_old = 0.f, x_old = 0.f;
    if (active) {
      r_old = __ldcg(ro + row);
      w_old = __ldcg(wo + row) - muw;
      s_old = __ldcg(so + row);
      p_old = __ldcg(p + row);
      x_old = __ldcg(xd + row);
    }
    const bool got = mbar_wait_bounded(&mbar[st.cur], st.ph[st.cur], timeout_ns);
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    st.ph[st.cur] ^= 1u;
    st.pend[st.cur] = 0;
    const unsigned char* stage = stages + (size_t)st.cur * C::STAGE;
    const int32_t* s_col = reinterpret_cast<const int32_t*>(stage + C::COLS);
    for (int i = threadIdx.x; i < nt * 4 * NPHI; i += blockDim.x) {
      const int tb = i / NPHI, kk = i - tb * NPHI;
      const size_t cidx = (size_t)s_col[(tb & 3) * TT + (tb >> 2)] * NPHI + kk;
      s_rn[i] = fmaf(-alpha, fmaf(beta, __ldcg(so + cidx), __ldcg(wo + cidx) - muw), __ldcg(ro + cidx));
    }
    __syncthreads();
    if (active) {
      const unsigned char* sv = stage + (size_t)threadIdx.x * 16;
      const float* xs = s_rn + lt * 4 * NPHI;
      float wv = 0.f;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        float v[VEC];
        b_lds<T, VEC>(sv + (size_t)g * C::TR * 16, v);
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          const int cc = g * VEC + u;
          if (cc < NC) wv = fmaf(v[u], xs[cc], wv);
        }
      }
      wv *= coefK;
      if (coefM != 0.f) {
        float mv = 0.f;
#pragma unroll
        for (int kk = 0; kk < NPHI; ++kk) mv = fmaf((float)__ldg(d.Mref + k * NPHI + kk), xs[kk], mv);
        wv = fmaf(coefM * (float)__ldg(d.area + tri0 + lt), mv, wv);
      }
      const float p_new = fmaf(beta, p_old, r_old);
      const float s_new = fmaf(beta, s_old, w_old);
      xd[row] = fmaf(alpha, p_new, x_old);
      const float r_new = xs[k];
      p[row] = p_new;
      sn[row] = s_new;
      rn[row] = r_new;
      wn[row] = wv;
      g_rr = fmaf(r_new, r_new, g_rr);
      g_wr = fmaf(wv, r_new, g_wr);
      g_w += wv;
      g_r += r_new;
    }
    __syncthreads();
    st.cur ^= 1;
  }
  acc[0] += g_rr;
  acc[1] += g_wr;
  acc[2] += g_w;
  acc[3] += g_r;
  return ok;
}


// ---------------------------------------------------------------- slot transitions

__device__ __forceinline__ void complete_slot(const EngineParams& E, int sid, const BSlotDesc& d, BState* st) {
  BCompletion* c = &E.done[sid];
  c->status = st->status;
  c->iters = st->iters;
  c->refinements = st->refinements;
  c->relres = st->relres;
  c->ticket = d.ticket;
  __threadfence_system();
  *((volatile int*)&c->done) = 1;
  __threadfence_system();
  E.sh->list_dirty = 1;
}

// Advances slot `sid` after a pass, from the slot's summed partials (thread 0).
__device__ __noinline__ void slot_transition(const EngineParams& E, int sid, const BSlotDesc& d, const double (&t)[4]) {
  BState* st = &E.state[sid];
  volatile BState* vs = st;
  const double n = (double)d.n;
  const int mz = d.mean_zero;
  int ph = vs->phase;
  switch (ph) {
    case PH_BSUM: {
      const double bm = mz ? t[0] / n : 0.0;
      const double bn2 = mz ? fmax(0.0, t[1] - n * bm * bm) : t[1];
      st->bmean = bm;
      st->bnorm = sqrt(bn2);
      st->best = INFINITY;
      if (!(bn2 > 0.0)) {
        st->relres = 0.0;
        st->status = 0;
        st->phase = PH_DONE;
        complete_slot(E, sid, d, st);
      } else {
        st->phase = PH_RESID;
      }
      break;
    }
    case PH_RESID: {
      const double rn = sqrt(t[0]);
      const double rel = rn / vs->bnorm;
      st->rnorm = rn;
      st->relres = rel;
      int fin = 0, status = 0;
      if (rel <= d.tol) {
        fin = 1;
      } else if (vs->iters >= d.max_iters || vs->refinements >= d.max_refine) {
        fin = 1;
        status = 5;  // DGSL_ENOTCONV
      } else if (rel < 0.9 * vs->best) {
        st->best = rel;
        st->stall = 0;
      } else if (vs->stall + 1 >= 3) {
        fin = 1;
        status = 5;
      } else {
        st->stall = vs->stall + 1;
      }
      if (fin) {
        st->status = status;
        st->phase = mz ? PH_XSUM : PH_DONE;
        if (!mz) complete_slot(E, sid, d, st);
      } else {
        st->stop_rel = fmin(1.0, fmax(d.inner_tol, 0.5 * d.tol / rel));
        st->scale = 1.0 / rn;
        st->phase = PH_SCALE;
      }
      break;
    }
    case PH_SCALE:
      st->rmean = mz ? t[0] / n : 0.0;
      st->phase = PH_PROJ;
      break;
    case PH_PROJ:
      st->first = 1;
      st->cur = 0;
      st->alpha = 0.0;
      st->beta = 0.0;
      st->muw = 0.0;
      st->phase = PH_CG;
      break;
    case PH_CG: {
      const double g = t[0];
      const double mu = mz ? t[2] / n : 0.0;
      const double dd = t[1] - mu * t[3];
      double an, bn;
      int iters = vs->iters;
      if (vs->first) {
        st->stop = vs->stop_rel * vs->stop_rel * g;
        st->first = 0;
        bn = 0.0;
        an = g / dd;
      } else {
        ++iters;
        bn = g / vs->g_old;
        an = g / (dd - bn * g / vs->a_old);
      }
      st->iters = iters;
      st->cur = vs->cur ^ 1;
      if (!(g > vs->stop) || iters >= d.max_iters || !(an > 0.0) || !isfinite(an)) {
        st->phase = PH_UPDATE;
      } else {
        st->alpha = an;
        st->beta = bn;
        st->muw = mu;
        st->g_old = g;
        st->a_old = an;
      }
      break;
    }
    case PH_UPDATE:
      st->refinements = vs->refinements + 1;
      st->phase = PH_RESID;
      break;
    case PH_XSUM:
      st->xmean = t[0] / n;
      st->phase = PH_XFIX;
      break;
    case PH_XFIX:
      st->phase = PH_DONE;
      complete_slot(E, sid, d, st);
      break;
    default:
      break;
  }
  __threadfence();
}

// ---------------------------------------------------------------- barrier hook

__device__ __forceinline__ void copy_desc(BSlotDesc* dst, const BSlotDesc* src) {
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* o = reinterpret_cast<unsigned long long*>(dst);
  constexpr int W = (int)(sizeof(BSlotDesc) / 8);
  for (int i = threadIdx.x; i < W; i += blockDim.x) o[i] = *((volatile const unsigned long long*)(s + i));
}

// Admission of newly published slots and rebuild of the active-chunk list
// (whole CTA of the last arriver).
__device__ __noinline__ void engine_hook(const EngineParams& E) {
  __shared__ int s_count, s_adm, s_dirty, s_run[kBThreads];
  EngineShared* sh = E.sh;
  if (threadIdx.x == 0) {
    s_adm = *((volatile int*)&sh->admitted);
    int cnt = *((volatile int*)&E.inbox->count);
    __threadfence_system();
    s_count = min(cnt, kMaxSlots);
    s_dirty = *((volatile int*)&sh->list_dirty);
  }
  __syncthreads();
  for (int i = s_adm; i < s_count; ++i) {
    copy_desc(&E.slots[i], &E.inbox->slots[i]);
    if (threadIdx.x == 0) {
      BState z = {};
      z.phase = PH_BSUM;
      E.state[i] = z;
    }
  }
  __syncthreads();
  if (s_count > s_adm || s_dirty) {
    // active slots in slot order, chunk offsets by a block scan; each thread
    // owns PER consecutive slots and reads their state twice (count, write)
    constexpr int PER = kMaxSlots / kBThreads;
    int cnt = 0, chunks = 0;
    for (int j = 0; j < PER; ++j) {
      const int sidx = threadIdx.x * PER + j;
      if (sidx < s_count && __ldcg(&E.state[sidx].phase) != PH_DONE) {
        ++cnt;
        chunks += __ldcg(&E.slots[sidx].nchunk);
      }
    }
    s_run[threadIdx.x] = cnt;
    __shared__ int s_runc[kBThreads];
    s_runc[threadIdx.x] = chunks;
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive scans (kBThreads entries)
      int a = 0, b = 0;
      for (int i = 0; i < kBThreads; ++i) {
        const int ta = s_run[i], tb = s_runc[i];
        s_run[i] = a;
        s_runc[i] = b;
        a += ta;
        b += tb;
      }
      sh->n_act = a;
      sh->total_chunks = b;
      E.act_chunk0[a] = b;
    }
    __syncthreads();
    int k = s_run[threadIdx.x], c0 = s_runc[threadIdx.x];
    for (int j = 0; j < PER; ++j) {
      const int sidx = threadIdx.x * PER + j;
      if (sidx < s_count && __ldcg(&E.state[sidx].phase) != PH_DONE) {
        E.act_slot[k] = sidx;
        E.act_chunk0[k] = c0;
        ++k;
        c0 += __ldcg(&E.slots[sidx].nchunk);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      sh->admitted = s_count;
      sh->list_dirty = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int exit_now = 0;
    if (*((volatile int*)&sh->n_act) == 0) {
      // idle: wait (bounded) for the host to publish more slots
      const uint64_t t0 = globaltimer_ns();
      exit_now = 1;
      while (globaltimer_ns() - t0 < E.idle_ns) {
        if (*((volatile int*)&E.inbox->stop)) break;
        if (*((volatile int*)&E.inbox->count) > s_count) {
          exit_now = 0;
          break;
        }
        __nanosleep(1000);
      }
    }
    sh->exit_now = exit_now;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- kernel

__device__ __forceinline__ void load_desc(BSlotDesc& d, const BSlotDesc* src) {
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* o = reinterpret_cast<unsigned long long*>(&d);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(BSlotDesc) / 8); ++i) o[i] = __ldcg(s + i);
}

template <typename T, int NPHI>
__device__ __forceinline__ bool chunk_work(const BSlotDesc& d, const ChunkCtx& c, int t0, int t1,
                                           unsigned char* stages, uint64_t* mbar, BStages& st, uint64_t timeout_ns,
                                           double (&acc)[4]) {
  if (c.phase == PH_CG) return cg_chunk<NPHI, T>(d, c, t0, t1, stages, mbar, st, timeout_ns, acc);
  stream_chunk<NPHI>(d, c, (int64_t)t0 * NPHI, (int64_t)t1 * NPHI, acc);
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kBThreads, 4) k_engine(EngineParams E) {
  extern __shared__ __align__(128) unsigned char stages[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_last;
  const unsigned nb = gridDim.x;
  unsigned long long epoch = 0;
  BStages st;
  st.cur = 0;
  st.ph[0] = st.ph[1] = 0u;
  st.pend[0] = st.pend[1] = 0;
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  auto hook = [&E]() { engine_hook(E); };
  if (!grid_sync_hook(E.sh, nb, epoch, E.timeout_ns, hook)) goto done;
  for (;;) {
    if (__ldcg(&E.sh->exit_now)) break;
    const int n_act = __ldcg(&E.sh->n_act);
    const int total = __ldcg(&E.sh->total_chunks);
    // contiguous chunk range per CTA: one search per pass, the slot descriptor
    // is reloaded only when the range crosses into the next slot
    const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
    const int c_begin = min(total, (int)blockIdx.x * per);
    const int c_end = min(total, c_begin + per);
    int k = 0;
    {
      int lo = 0, hi = n_act;  // last k with act_chunk0[k] <= c_begin
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldcg(E.act_chunk0 + mid) <= c_begin) lo = mid; else hi = mid;
      }
      k = lo;
    }
    int cur_sid = -1, chunk0 = 0, next0 = 0;
    // the slot descriptor and its per-pass scalars live in shared memory
    // (registers stay free for the tile loop)
    __shared__ BSlotDesc s_desc;
    __shared__ ChunkCtx s_ctx;
    const BSlotDesc& d = s_desc;
    const ChunkCtx& c = s_ctx;
    for (int cidx = c_begin; cidx < c_end; ++cidx) {
      if (cur_sid < 0 || cidx >= next0) {
        while (k + 1 < n_act && __ldcg(E.act_chunk0 + k + 1) <= cidx) ++k;
        cur_sid = __ldcg(E.act_slot + k);
        chunk0 = __ldcg(E.act_chunk0 + k);
        next0 = __ldcg(E.act_chunk0 + k + 1);
        __syncthreads();
        if (threadIdx.x == 0) {
          load_desc(s_desc, &E.slots[cur_sid]);
          s_ctx = load_ctx(s_desc, &E.state[cur_sid]);
        }
        __syncthreads();
      }
      const int sid = cur_sid;
      const int lc = cidx - chunk0;
      const int t0 = lc * d.chunk_tris;
      const int t1 = min(d.ne, t0 + d.chunk_tris);
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      bool ok = true;
      switch (d.p) {
        case 1: ok = chunk_work<T, 3>(d, c, t0, t1, stages, mbar, st, E.timeout_ns, acc); break;
        case 2: ok = chunk_work<T, 6>(d, c, t0, t1, stages, mbar, st, E.timeout_ns, acc); break;
        case 3: ok = chunk_work<T, 10>(d, c, t0, t1, stages, mbar, st, E.timeout_ns, acc); break;
        default: ok = chunk_work<T, 15>(d, c, t0, t1, stages, mbar, st, E.timeout_ns, acc); break;
      }
      if (!ok) {
        if (threadIdx.x == 0) atomicCAS(&E.sh->status, kStatusOk, kStatusTimeout);
        goto done;
      }
      block_sum<4>(acc);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) d.part[4 * lc + i] = acc[i];
        unsigned long long v;
        asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(v) : "l"(&E.state[sid].arrivals) : "memory");
        s_last = ((v + 1) % (unsigned long long)d.nchunk) == 0ull;
      }
      __syncthreads();
      if (s_last) {
        double tot[4];
        sum_partials<4>(d.part, d.nchunk, tot);
        if (threadIdx.x == 0) slot_transition(E, sid, d, tot);
      }
      __syncthreads();
    }
    if (!grid_sync_hook(E.sh, nb, epoch, E.timeout_ns, hook)) goto done;
  }
done:
  if (threadIdx.x == 0)
    for (int s2 = 0; s2 < 2; ++s2)
      if (st.pend[s2] && !mbar_wait_bounded(&mbar[s2], st.ph[s2], E.timeout_ns))
        atomicCAS(&E.sh->status, kStatusOk, kStatusTimeout);
  __syncthreads();
}

// ---------------------------------------------------------------- host side

int engine_chunk_tris(int p) {
  const int nphi = (p + 1) * (p + 2) / 2;
  const int tt = (kBThreads / nphi) / 4 * 4;
  return tt * 8;  // 8 tiles per chunk
}

size_t engine_state_bytes() {
  return sizeof(BSlotDesc) * kMaxSlots + sizeof(BState) * kMaxSlots + 256 + sizeof(int) * (2 * kMaxSlots + 1) + 1024;
}

void engine_layout(void* base, EngineParams& P) {
  char* p = static_cast<char*>(base);
  auto take = [&p](size_t bytes) {
    char* q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  P.slots = reinterpret_cast<BSlotDesc*>(take(sizeof(BSlotDesc) * kMaxSlots));
  P.state = reinterpret_cast<BState*>(take(sizeof(BState) * kMaxSlots));
  P.sh = reinterpret_cast<EngineShared*>(take(sizeof(EngineShared)));
  P.act_slot = reinterpret_cast<int*>(take(sizeof(int) * kMaxSlots));
  P.act_chunk0 = reinterpret_cast<int*>(take(sizeof(int) * (kMaxSlots + 1)));
}

size_t engine_shared_bytes() { return sizeof(EngineShared); }

int engine_shared_status(const void* sh_host_copy) {
  return static_cast<const EngineShared*>(sh_host_copy)->status;
}
int engine_shared_admitted(const void* sh_host_copy) {
  return static_cast<const EngineShared*>(sh_host_copy)->admitted;
}

template <typename T>
static size_t engine_smem() {
  size_t m = BTile<3, T>::STAGE;
  m = std::max(m, (size_t)BTile<6, T>::STAGE);
  m = std::max(m, (size_t)BTile<10, T>::STAGE);
  m = std::max(m, (size_t)BTile<15, T>::STAGE);
  return 2 * m;
}

template <typename T>
static cudaError_t launch_engine_t(const EngineParams& e, cudaStream_t s, int* grid_used) {
  auto kern = k_engine<T>;
  const size_t dyn = engine_smem<T>();
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBThreads, dyn);
  if (err != cudaSuccess) return err;
  per = std::max(1, std::min(per, 8));
  const int blocks = sms * per;
  if (grid_used) *grid_used = blocks;
  EngineParams a = e;
  void* args[] = {&a};
  err = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kBThreads), args, dyn, s);
  count_launch();
  return err;
}

cudaError_t launch_engine(const EngineParams& e, int bf16, cudaStream_t s, int* grid_used) {
  return bf16 ? launch_engine_t<uint16_t>(e, s, grid_used) : launch_engine_t<float>(e, s, grid_used);
}

}  // namespace dgsl
