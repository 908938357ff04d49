// Device code of the batched persistent solver engine, shared by the two
// translation units that instantiate it: k_batch.cu (plain CG slots) and
// k_batch_pc.cu (kernels that also run block-Jacobi preconditioned slots).
#pragma once
//
// Batched persistent solver engine of dgsl: many independent Schur / Helmholtz
// requests (different meshes, degrees and sizes, each with 1..8 right-hand
// sides) iterated by one cooperative launch, each right-hand side with its own
// FP64 iterative refinement around an FP32 (or BF16-coupling) CG, as
// dgsl_cg_solve does for one solve.
//
// A slot is one request.  Each grid pass processes the chunks (contiguous
// groups of triangles) of every active slot according to that slot's phase;
// the CTA that completes a slot's pass sums the slot's per-chunk partials in
// chunk order (deterministic) and advances the slot's state machine, one lane
// per right-hand side:
//   BSUM   sum b, sum b^2; x = 0
//   RESID  r64 = (b - mean b) - A64 x  (FP64 couplings), sum r^2, sum r
//   SCALE  r = (r64 - mean r64) / ||r64|| in FP32; d = p = w = s = 0
//   CG0, CG  fused Chronopoulos-Gear passes (as in k_cg.cu):
//            p = r + beta p;  s = w' + beta s;  d += alpha p;  r <- r - alpha s;
//            w <- A r;  sums (r.r, w.r, sum w, sum r);
//            beta' = g'/g, alpha' = g' / (dw' - beta' g'/alpha)   (CG0: beta' = 0)
//          (w' = w - mean w for the periodic pressure operator); with the
//          block-Jacobi preconditioner (as in k_cg.cu) p = u' + beta p,
//          w <- (A P) r, u = P_i r on the own block, sums (r.u, w.u, sum w,
//          sum u, r.r, sum r), u' = u - mean u for the pressure operator
//   UPDATE x += ||r64|| d  (FP64), then RESID again
//   XSUM / XFIX  final mean removal (pressure), then DONE
// The right-hand sides of a slot share every coupling tile; a right-hand side
// whose inner CG has stopped, or whose refinement has finished, is frozen
// (alpha = beta = 0 leaves its d and r unchanged), and the tile geometry does
// not depend on the number of right-hand sides, so each one gets the same
// arithmetic, bit for bit, as when solved alone.
//
// CG passes are tiled and warp-specialised as in k_cg.cu: a coupling warp
// streams coupling tiles with TMA bulk copies, a gather warp copies the
// previous r, w, s of the neighbour blocks and the own d, p with cp.async,
// eight consumer warps form the new residual of the gathered blocks and
// compute (the two threads of a matrix row take half of its right-hand sides
// each).  One grid barrier per pass serves all slots.  At every barrier the
// last CTA to arrive rebuilds the list of active chunks and admits slots the
// host has published in a mapped inbox since the previous pass (continuous
// batching).  Completion records are written to host-mapped memory.  Every
// wait is bounded.
#include <algorithm>
#include <cuda_bf16.h>

#include "kassembled.cuh"
#include "kbatch.h"
#include "kernels.h"

namespace dgsl {

constexpr int kERows = 128;                       // matrix rows per tile
constexpr int kEConsumers = 2 * kERows;           // 8 warps: two threads per row share its right-hand sides
constexpr int kECWarps = kEConsumers / 32;
constexpr int kEThreads = kEConsumers + 64;       // + coupling warp + gather warp
constexpr int kECouplingWarp = kECWarps;
constexpr int kEGatherWarp = kECouplingWarp + 1;
constexpr int kEMaxStages = 8;
constexpr int kEDynSmem = 184 * 1024;             // the stage ring; each pass divides it into stages
constexpr int kNV = kEngineSums;                  // partial sums per chunk (4, or 6 preconditioned, per RHS)
// Partials stored per chunk of a slot: 4 per right-hand side, 6 preconditioned.
__host__ __device__ constexpr int e_part_stride(int precond) { return precond ? kNV : 4 * kMaxRhs; }

// ---------------------------------------------------------------- state
enum : int { PH_BSUM = 0, PH_RESID, PH_SCALE, PH_CG0, PH_CG, PH_UPDATE, PH_XSUM, PH_XFIX, PH_DONE };

struct BRhs {                      // per right-hand side (kernel-owned)
  int status, iters, refinements, stall;
  int done;                        // refinement finished (converged or failed)
  int inner;                       // inner CG running in the current refinement step
  double bmean, bnorm, rnorm, rmean, relres, best, xmean, stop;
  float alpha, beta, muw, g_old, a_old, muu;  // muu: mean of u (preconditioned pressure solves)
};

struct BState {                    // kernel-owned, one per slot (device memory)
  unsigned long long arrivals;     // chunk completions (monotonic)
  int phase, cur, pass, pad;
  BRhs rhs[kMaxRhs];
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
  int ring_S, ring_SB;             // stage ring of the next pass (stages, bytes per stage)
};

// Geometry of a tile for degree NPHI and coupling type T (as k_cg.cu), and of
// the per-triangle vector blocks for RP right-hand sides: a block holds
// NPHI x RP values (right-hand side innermost), padded to a multiple of 4
// floats so that every block starts on a 16-byte boundary.
template <int NPHI, typename T>
struct ETile {
  static constexpr int VEC = Pack<T>::VEC;
  static constexpr int NC = 4 * NPHI;
  static constexpr int NG = (NC + VEC - 1) / VEC;
  static constexpr int TT = (kERows / NPHI) / 4 * 4;
  static constexpr int TR = TT * NPHI;
  static constexpr int NB = 4 * TT;
  static constexpr int COUPLE = NG * TR * 16;
};
__host__ __device__ constexpr int e_block_len(int nphi, int rp) { return (nphi * rp + 3) / 4 * 4; }
__host__ __device__ constexpr int e_nphi(int p) { return (p + 1) * (p + 2) / 2; }
__host__ __device__ constexpr int e_tt(int nphi) { return (kERows / nphi) / 4 * 4; }
// Stage byte offsets for (NPHI, T, RP, PRE): couplings | PRE: rows of P (NGP
// chunks of TR 16-byte vectors) | gathered r, w, s of the 4 TT coupled blocks |
// own blocks of d, p (PRE: and u; TT each) | areas (TT doubles).
__host__ __device__ constexpr int e_ngp(int nphi, bool pre) { return pre ? (nphi + 3) / 4 : 0; }
template <int NPHI, typename T, int RP, bool PRE>
struct EStage {
  using C = ETile<NPHI, T>;
  static constexpr int BL = e_block_len(NPHI, RP);
  static constexpr int NGP = e_ngp(NPHI, PRE);
  static constexpr int PBLK = C::COUPLE;
  static constexpr int GATHER = C::COUPLE + NGP * C::TR * 16;
  static constexpr int OWN = GATHER + 3 * C::NB * BL * 4;
  static constexpr int AREA = OWN + (PRE ? 3 : 2) * C::TT * BL * 4;
};
// New-residual values of one tile (4 TT padded blocks) for every degree and RP.
constexpr int kRnMax = 4 * kERows * kMaxRhs;
// Padded right-hand-side count of a slot.
__host__ __device__ inline int e_rp(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : 8; }

// Barrier whose last arriving CTA runs `hook` (whole CTA) before releasing the
// others; bounded waits as in k_cg.cu.  Returns false on timeout / error.
template <class Hook>
__device__ __forceinline__ bool grid_sync_hook(EngineShared* e, unsigned nblocks, unsigned long long& epoch,
                                               uint64_t timeout_ns, Hook hook) {
  __shared__ int s_last;
  __shared__ int s_ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    unsigned long long v;
    asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(v) : "l"(&e->count) : "memory");
    s_last = v + 1 == epoch * (unsigned long long)nblocks ? 1 : 0;
  }
  __syncthreads();
  if (s_last) {
    hook();
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("st.release.gpu.u64 [%0], %1;" ::"l"(&e->gen), "l"(epoch) : "memory");
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
  if (threadIdx.x == 0) s_ok = *((volatile int*)&e->status) == kStatusOk;
  __syncthreads();
  return s_ok != 0;
}

// ---- consumer-only synchronisation (named barrier 1) and async-copy helpers
__device__ __forceinline__ void ecbar() { asm volatile("bar.sync 1, %0;" ::"n"(kEConsumers) : "memory"); }
__device__ __forceinline__ bool ecbar_and(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"((unsigned)v), "n"(kEConsumers)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void e_mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// 16-byte global -> shared copy through L2 only (the CG vectors are rewritten
// by other CTAs during the launch).
__device__ __forceinline__ void e_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// Arrive on `bar` once this thread's earlier cp.async copies have landed.
__device__ __forceinline__ void e_cp_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void e_cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------- chunk work

// What a chunk needs of its slot, copied to shared memory when a CTA's chunk
// range enters the slot (L2-coherent loads).
struct ChunkCtx {
  int phase, cur, rp, bl;
  int done_mask, inner_mask;        // bit r: right-hand side r finished / runs an inner CG
  double bmean[kMaxRhs], scale[kMaxRhs], rmean[kMaxRhs], rnorm[kMaxRhs], xmean[kMaxRhs];
  float alpha[kMaxRhs], beta[kMaxRhs], muw[kMaxRhs], muu[kMaxRhs];
};

// The slot's descriptor and per-pass scalars into shared memory (one warp:
// lane i copies word i of the descriptor and the scalars of right-hand side i).
__device__ __forceinline__ void load_slot(BSlotDesc& d, ChunkCtx& c, const BSlotDesc* src, const BState* st) {
  const int lane = threadIdx.x & 31;
  constexpr int W = (int)(sizeof(BSlotDesc) / 8);
  static_assert(W <= 32, "descriptor words per lane");
  if (lane < W)
    reinterpret_cast<unsigned long long*>(&d)[lane] = __ldcg(reinterpret_cast<const unsigned long long*>(src) + lane);
  int done = 0, inner = 0;
  if (lane < kMaxRhs) {
    const BRhs* q = &st->rhs[lane];
    done = __ldcg(&q->done);
    inner = __ldcg(&q->inner);
    c.bmean[lane] = __ldcg(&q->bmean);
    const double rn = __ldcg(&q->rnorm);
    c.rnorm[lane] = rn;
    c.scale[lane] = rn > 0.0 ? 1.0 / rn : 0.0;
    c.rmean[lane] = __ldcg(&q->rmean);
    c.xmean[lane] = __ldcg(&q->xmean);
    c.alpha[lane] = __ldcg(&q->alpha);
    c.beta[lane] = __ldcg(&q->beta);
    c.muw[lane] = __ldcg(&q->muw);
    c.muu[lane] = __ldcg(&q->muu);
  }
  const unsigned dm = __ballot_sync(0xffffffffu, lane < kMaxRhs && done);
  const unsigned im = __ballot_sync(0xffffffffu, lane < kMaxRhs && inner);
  if (lane == 0) {
    c.phase = __ldcg(&st->phase);
    c.cur = __ldcg(&st->cur);
    c.done_mask = (int)dm;
    c.inner_mask = (int)im;
  }
  __syncwarp();
  if (lane == 0) {
    c.rp = d.rp;
    c.bl = d.bl;
  }
}

// Sum over the consumer threads of v[0..NV) (fixed shuffle tree, then the
// warp sums in order); out[0..NV) in shared memory, valid after the call.
template <int NV, int NR, typename W>
__device__ __forceinline__ void e_reduce(W (&v)[NV], double* out, double (*s_red)[NR]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) s_red[wid][i] = (double)v[i];
  ecbar();
  if ((int)threadIdx.x < NV) {
    const int t = threadIdx.x;
    double a = s_red[0][t];
#pragma unroll
    for (int w = 1; w < kECWarps; ++w) a += s_red[w][t];
    out[t] = a;
  }
  ecbar();
}

// Streaming phases (consumer threads) over triangles [t0, t1) of one slot; the
// chunk's partial sums (4 per right-hand side) go to sums[0..NR).
template <int NPHI, int NR>
__device__ __forceinline__ void stream_chunk(const BSlotDesc& d, const ChunkCtx& c, int t0, int t1, double* sums,
                                             double (*s_red)[NR]) {
  const int64_t n = d.n;
  const int64_t r0 = (int64_t)t0 * NPHI, r1 = (int64_t)t1 * NPHI;
  const int R = d.nrhs, RP = c.rp, BL = c.bl;
  const int64_t L = (int64_t)d.ne * BL;  // floats per padded vector
  if ((int)threadIdx.x < NR) sums[threadIdx.x] = 0.0;
  ecbar();
  if (c.phase == PH_SCALE) {
    // padded, right-hand-side-interleaved FP32 vectors: r0 scaled and projected,
    // d = p = w0 = s0 = 0 (every lane < RP is written, so the unused ones are 0)
    float* fd = d.fvec;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += kEConsumers) {
      const int64_t tri = row / NPHI;
      const int k = (int)(row - tri * NPHI);
      const int64_t base = tri * BL + (int64_t)k * RP;
      for (int r = 0; r < RP; ++r) {
        float v = 0.f;
        if (r < R && ((c.inner_mask >> r) & 1))
          v = (float)((__ldcg(d.r64 + (int64_t)r * n + row) - c.rmean[r]) * c.scale[r]);
        fd[0 * L + base + r] = 0.f;  // d
        fd[1 * L + base + r] = 0.f;  // p
        fd[2 * L + base + r] = v;    // r0
        fd[4 * L + base + r] = 0.f;  // w0
        fd[6 * L + base + r] = 0.f;  // s0
        if (d.precond) fd[8 * L + base + r] = 0.f;  // u
      }
    }
    ecbar();
    return;
  }
  for (int r = 0; r < R; ++r) {
    const bool done = (c.done_mask >> r) & 1;
    const double* b = d.b + (int64_t)r * n;
    double* x = d.x + (int64_t)r * n;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t row = r0 + threadIdx.x; row < r1; row += kEConsumers) {
      switch (c.phase) {
        case PH_BSUM: {
          const double v = __ldg(b + row);
          acc[0] += v;
          acc[1] = fma(v, v, acc[1]);
          x[row] = 0.0;
          break;
        }
        case PH_RESID: {
          if (done) break;
          double ax = d.coefK * assembled_row<NPHI, double, double, true>(d.K64, d.cols, d.ne_pad, n, row, x);
          if (d.coefM != 0.0) ax += d.coefM * mass_row<NPHI, double, true>(d.area, d.Mref, row, x);
          const double v = (__ldg(b + row) - c.bmean[r]) - ax;
          d.r64[(int64_t)r * n + row] = v;
          acc[0] = fma(v, v, acc[0]);
          acc[1] += v;
          break;
        }
        case PH_UPDATE: {
          if (done) break;
          const int64_t tri = row / NPHI;
          const int k = (int)(row - tri * NPHI);
          const float dv = __ldcg(d.fvec + tri * BL + (int64_t)k * RP + r);
          x[row] = fma(c.rnorm[r], (double)dv, __ldcg(x + row));
          break;
        }
        case PH_XSUM:
          acc[0] += __ldcg(x + row);
          break;
        case PH_XFIX:
          x[row] = __ldcg(x + row) - c.xmean[r];
          break;
        default:
          break;
      }
    }
    e_reduce<4, NR, double>(acc, sums + 4 * r, s_red);
  }
}

// RP consecutive floats (16-byte aligned when RP >= 4, 8-byte when RP = 2).
template <int RP>
__device__ __forceinline__ void ld_rp(const float* p, float (&o)[RP]) {
  if constexpr (RP >= 4) {
#pragma unroll
    for (int i = 0; i < RP; i += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + i);
      o[i] = t.x;
      o[i + 1] = t.y;
      o[i + 2] = t.z;
      o[i + 3] = t.w;
    }
  } else if constexpr (RP == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  } else {
    o[0] = *p;
  }
}
template <int RP>
__device__ __forceinline__ void st_rp(float* p, const float (&v)[RP]) {
  if constexpr (RP >= 4) {
#pragma unroll
    for (int i = 0; i < RP; i += 4) *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  } else if constexpr (RP == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    *p = v[0];
  }
}
template <typename T, int VEC>
__device__ __forceinline__ void e_lds(const unsigned char* p, float (&v)[VEC]) {
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

// One Chronopoulos-Gear tile of a slot, RP right-hand sides.  Combine (all
// consumer threads, float4 at a time): the new residual r - alpha (w' + beta s)
// of the 4 TT gathered blocks into rn ([block][BL]).  Then (after the
// caller's barrier) the two threads of each matrix row: w = A r_new, and the
// row updates, each for half of the right-hand sides.
template <int NPHI, typename T, int RP, bool PRE>
__device__ __forceinline__ void cg_combine(const ChunkCtx& c, int nt, const unsigned char* st, float* rn) {
  using C = ETile<NPHI, T>;
  using S = EStage<NPHI, T, RP, PRE>;
  constexpr int BL = S::BL, NB = C::NB, Q = BL / 4;  // float4 per block
  const float4* gr = reinterpret_cast<const float4*>(st + S::GATHER);
  const float4* gw = gr + NB * Q;
  const float4* gs = gw + NB * Q;
  float4* o = reinterpret_cast<float4*>(rn);
  // right-hand-side lanes of a float4: RP = 8 alternates lanes 0-3 / 4-7 within
  // a block, RP = 4 is lanes 0-3, RP = 2 is 0,1,0,1 and RP = 1 is 0,0,0,0
  float al[2][4], be[2][4], mu[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (h * 4 + i) % RP;
      al[h][i] = c.alpha[r];
      be[h][i] = c.beta[r];
      mu[h][i] = c.muw[r];
    }
  for (int f = threadIdx.x; f < nt * 4 * Q; f += kEConsumers) {
    const bool hi = RP == 8 && ((f % Q) & 1);
    float a[4], b[4], m[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {  // selects, not indexing: the patterns stay in registers
      a[i] = hi ? al[1][i] : al[0][i];
      b[i] = hi ? be[1][i] : be[0][i];
      m[i] = hi ? mu[1][i] : mu[0][i];
    }
    const float4 r4 = gr[f], w4 = gw[f], s4 = gs[f];
    float4 x;
    x.x = fmaf(-a[0], fmaf(b[0], s4.x, w4.x - m[0]), r4.x);
    x.y = fmaf(-a[1], fmaf(b[1], s4.y, w4.y - m[1]), r4.y);
    x.z = fmaf(-a[2], fmaf(b[2], s4.z, w4.z - m[2]), r4.z);
    x.w = fmaf(-a[3], fmaf(b[3], s4.w, w4.w - m[3]), r4.w);
    o[f] = x;
  }
}

// Right-hand sides per consumer thread: the two threads of a row (one in each
// half of the consumer warps) take half of the slot's right-hand sides each.
template <int RP>
struct RhsSplit {
  static constexpr int RT = RP >= 2 ? RP / 2 : 1;
};

template <int NPHI, typename T, int RP, bool PRE>
__device__ __forceinline__ void cg_rows(const BSlotDesc& d, const ChunkCtx& c, int tri0, int nt,
                                        const unsigned char* st, const float* rn,
                                        float (&acc)[PRE ? 6 : 4][RhsSplit<RP>::RT]) {
  using C = ETile<NPHI, T>;
  using S = EStage<NPHI, T, RP, PRE>;
  constexpr int BL = S::BL, TT = C::TT, TR = C::TR, NG = C::NG, VEC = C::VEC, NC = C::NC, NB = C::NB;
  constexpr int RT = RhsSplit<RP>::RT;
  const int row = threadIdx.x & (kERows - 1), half = threadIdx.x / kERows;
  if (row >= nt * NPHI || (RP == 1 && half == 1)) return;
  const int h0 = half * RT;  // first right-hand side of this thread
  const int lt = row / NPHI, k = row - lt * NPHI;
  const float* xs = rn + lt * 4 * BL + h0;  // new residual of the 4 blocks of triangle lt: [block][BL]
  float q[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) q[r] = 0.f;
  // the operator's FP32 / BF16 couplings are in difference form, those of A P plain
  float xr[RT];
  ld_rp<RT>(xs + k * RP, xr);
#pragma unroll
  for (int r = 0; r < RT; ++r) xr[r] = PRE ? 0.f : xr[r];
  const unsigned char* sv = st + (size_t)row * 16;
#pragma unroll
  for (int gg = 0; gg < NG; ++gg) {
    float v[VEC];
    e_lds<T, VEC>(sv + (size_t)gg * TR * 16, v);
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
      const int cc = gg * VEC + u;
      if (cc < NC) {
        float x[RT];
        ld_rp<RT>(xs + (cc / NPHI) * BL + (cc % NPHI) * RP, x);
#pragma unroll
        for (int r = 0; r < RT; ++r) q[r] = fmaf(v[u], x[r] - xr[r], q[r]);
      }
    }
  }
  // (PRE: the couplings of A P include coefK and the mass term)
  const float coefK = PRE ? 1.f : (float)d.coefK;
#pragma unroll
  for (int r = 0; r < RT; ++r) q[r] *= coefK;
  if (!PRE && d.coefM != 0.0) {
    float mv[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) mv[r] = 0.f;
#pragma unroll
    for (int kk = 0; kk < NPHI; ++kk) {
      const float m = (float)__ldg(d.Mref + k * NPHI + kk);
      float x[RT];
      ld_rp<RT>(xs + kk * RP, x);
#pragma unroll
      for (int r = 0; r < RT; ++r) mv[r] = fmaf(m, x[r], mv[r]);
    }
    const float ca = (float)d.coefM * (float)reinterpret_cast<const double*>(st + S::AREA)[lt];
#pragma unroll
    for (int r = 0; r < RT; ++r) q[r] = fmaf(ca, mv[r], q[r]);
  }
  const float* gr = reinterpret_cast<const float*>(st + S::GATHER) + lt * 4 * BL + k * RP + h0;  // own block
  const float* own = reinterpret_cast<const float*>(st + S::OWN) + lt * BL + k * RP + h0;
  float ro[RT], wo[RT], so[RT], dd[RT], pp[RT], rr[RT];
  ld_rp<RT>(gr, ro);
  ld_rp<RT>(gr + NB * BL, wo);
  ld_rp<RT>(gr + 2 * NB * BL, so);
  ld_rp<RT>(own, dd);
  ld_rp<RT>(own + TT * BL, pp);
  ld_rp<RT>(xs + k * RP, rr);
  float u[RT];
  if constexpr (PRE) {
    // p = Pi u + beta p from the own u of the previous pass; u = P_i r_new
    // from the streamed rows of P and the own block of the new residual
    ld_rp<RT>(own + 2 * TT * BL, ro);
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      ro[r] -= c.muu[h0 + r];
      u[r] = 0.f;
    }
    const unsigned char* pv = st + S::PBLK + (size_t)row * 16;
#pragma unroll
    for (int gg = 0; gg < S::NGP; ++gg) {
      const float4 p4 = *reinterpret_cast<const float4*>(pv + (size_t)gg * TR * 16);
      const float pl[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
      for (int l4 = 0; l4 < 4; ++l4) {
        const int l = gg * 4 + l4;
        if (l < NPHI) {
          float x[RT];
          ld_rp<RT>(xs + l * RP, x);
#pragma unroll
          for (int r = 0; r < RT; ++r) u[r] = fmaf(pl[l4], x[r], u[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const float al = c.alpha[h0 + r], be = c.beta[h0 + r];
    pp[r] = fmaf(be, pp[r], ro[r]);
    so[r] = fmaf(be, so[r], wo[r] - c.muw[h0 + r]);
    dd[r] = fmaf(al, pp[r], dd[r]);
    if constexpr (PRE) {
      acc[0][r] = fmaf(rr[r], u[r], acc[0][r]);
      acc[1][r] = fmaf(q[r], u[r], acc[1][r]);
      acc[2][r] += q[r];
      acc[3][r] += u[r];
      acc[4][r] = fmaf(rr[r], rr[r], acc[4][r]);
      acc[5][r] += rr[r];
    } else {
      acc[0][r] = fmaf(rr[r], rr[r], acc[0][r]);
      acc[1][r] = fmaf(q[r], rr[r], acc[1][r]);
      acc[2][r] += q[r];
      acc[3][r] += rr[r];
    }
  }
  const int64_t L = (int64_t)d.ne * BL;
  const int64_t idx = (int64_t)(tri0 + lt) * BL + (int64_t)k * RP + h0;
  const int nx = c.cur ^ 1;
  float* const fv = d.fvec;
  st_rp<RT>(fv + 0 * L + idx, dd);
  st_rp<RT>(fv + 1 * L + idx, pp);
  st_rp<RT>(fv + (2 + nx) * L + idx, rr);
  st_rp<RT>(fv + (4 + nx) * L + idx, q);
  st_rp<RT>(fv + (6 + nx) * L + idx, so);
  if constexpr (PRE) st_rp<RT>(fv + 8 * L + idx, u);
}

// Runtime tile geometry of a slot (producers; the offsets of EStage).
struct EGeom {
  int nphi, tt, tr, ng, ngp, bl, gather, own, area;
};
template <typename T>
__device__ __forceinline__ EGeom e_geom(int p, int rp, int pre) {
  EGeom g;
  g.nphi = e_nphi(p);
  g.tt = e_tt(g.nphi);
  g.tr = g.tt * g.nphi;
  g.ng = (4 * g.nphi + Pack<T>::VEC - 1) / Pack<T>::VEC;
  g.ngp = e_ngp(g.nphi, pre != 0);
  g.bl = e_block_len(g.nphi, rp);
  g.gather = (g.ng + g.ngp) * g.tr * 16;
  g.own = g.gather + 3 * 4 * g.tt * g.bl * 4;
  g.area = g.own + (pre ? 3 : 2) * g.tt * g.bl * 4;
  return g;
}

// ---------------------------------------------------------------- slot transitions

// Completion record of a slot (aggregated over its right-hand sides: first
// non-OK status, largest iteration / refinement count and relative residual).
__device__ __forceinline__ void complete_slot(const EngineParams& E, int sid, const BSlotDesc& d, BState* st) {
  BCompletion* c = &E.done[sid];
  int status = 0, iters = 0, refs = 0;
  double rel = 0.0;
  for (int r = 0; r < d.nrhs; ++r) {
    const volatile BRhs* q = &st->rhs[r];
    if (status == 0) status = q->status;
    iters = max(iters, q->iters);
    refs = max(refs, q->refinements);
    rel = fmax(rel, q->relres);
  }
  c->status = status;
  c->iters = iters;
  c->refinements = refs;
  c->relres = rel;
  c->ticket = d.ticket;
  __threadfence_system();
  *((volatile int*)&c->done) = 1;
  __threadfence_system();
  E.sh->list_dirty = 1;
}

// Advances slot `sid` after a pass from the slot's summed partials t[4 r + j]
// (consumer warp 0: lane r handles right-hand side r, lane 0 the slot).
static __device__ __noinline__ void slot_transition(const EngineParams& E, int sid, const BSlotDesc& d, const double* t) {
  const int lane = threadIdx.x & 31;
  BState* st = &E.state[sid];
  volatile BState* vs = st;
  const double n = (double)d.n;
  const int mz = d.mean_zero;
  const int ph = vs->phase;
  const bool mine = lane < d.nrhs;
  BRhs* q = &st->rhs[lane < kMaxRhs ? lane : 0];
  volatile BRhs* vq = q;
  int next = ph;
  switch (ph) {
    case PH_BSUM: {
      if (mine) {
        const double bm = mz ? t[4 * lane] / n : 0.0;
        const double bn2 = mz ? fmax(0.0, t[4 * lane + 1] - n * bm * bm) : t[4 * lane + 1];
        q->bmean = bm;
        q->bnorm = sqrt(bn2);
        q->best = INFINITY;
        if (!(bn2 > 0.0)) {
          q->relres = 0.0;
          q->status = 0;
          q->done = 1;
        }
      } else if (lane < kMaxRhs) {
        q->done = 1;
      }
      const bool all_done = __all_sync(0xffffffffu, !mine || vq->done);
      next = all_done ? PH_DONE : PH_RESID;
      break;
    }
    case PH_RESID: {
      if (mine && !vq->done) {
        const double rn = sqrt(t[4 * lane]);
        const double rel = rn / vq->bnorm;
        q->rnorm = rn;
        q->rmean = mz ? t[4 * lane + 1] / n : 0.0;
        q->relres = rel;
        int fin = 0, status = 0;
        if (rel <= d.tol) {
          fin = 1;
        } else if (vq->iters >= d.max_iters || vq->refinements >= d.max_refine) {
          fin = 1;
          status = 5;  // DGSL_ENOTCONV
        } else if (rel < 0.9 * vq->best) {
          q->best = rel;
          q->stall = 0;
        } else if (vq->stall + 1 >= 3) {
          fin = 1;
          status = 5;
        } else {
          q->stall = vq->stall + 1;
        }
        if (fin) {
          q->status = status;
          q->done = 1;
          q->inner = 0;
        } else {
          const double stop_rel = fmin(1.0, fmax(d.inner_tol, 0.5 * d.tol / rel));
          q->stop = stop_rel * stop_rel;  // relative to the first inner r.r (set in CG0)
          q->inner = 1;
        }
      }
      const bool all_done = __all_sync(0xffffffffu, !mine || vq->done);
      next = all_done ? (mz ? PH_XSUM : PH_DONE) : PH_SCALE;
      break;
    }
    case PH_SCALE:
      if (lane == 0) st->cur = 0;
      next = PH_CG0;
      break;
    case PH_CG0:
    case PH_CG: {
      if (mine && vq->inner) {
        // sums per right-hand side: (r.r, w.r, sum w, sum r), preconditioned
        // (r.u, w.u, sum w, sum u, r.r, sum r)
        const int ns = d.precond ? 6 : 4;
        const double* tr = t + ns * lane;
        const double mu = mz ? tr[2] / n : 0.0;
        const double mu_u = d.precond && mz ? tr[3] / n : 0.0;
        const float g = (float)(d.precond ? tr[0] - mu_u * tr[5] : tr[0]);
        const float dw = (float)(tr[1] - mu * tr[3]);
        const double rr = d.precond ? tr[4] : tr[0];
        float an, bn;
        int iters = vq->iters;
        if (ph == PH_CG0) {
          q->stop = vq->stop * rr;
          bn = 0.f;
          an = g / dw;
        } else {
          ++iters;
          bn = g / vq->g_old;
          an = g / (dw - bn * g / vq->a_old);
        }
        q->iters = iters;
        if (!(rr > vq->stop) || iters >= d.max_iters || !(an > 0.f) || !isfinite(an)) {
          q->inner = 0;  // frozen: alpha = beta = 0 leaves d and r as they are
          q->alpha = 0.f;
          q->beta = 0.f;
          q->muw = 0.f;
          q->muu = 0.f;
        } else {
          q->alpha = an;
          q->beta = bn;
          q->muw = (float)mu;
          q->muu = (float)mu_u;
          q->g_old = g;
          q->a_old = an;
        }
      }
      const bool any_inner = __any_sync(0xffffffffu, mine && vq->inner);
      if (lane == 0) st->cur = vs->cur ^ 1;  // the pass wrote r, w, s into the other buffers
      next = any_inner ? PH_CG : PH_UPDATE;
      break;
    }
    case PH_UPDATE:
      if (mine && !vq->done) q->refinements = vq->refinements + 1;
      next = PH_RESID;
      break;
    case PH_XSUM:
      if (mine) q->xmean = t[4 * lane] / n;
      next = PH_XFIX;
      break;
    case PH_XFIX:
      next = PH_DONE;
      break;
    default:
      break;
  }
  __syncwarp();
  __threadfence();
  if (lane == 0) {
    st->phase = next;
    if (next == PH_DONE) complete_slot(E, sid, d, st);
    __threadfence();
  }
  __syncwarp();
}

// ---------------------------------------------------------------- barrier hook

__device__ __forceinline__ void copy_desc(BSlotDesc* dst, const BSlotDesc* src) {
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* o = reinterpret_cast<unsigned long long*>(dst);
  constexpr int W = (int)(sizeof(BSlotDesc) / 8);
  for (int i = threadIdx.x; i < W; i += blockDim.x) o[i] = *((volatile const unsigned long long*)(s + i));
}

// Admission of newly published slots, rebuild of the active-chunk list with
// each CTA's starting list index, and the stage ring of the next pass (whole
// CTA of the last arriver; the indexed work uses the consumer threads).
template <typename T, bool PC>
__device__ __noinline__ void engine_hook(const EngineParams& E) {
  constexpr int H = kEConsumers;
  __shared__ int s_count, s_adm, s_dirty, s_per, s_mx, s_run[H], s_runc[H];
  EngineShared* sh = E.sh;
  const bool w = threadIdx.x < H;
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
    constexpr int PER = kMaxSlots / H;
    if (w) {
      int cnt = 0, chunks = 0;
      for (int j = 0; j < PER; ++j) {
        const int sidx = threadIdx.x * PER + j;
        if (sidx < s_count && __ldcg(&E.state[sidx].phase) != PH_DONE) {
          ++cnt;
          chunks += __ldcg(&E.slots[sidx].nchunk);
        }
      }
      s_run[threadIdx.x] = cnt;
      s_runc[threadIdx.x] = chunks;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive scans
      int a = 0, b = 0;
      for (int i = 0; i < H; ++i) {
        const int ta = s_run[i], tb = s_runc[i];
        s_run[i] = a;
        s_runc[i] = b;
        a += ta;
        b += tb;
      }
      sh->n_act = a;
      sh->total_chunks = b;
      E.act_chunk0[a] = b;
      s_per = (b + (int)gridDim.x - 1) / (int)gridDim.x;  // chunks per CTA (the pass splits as the kernel does)
    }
    __syncthreads();
    if (w) {
      int k = s_run[threadIdx.x], c0 = s_runc[threadIdx.x];
      const int per = s_per;
      for (int j = 0; j < PER; ++j) {
        const int sidx = threadIdx.x * PER + j;
        if (sidx < s_count && __ldcg(&E.state[sidx].phase) != PH_DONE) {
          const int nc = __ldcg(&E.slots[sidx].nchunk);
          E.act_slot[k] = sidx;
          E.act_chunk0[k] = c0;
          // the CTAs whose range starts inside this slot's chunks start their walk at k
          if (per > 0)
            for (int cta = (c0 + per - 1) / per; cta < (int)gridDim.x && cta * per < c0 + nc; ++cta) E.cta_k[cta] = k;
          ++k;
          c0 += nc;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      sh->admitted = s_count;
      sh->list_dirty = 0;
    }
  }
  __syncthreads();
  // stage ring of the next pass: the largest tile footprint among the active CG slots
  if (threadIdx.x == 0) s_mx = 128;
  __syncthreads();
  {
    const int na = *((volatile int*)&sh->n_act);
    int mx = 128;
    for (int k = threadIdx.x; k < na; k += blockDim.x) {
      const int sid = __ldcg(E.act_slot + k);
      const int ph = __ldcg(&E.state[sid].phase);
      if (ph == PH_CG0 || ph == PH_CG) {
        const EGeom g = e_geom<T>(__ldcg(&E.slots[sid].p), __ldcg(&E.slots[sid].rp), PC ? __ldcg(&E.slots[sid].precond) : 0);
        mx = max(mx, g.area + (g.tt * 8 + 15) / 16 * 16);
      }
    }
    atomicMax(&s_mx, mx);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int SB = (s_mx + 127) / 128 * 128;
    sh->ring_SB = SB;
    sh->ring_S = min(kEMaxStages, kEDynSmem / SB);
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

// ---------------------------------------------------------------- pass roles

// Walk of a CTA's chunk range over the active list: slot of chunk `cidx`.
struct EWalk {
  int k, sid, chunk0, next0;
};
__device__ __forceinline__ void walk_to(const EngineParams& E, int n_act, int cidx, EWalk& w) {
  if (w.sid >= 0 && cidx < w.next0) return;
  while (w.k + 1 < n_act && __ldcg(E.act_chunk0 + w.k + 1) <= cidx) ++w.k;
  w.sid = __ldcg(E.act_slot + w.k);
  w.chunk0 = __ldcg(E.act_chunk0 + w.k);
  w.next0 = __ldcg(E.act_chunk0 + w.k + 1);
}
// A CTA's walk starts at the list index the barrier hook recorded for it.
__device__ __forceinline__ EWalk walk_from(int k0) {
  EWalk w;
  w.k = k0;
  w.sid = -1;
  w.chunk0 = w.next0 = 0;
  return w;
}
__device__ __forceinline__ bool is_cg(int phase) { return phase == PH_CG0 || phase == PH_CG; }

// Bounded wait for a stage's release that also gives up when the CTA has
// recorded an error (s_err).
__device__ __forceinline__ bool e_wait_empty(uint64_t* bar, unsigned parity, uint64_t timeout_ns,
                                             volatile int* s_err) {
  const uint64_t t0 = globaltimer_ns();
  for (unsigned spins = 1;; ++spins) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*s_err) return false;
    if ((spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) return false;
  }
}

// Stage ring of one pass: S stages of SB bytes (SB = the largest tile
// footprint among the active CG slots, set by the barrier hook).
struct ERing {
  unsigned char* base;
  int S, SB;
};

// Coupling warp (lane 0): TMA bulk copies of every CG tile of the range.
template <typename T, bool PC>
__device__ void coupling_pass(const EngineParams& E, int n_act, int cb, int ce, int k0, const ERing& ring,
                              uint64_t* full, uint64_t* empty, unsigned& gt, volatile int* s_err) {
  const uint64_t pol = l2_evict_first_policy();
  EWalk w = walk_from(k0);
  for (int cidx = cb; cidx < ce; ++cidx) {
    walk_to(E, n_act, cidx, w);
    const BSlotDesc* dp = &E.slots[w.sid];
    if (!is_cg(__ldcg(&E.state[w.sid].phase))) continue;
    const int p = __ldcg(&dp->p), ne = __ldcg(&dp->ne), ct = __ldcg(&dp->chunk_tris);
    const int64_t n = __ldcg(&dp->n);
    const T* vals = static_cast<const T*>(*((const void* const volatile*)&dp->Kin));
    const int pre = PC ? __ldcg(&dp->precond) : 0;
    const float* pin = pre ? *((const float* const volatile*)&dp->Pin) : nullptr;
    const EGeom g = e_geom<T>(p, 1, pre);
    const int t0 = (cidx - w.chunk0) * ct, t1 = min(ne, t0 + ct);
    for (int tri0 = t0; tri0 < t1; tri0 += g.tt, ++gt) {
      const int s = (int)(gt % ring.S);
      if (gt >= (unsigned)ring.S && !e_wait_empty(&empty[s], ((gt / ring.S) - 1u) & 1u, E.timeout_ns, s_err)) {
        *s_err = 1;
        atomicCAS(&E.sh->status, kStatusOk, kStatusTimeout);
        return;
      }
      const int nt = min(g.tt, t1 - tri0);
      const uint32_t bytes = (uint32_t)(nt * g.nphi * 16);
      unsigned char* dst = ring.base + (size_t)s * ring.SB;
      fence_proxy_async_smem();
      mbar_expect_tx(&full[s], bytes * (g.ng + g.ngp));
      for (int c = 0; c < g.ng; ++c)
        bulk_g2s_hint(dst + (size_t)c * g.tr * 16, vals + ((size_t)c * n + (size_t)tri0 * g.nphi) * Pack<T>::VEC, bytes,
                      &full[s], pol);
      for (int c = 0; c < g.ngp; ++c)  // rows of P (preconditioned slots)
        bulk_g2s_hint(dst + (size_t)(g.ng + c) * g.tr * 16, pin + ((size_t)c * n + (size_t)tri0 * g.nphi) * 4, bytes,
                      &full[s], pol);
    }
  }
}

// Gather warp (32 lanes): 16-byte cp.async of the previous r, w, s of the
// 4 TT coupled blocks of every CG tile, of the own d and p blocks and of the
// areas (Helmholtz), completing on gfull (one arrival per lane).  (Bulk TMA
// copies of each small block were several times slower: the blocks are
// 48-480 bytes each.)
template <typename T, bool PC>
__device__ void gather_pass(const EngineParams& E, int n_act, int cb, int ce, int k0, const ERing& ring,
                            uint64_t* gfull, uint64_t* empty, unsigned& gt, volatile int* s_err) {
  __shared__ int s_gcol[4 * kERows];  // column indices of the current tile (4 TT <= 4 kERows / 3)
  const int lane = threadIdx.x & 31;
  EWalk w = walk_from(k0);
  for (int cidx = cb; cidx < ce; ++cidx) {
    walk_to(E, n_act, cidx, w);
    const BSlotDesc* dp = &E.slots[w.sid];
    const int phase = __ldcg(&E.state[w.sid].phase);
    if (!is_cg(phase)) continue;
    const int cur = __ldcg(&E.state[w.sid].cur);
    const int p = __ldcg(&dp->p), ne = __ldcg(&dp->ne), ne_pad = __ldcg(&dp->ne_pad), ct = __ldcg(&dp->chunk_tris);
    const int rp = __ldcg(&dp->rp);
    const int32_t* cols = *((const int32_t* const volatile*)&dp->cols);
    const double* area = *((const double* const volatile*)&dp->area);
    float* fvec = *((float* const volatile*)&dp->fvec);
    const int pre = PC ? __ldcg(&dp->precond) : 0;
    const bool mass = !pre && __ldcg(&dp->coefM) != 0.0;  // (A P holds the mass term)
    const EGeom g = e_geom<T>(p, rp, pre);
    const int64_t L = (int64_t)ne * g.bl;
    const float* ro = fvec + (2 + cur) * L;
    const float* wo = fvec + (4 + cur) * L;
    const float* so = fvec + (6 + cur) * L;
    const int cpb = g.bl / 4;                                  // 16-byte chunks per block (<= 30)
    const size_t vstride = (size_t)4 * g.tt * g.bl * 4;        // bytes between the gathered r, w, s
    const int t0 = (cidx - w.chunk0) * ct, t1 = min(ne, t0 + ct);
    for (int tri0 = t0; tri0 < t1; tri0 += g.tt, ++gt) {
      const int s = (int)(gt % ring.S);
      if (gt >= (unsigned)ring.S) {
        const bool got = e_wait_empty(&empty[s], ((gt / ring.S) - 1u) & 1u, E.timeout_ns, s_err);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) {
            *s_err = 1;
            atomicCAS(&E.sh->status, kStatusOk, kStatusTimeout);
          }
          e_cp_wait_all();
          return;
        }
      }
      const int nt = min(g.tt, t1 - tri0);
      unsigned char* st = ring.base + (size_t)s * ring.SB;
      // the tile's column indices, then the (block, chunk) pairs spread evenly
      // over the lanes, walked without division
      __syncwarp();
      for (int b = lane; b < 4 * nt; b += 32) s_gcol[b] = __ldg(cols + (size_t)(b & 3) * ne_pad + tri0 + (b >> 2));
      __syncwarp();
      const int nbc = 4 * nt * cpb;
      int b = lane / cpb, c = lane - b * cpb;
      const int sb = 32 / cpb, sc = 32 - sb * cpb;
      for (int e = lane; e < nbc; e += 32) {
        unsigned char* db = st + g.gather + ((size_t)b * g.bl + 4 * c) * 4;
        const int64_t o = (int64_t)s_gcol[b] * g.bl + 4 * c;
        e_cp16(db, ro + o);
        e_cp16(db + vstride, wo + o);
        e_cp16(db + 2 * vstride, so + o);
        b += sb;
        c += sc;
        if (c >= cpb) {
          c -= cpb;
          ++b;
        }
      }
      const int per = nt * cpb;  // chunks of one own vector: d, p (and u, vector 8)
      for (int q = lane; q < (pre ? 3 : 2) * per; q += 32) {
        const int v = q >= 2 * per ? 2 : q >= per ? 1 : 0, cx = q - v * per;
        e_cp16(st + g.own + ((size_t)v * g.tt * g.bl + 4 * cx) * 4,
               fvec + (v == 2 ? 8 : v) * L + (int64_t)tri0 * g.bl + 4 * cx);
      }
      if (mass)
        for (int q = lane; q < (nt + 1) / 2; q += 32) e_cp16(st + g.area + q * 16, area + tri0 + 2 * q);
      e_cp_arrive(&gfull[s]);
    }
  }
}

// Consumers: the CG tiles of one chunk (RP right-hand sides), partial sums of
// the chunk into sums[NA r + j] (NA = 4, or 6 preconditioned).
template <int NPHI, typename T, int RP, bool PRE, int NR>
__device__ __forceinline__ bool cg_chunk(const BSlotDesc& d, const ChunkCtx& c, int t0, int t1, const ERing& ring,
                                         uint64_t* full, uint64_t* gfull, uint64_t* empty, unsigned& gt,
                                         uint64_t timeout_ns, double* sums, double (*s_red)[NR], float* s_rn) {
  constexpr int TT = ETile<NPHI, T>::TT;
  constexpr int RT = RhsSplit<RP>::RT;
  constexpr int NA = PRE ? 6 : 4;
  float acc[NA][RT];
#pragma unroll
  for (int j = 0; j < NA; ++j)
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[j][r] = 0.f;
  for (int tri0 = t0; tri0 < t1; tri0 += TT, ++gt) {
    const int s = (int)(gt % ring.S);
    const unsigned par = (gt / ring.S) & 1u;
    const int nt = min(TT, t1 - tri0);
    const unsigned char* st = ring.base + (size_t)s * ring.SB;
    bool got = mbar_wait_bounded(&full[s], par, timeout_ns);
    got = got && mbar_wait_bounded(&gfull[s], par, timeout_ns);
    float* rn = s_rn + (gt & 1u) * kRnMax;
    cg_combine<NPHI, T, RP, PRE>(c, nt, st, rn);
    if (!ecbar_and(got)) return false;  // also: the combined tile is complete
    cg_rows<NPHI, T, RP, PRE>(d, c, tri0, nt, st, rn, acc);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) e_mbar_arrive(&empty[s]);  // this warp is done with the stage
  }
  // each right-hand side's sums come from one half of the consumer threads; the
  // other half adds exact zeros, so the reduction matches a one-RHS slot's
  const int half = threadIdx.x / kERows;
  float v[NA * RP];
#pragma unroll
  for (int r = 0; r < RP; ++r)
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      float a = 0.f;
      if (r < RT) {
        if (half == 0) a = acc[j][r];
      } else {
        if (half == 1) a = acc[j][r - RT];
      }
      v[NA * r + j] = a;
    }
  if ((int)threadIdx.x < NR) sums[threadIdx.x] = 0.0;
  ecbar();
  e_reduce<NA * RP, NR, float>(v, sums, s_red);
  return true;
}

// PC: the launch may carry preconditioned slots (the kernel then holds both
// CG forms; a launch without them keeps the plain form's code alone).
template <typename T, int NPHI, bool PC, int NR>
__device__ __forceinline__ bool chunk_work(const BSlotDesc& d, const ChunkCtx& c, int t0, int t1, const ERing& ring,
                                           uint64_t* full, uint64_t* gfull, uint64_t* empty, unsigned& gt,
                                           uint64_t timeout_ns, double* sums, double (*s_red)[NR], float* s_rn) {
  if (is_cg(c.phase)) {
#define DGSL_E_CG(RP, PRE) cg_chunk<NPHI, T, RP, PRE, NR>(d, c, t0, t1, ring, full, gfull, empty, gt, timeout_ns, sums, s_red, s_rn)
    if (PC && d.precond) {
      switch (c.rp) {
        case 1: return DGSL_E_CG(1, true);
        case 2: return DGSL_E_CG(2, true);
        case 4: return DGSL_E_CG(4, true);
        default: return DGSL_E_CG(8, true);
      }
    }
    switch (c.rp) {
      case 1: return DGSL_E_CG(1, false);
      case 2: return DGSL_E_CG(2, false);
      case 4: return DGSL_E_CG(4, false);
      default: return DGSL_E_CG(8, false);
    }
#undef DGSL_E_CG
  }
  stream_chunk<NPHI, NR>(d, c, t0, t1, sums, s_red);
  return true;
}

// Consumer warps: every chunk of the range.  Each chunk's partial sums are
// published; one arrival per (slot, pass) covers this CTA's chunks of the
// slot, and the CTA whose arrival completes the slot's pass sums the slot's
// partials in chunk order and advances the slot.
template <typename T, bool PC>
__device__ bool consumer_pass(const EngineParams& E, int n_act, int cb, int ce, int k0, const ERing& ring, uint64_t* full,
                              uint64_t* gfull, uint64_t* empty, unsigned& gt) {
  __shared__ BSlotDesc s_desc;
  __shared__ ChunkCtx s_ctx;
  constexpr int NR = e_part_stride(PC);  // partial sums per chunk in this launch
  __shared__ double s_red[kECWarps][NR];
  __shared__ double s_sum[NR], s_tot[NR];
  __shared__ int s_last;
  __shared__ __align__(16) float s_rn[2 * kRnMax];  // new residual of a tile, double-buffered
  const BSlotDesc& d = s_desc;
  const ChunkCtx& c = s_ctx;
  EWalk w = walk_from(k0);
  int cur_sid = -1, pend = 0;
  auto flush = [&]() {
    if (pend == 0) return;
    ecbar();  // every partial of these chunks is written
    if (threadIdx.x == 0) {
      unsigned long long v;
      asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], %2;"
                   : "=l"(v)
                   : "l"(&E.state[cur_sid].arrivals), "l"((unsigned long long)pend)
                   : "memory");
      s_last = ((v + (unsigned long long)pend) % (unsigned long long)d.nchunk) == 0ull;
    }
    ecbar();
    pend = 0;
    if (s_last) {
      const int grp = threadIdx.x >> 5;
      const int nv = e_part_stride(PC && d.precond);
      for (int v = threadIdx.x & 31; v < nv; v += 32) {
        double a = 0.0;
        for (int ch = grp; ch < d.nchunk; ch += kECWarps) a += __ldcg(d.part + (size_t)ch * nv + v);
        s_red[grp][v] = a;
      }
      ecbar();
      if (threadIdx.x < 32)
        for (int v = threadIdx.x; v < nv; v += 32) {
          double t = s_red[0][v];
          for (int q = 1; q < kECWarps; ++q) t += s_red[q][v];
          s_tot[v] = t;
        }
      ecbar();
      if (threadIdx.x < 32) slot_transition(E, cur_sid, d, s_tot);
      ecbar();
    }
  };
  for (int cidx = cb; cidx < ce; ++cidx) {
    walk_to(E, n_act, cidx, w);
    if (w.sid != cur_sid) {
      flush();
      ecbar();
      if (threadIdx.x < 32) load_slot(s_desc, s_ctx, &E.slots[w.sid], &E.state[w.sid]);
      ecbar();
      cur_sid = w.sid;
    }
    const int lc = cidx - w.chunk0;
    const int t0 = lc * d.chunk_tris;
    const int t1 = min(d.ne, t0 + d.chunk_tris);
    bool ok;
    switch (d.p) {
      case 1: ok = chunk_work<T, 3, PC, NR>(d, c, t0, t1, ring, full, gfull, empty, gt, E.timeout_ns, s_sum, s_red, s_rn); break;
      case 2: ok = chunk_work<T, 6, PC, NR>(d, c, t0, t1, ring, full, gfull, empty, gt, E.timeout_ns, s_sum, s_red, s_rn); break;
      case 3: ok = chunk_work<T, 10, PC, NR>(d, c, t0, t1, ring, full, gfull, empty, gt, E.timeout_ns, s_sum, s_red, s_rn); break;
      default: ok = chunk_work<T, 15, PC, NR>(d, c, t0, t1, ring, full, gfull, empty, gt, E.timeout_ns, s_sum, s_red, s_rn); break;
    }
    if (!ok) return false;
    {
      const int nv = e_part_stride(PC && d.precond);
      if ((int)threadIdx.x < nv) d.part[(size_t)lc * nv + threadIdx.x] = s_sum[threadIdx.x];
    }
    ++pend;
  }
  flush();
  return true;
}

// ---------------------------------------------------------------- kernel

template <typename T, bool PC>
__global__ void __launch_bounds__(kEThreads, 1) k_engine(EngineParams E) {
  extern __shared__ __align__(128) unsigned char stages[];
  __shared__ __align__(8) uint64_t full[kEMaxStages], gfull[kEMaxStages], empty[kEMaxStages];
  __shared__ volatile int s_err;
  const unsigned nb = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long epoch = 0;
  unsigned gt = 0;  // this role's CG tiles in the current pass (stage gt % S, parity (gt / S) & 1)
  ERing ring{stages, 2, 128};
  if (threadIdx.x == 0) {
    for (int i = 0; i < kEMaxStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&gfull[i], 32);
      mbar_init(&empty[i], kECWarps);
    }
    s_err = 0;
    fence_proxy_async_smem();
  }
  __syncthreads();
  auto hook = [&E]() { engine_hook<T, PC>(E); };
  bool ok = grid_sync_hook(E.sh, nb, epoch, E.timeout_ns, hook);
  while (ok) {
    if (__ldcg(&E.sh->exit_now)) break;
    const int n_act = __ldcg(&E.sh->n_act);
    const int total = __ldcg(&E.sh->total_chunks);
    // contiguous chunk range per CTA
    const int per = (total + (int)nb - 1) / (int)nb;
    const int cb = min(total, (int)blockIdx.x * per);
    const int ce = min(total, cb + per);
    // this pass's stage ring (set by the hook); every copy of the previous pass
    // has been consumed, so the barriers start afresh
    const int k0 = cb < ce ? __ldcg(E.cta_k + blockIdx.x) : 0;
    ring.S = __ldcg(&E.sh->ring_S);
    ring.SB = __ldcg(&E.sh->ring_SB);
    if (threadIdx.x == 0) {
      for (int i = 0; i < kEMaxStages; ++i) {
        mbar_inval(&full[i]);
        mbar_inval(&gfull[i]);
        mbar_inval(&empty[i]);
        mbar_init(&full[i], 1);
        mbar_init(&gfull[i], 32);
        mbar_init(&empty[i], kECWarps);
      }
      fence_proxy_async_smem();
    }
    __syncthreads();
    gt = 0;
    if (warp < kECouplingWarp) {
      if (!consumer_pass<T, PC>(E, n_act, cb, ce, k0, ring, full, gfull, empty, gt)) {
        if (threadIdx.x == 0) {
          s_err = 1;
          atomicCAS(&E.sh->status, kStatusOk, kStatusTimeout);
        }
      }
    } else if (warp == kECouplingWarp) {
      if (lane == 0) coupling_pass<T, PC>(E, n_act, cb, ce, k0, ring, full, empty, gt, &s_err);
    } else {
      gather_pass<T, PC>(E, n_act, cb, ce, k0, ring, gfull, empty, gt, &s_err);
    }
    ok = grid_sync_hook(E.sh, nb, epoch, E.timeout_ns, hook);
  }
  // no CTA leaves with a copy still writing its shared memory
  if (warp == kECouplingWarp && lane == 0)
    for (unsigned h = gt > (unsigned)ring.S ? gt - ring.S : 0u; h < gt; ++h)
      if (!mbar_wait_bounded(&full[h % ring.S], (h / ring.S) & 1u, E.timeout_ns))
        atomicCAS(&E.sh->status, kStatusOk, kStatusTimeout);
  if (warp == kEGatherWarp) e_cp_wait_all();
  __syncthreads();
}

template <typename T, bool PC>
inline cudaError_t launch_engine_t(const EngineParams& e, cudaStream_t s, int* grid_used) {
  auto kern = k_engine<T, PC>;
  const size_t dyn = kEDynSmem;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kEThreads, dyn);
  if (err != cudaSuccess) return err;
  if (per < 1) return cudaErrorLaunchOutOfResources;
  per = std::min(per, 8);
  const int blocks = std::min(sms * per, kMaxCtas);
  if (grid_used) *grid_used = blocks;
  EngineParams a = e;
  void* args[] = {&a};
  err = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kEThreads), args, dyn, s);
  count_launch();
  return err;
}

// Launch of the kernels that also run preconditioned slots (k_batch_pc.cu).
cudaError_t launch_engine_precond(const EngineParams& e, int bf16, cudaStream_t s, int* grid_used);

}  // namespace dgsl
