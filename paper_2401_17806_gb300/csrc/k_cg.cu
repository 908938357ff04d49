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
// The pass is tiled by triangles and warp-specialised.  Each CTA has three
// roles working through the same ring of shared-memory stages:
//  - a coupling warp streams each tile's coupling coefficients with TMA bulk
//    copies (L2 evict-first), running ahead across pass boundaries (the
//    couplings are constant);
//  - a gather warp copies, with 16-byte cp.async, the previous r, w and s of
//    each tile triangle and its three neighbours and the own p and x, after the
//    grid all-reduce that opens the pass (they are written by other CTAs);
//  - four consumer warps form the new residual of the gathered blocks,
//    r - alpha (w' + beta s), once per tile, then each thread owns one matrix
//    row: it streams the row's 4 N_phi couplings against those values and
//    updates p, s, x, r and w.
// So that every gathered block starts on a 16-byte boundary, the CG's own
// vectors are stored per triangle with N_phi padded to a multiple of the
// 16-byte vector width (the caller's r and x stay unpadded).  Partial sums
// are reduced per CTA and, once every CTA has arrived, summed by every CTA in
// the same fixed order, so all CTAs take identical, deterministic decisions.
//
// Block-Jacobi preconditioned variant (PRE; an extension, the paper runs CG
// unpreconditioned): u = P r with P = blockdiag(D_i)^-1, D_i the N_phi x N_phi
// diagonal block of A on triangle i.  The preconditioned Chronopoulos-Gear
// iteration needs w = A u; since A u = (A P) r and A P has the sparsity of A
// (block (i, j) = A_ij P_j), the couplings streamed are those of A P, so the
// pass still gathers r, w, s and recomputes the coupled residual blocks as
// above, and u = P_i r is formed for the own block only, from the residual
// block already in shared memory and the streamed rows of P.  u is thus
// explicit (a recurrence for u loses the attainable accuracy of the FP32
// inner solve).  One reduction per pass carries (r.u, w.u, sum w, sum u, r.r,
// sum r); gamma = r.u replaces r.r in the scalar recurrences.  For the
// periodic pressure operator the preconditioner is Pi P Pi (Pi: projection
// to mean zero; symmetric and positive definite on the mean-free vectors), u
// being projected by its mean from that reduction where it is used, so p and
// x stay mean-free.
#include <cstdlib>

#include "kassembled.cuh"
#include "kernels.h"

namespace dgsl {

constexpr int kCgConsumers = 128;                // 4 warps, one matrix row per thread
constexpr int kCouplingWarp = kCgConsumers / 32;
constexpr int kGatherWarp = kCouplingWarp + 1;   // the first of NGW gather warps
// CTA size with NGW gather warps: the consumers, the coupling warp, the gather warps
template <int NGW>
struct CgThreads {
  static constexpr int value = kCgConsumers + 32 + 32 * NGW;
};

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
  V* x;          // result, unpadded (written at exit)
  const V* r0;   // right-hand side, unpadded
  const V* pinv; // PRE: inverse diagonal blocks, element (row, l) at ((l / VP) n + row) VP + l % VP
  V* vec;        // padded vectors of ne * NPAD: p | x | r0 | r1 | w0 | w1 | s0 | s1, with PRE
                 // p | x | u | r0 | r1 | w0 | w1 | s0 | s1
  double* part;  // [2][max_parts][4 or 6 (PRE)] (epoch parity)
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

// ---- synchronisation among the consumer warps only (named barrier 1), so
// the two producer warps are never held by a consumer barrier.
__device__ __forceinline__ void cbar() { asm volatile("bar.sync 1, %0;" ::"n"(kCgConsumers) : "memory"); }
__device__ __forceinline__ bool cbar_and(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(r)
      : "r"((unsigned)v), "n"(kCgConsumers)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_addr(bar)) : "memory");
}
// 16-byte global -> shared copy through L2 only (no L1: the CG vectors are
// rewritten by other CTAs during the launch).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// Arrive on `bar` once this thread's earlier cp.async copies have landed (the
// barrier's expected count includes this arrival).
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Deterministic sum of v[NW] over the consumer threads, in type W; the result
// is valid in consumer thread 0 (fixed shuffle tree, then the 4 warp sums in order).
template <int NW, typename W>
__device__ __forceinline__ void consumer_sum(W (&v)[NW], W (*s_red)[NW]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NW; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NW; ++i) s_red[wid][i] = v[i];
  cbar();
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NW; ++i) v[i] = ((s_red[0][i] + s_red[1][i]) + s_red[2][i]) + s_red[3][i];
  cbar();
}

// Grid-wide sum of acc[0..NW-1] by the consumer warps.  Each CTA publishes its
// partial (summed over its threads in V, widened to FP64) and arrives on the
// counter; once every CTA has arrived, every CTA sums all partials itself in
// CTA order (FP64), so all obtain bit-identical totals one round trip after
// the last arrival.  The partials alternate between two halves of part[] by
// epoch parity: a CTA that has moved on to the next epoch writes the other
// half, never a partial that a slower CTA is still reading.  The acq_rel
// arrival also orders this CTA's vector writes (made before the consumer
// barrier) for every CTA that later sees the count.
template <int NW, typename V>
__device__ __forceinline__ bool consumer_allreduce(GridBarrier* b, double* part, unsigned nblocks,
                                                   unsigned long long& epoch, uint64_t timeout_ns,
                                                   V (&acc)[NW], double (&tot)[NW]) {
  __shared__ V s_redv[4][NW];
  __shared__ double s_red[4][NW];
  __shared__ double s_tot[NW];
  __shared__ int s_state;
  consumer_sum<NW, V>(acc, s_redv);
  ++epoch;
  double* pe = part + (size_t)(epoch & 1ull) * NW * nblocks;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NW; ++i) pe[NW * blockIdx.x + i] = (double)acc[i];
    const unsigned long long target = epoch * (unsigned long long)nblocks;
    unsigned long long v;
    asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(v) : "l"(&b->count) : "memory");
    int st = 0;
    if (v + 1 < target) {
      const uint64_t t0 = globaltimer_ns();
      for (unsigned spins = 1;; ++spins) {
        asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(&b->count) : "memory");
        if (v >= target) break;
        if (*((volatile int*)&b->status) != kStatusOk) { st = -1; break; }
        if ((spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
          atomicCAS(&b->status, kStatusOk, kStatusTimeout);
          st = -1;
          break;
        }
      }
    }
    if (*((volatile int*)&b->status) != kStatusOk) st = -1;
    s_state = st;  // one thread decides, so that every consumer thread takes the same branch
  }
  cbar();
  const bool ok = s_state >= 0;
  double t[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) t[i] = 0.0;
  if (ok)
    for (unsigned j = threadIdx.x; j < nblocks; j += kCgConsumers)
#pragma unroll
      for (int i = 0; i < NW; ++i) t[i] += __ldcg(pe + (size_t)j * NW + i);
  consumer_sum<NW, double>(t, s_red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NW; ++i) s_tot[i] = t[i];
  cbar();
#pragma unroll
  for (int i = 0; i < NW; ++i) tot[i] = s_tot[i];
  cbar();
  return ok;
}

// Tile geometry: TT triangles (a multiple of 4; TR = TT N_phi matrix rows, one
// per consumer thread) per tile.  A stage holds the tile's couplings (NG
// chunks of TR 16-byte vectors, each contiguous in global memory), with PRE
// the rows of P (NGP more chunks), the gathered r, w, s of the 4 TT coupled
// blocks, the own p, x (PRE: p, x, u) blocks, and the own triangles' areas
// (Helmholtz mass term).
template <int NPHI, typename T, typename V, bool PRE = false>
struct TileCfg {
  static constexpr int VEC = Pack<T>::VEC;
  static constexpr int NC = 4 * NPHI;
  static constexpr int NG = (NC + VEC - 1) / VEC;
  static constexpr int TT = (kCgConsumers / NPHI) / 4 * 4;
  static constexpr int TR = TT * NPHI;
  static constexpr int VPC = 16 / (int)sizeof(V);          // vector values per 16 bytes
  static constexpr int NPAD = (NPHI + VPC - 1) / VPC * VPC;  // padded block length
  static constexpr int CPB = NPAD / VPC;                     // 16-byte chunks per block
  static constexpr int NB = 4 * TT;                          // coupled blocks per tile
  static constexpr int COUPLE = NG * TR * 16;
  static constexpr int VP = 16 / (int)sizeof(V);                      // P values per 16 bytes
  static constexpr int NGP = PRE ? (NPHI + VP - 1) / VP : 0;         // P chunks per row
  static constexpr int PBLK = COUPLE;                                 // byte offset of the P rows
  static constexpr int GATHER = COUPLE + NGP * TR * 16;               // r | w | s blocks
  static constexpr int NOWN = PRE ? 3 : 2;                            // own p | x (PRE: | u)
  static constexpr int OWN = GATHER + 3 * NB * NPAD * (int)sizeof(V);
  static constexpr int AREA = OWN + NOWN * TT * NPAD * (int)sizeof(V);  // TT doubles
  static constexpr int STAGE = (AREA + TT * 8 + 127) / 128 * 128;
  // stages per CTA; PRE keeps two CTAs per SM where three stages allow it
  static constexpr int S = PRE ? (3 * STAGE <= 104 * 1024 ? 3 : 2) : (3 * STAGE <= 180 * 1024 ? 3 : 2);
};

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

__device__ __forceinline__ void cp_async8_ca(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

template <int NPHI, typename T, typename V, bool PRE, int NGW>
__device__ __forceinline__ void cg_body(const CGParams<T, V>& a) {
  using C = TileCfg<NPHI, T, V, PRE>;
  constexpr int S = C::S, TT = C::TT, TR = C::TR, NPAD = C::NPAD, NB = C::NB, CPB = C::CPB, VPC = C::VPC;
  constexpr int VEC = C::VEC, NC = C::NC, NG = C::NG, VP = C::VP, NGP = C::NGP, NOWN = C::NOWN;
  extern __shared__ __align__(128) unsigned char stages[];
  __shared__ __align__(8) uint64_t full[S], gfull[S], empty[S];
  __shared__ V s_rn[2][NB * NPHI];
  __shared__ double s_Mref[NPHI * NPHI];
  __shared__ volatile int s_stop;
  const unsigned nb = gridDim.x;
  const int ne = a.ne;
  const int ntiles = (ne + TT - 1) / TT;
  const int nq = ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)nb + 1 : 0;
  const int64_t npv = (int64_t)ne * NPAD;
  V* const pp = a.vec;
  V* const xp = a.vec + npv;
  V* const up = a.vec + 2 * npv;  // PRE: u (own rows only)
  constexpr int G0 = PRE ? 3 : 2;  // first gathered (double-buffered) vector
  auto rbuf = [&](int k) { return a.vec + (G0 + (k & 1)) * npv; };
  auto wbuf = [&](int k) { return a.vec + (G0 + 2 + (k & 1)) * npv; };
  auto sbuf = [&](int k) { return a.vec + (G0 + 4 + (k & 1)) * npv; };
  unsigned long long epoch = 0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&gfull[i], 32 * NGW);
      mbar_init(&empty[i], kCgConsumers / 32);
    }
    s_stop = 0;
    fence_proxy_async_smem();
  }
  for (int i = threadIdx.x; i < NPHI * NPHI; i += blockDim.x) s_Mref[i] = a.Mref[i];

  // prologue (all warps): padded copy of r0 and its sum; x = p = w = s = 0
  bool pro_ok;
  {
    V* const r0p = rbuf(0);
    V* const w0p = wbuf(0);
    V* const s0p = sbuf(0);
    const int64_t stride = (int64_t)nb * blockDim.x;
    V sum = V(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npv; i += stride) {
      const int64_t tri = i / NPAD;
      const int k = (int)(i - tri * NPAD);
      const V r = k < NPHI ? a.r0[tri * NPHI + k] : V(0);
      sum += r;
      r0p[i] = r;
      pp[i] = V(0);
      xp[i] = V(0);
      w0p[i] = V(0);
      s0p[i] = V(0);
      if constexpr (PRE) up[i] = V(0);
    }
    double acc[4] = {to_d(sum), 0.0, 0.0, 0.0}, tot[4];
    pro_ok = __syncthreads_and(grid_allreduce4(a.bar, a.part, nb, epoch, a.timeout_ns, acc, tot)) != 0;
    if (pro_ok && a.mean_zero) {
      const V mu = (V)(tot[0] / (double)a.n);
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npv; i += stride)
        if (i % NPAD < NPHI) r0p[i] -= mu;
    }
    if (pro_ok) pro_ok = grid_sync_epoch(a.bar, nb, epoch, a.timeout_ns);
  }
  // (no CTA-wide barrier below this point: the roles synchronise through mbarriers)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == kCouplingWarp) {
    // ---- coupling producer (one thread): TMA bulk copies, S tiles ahead
    if (lane != 0) return;
    const uint64_t pol = l2_evict_first_policy();
    unsigned g = 0;
    if (pro_ok && nq > 0) {
      for (;; ++g) {
        const int s = (int)(g % S);
        if (g >= (unsigned)S) {
          const unsigned par = ((g / S) - 1u) & 1u;
          bool got = false;
          const uint64_t t0 = globaltimer_ns();
          for (unsigned spins = 1;; ++spins) {
            if (mbar_try_wait(&empty[s], par)) { got = true; break; }
            if (s_stop) break;
            if ((spins & 63u) == 0u && globaltimer_ns() - t0 > a.timeout_ns) {
              atomicCAS(&a.bar->status, kStatusOk, kStatusTimeout);
              break;
            }
          }
          if (!got) break;
        }
        const int tri0 = ((int)blockIdx.x + (int)(g % (unsigned)nq) * (int)nb) * TT;
        const int nt = min(TT, ne - tri0);
        const uint32_t bytes = (uint32_t)(nt * NPHI * 16);
        unsigned char* dst = stages + (size_t)s * C::STAGE;
        fence_proxy_async_smem();
        mbar_expect_tx(&full[s], bytes * (NG + NGP));
#pragma unroll 1
        for (int c = 0; c < NG; ++c)
          bulk_g2s_hint(dst + (size_t)c * TR * 16, a.vals + ((size_t)c * a.n + (size_t)tri0 * NPHI) * VEC, bytes,
                        &full[s], pol);
#pragma unroll 1
        for (int c = 0; c < NGP; ++c)
          bulk_g2s_hint(dst + C::PBLK + (size_t)c * TR * 16, a.pinv + ((size_t)c * a.n + (size_t)tri0 * NPHI) * VP,
                        bytes, &full[s], pol);
      }
    }
    // no CTA leaves with a bulk copy still writing its shared memory
    for (unsigned h = g > (unsigned)S ? g - S : 0u; h < g; ++h)
      if (!mbar_wait_bounded(&full[h % S], (h / S) & 1u, a.timeout_ns))
        atomicCAS(&a.bar->status, kStatusOk, kStatusTimeout);
    return;
  }

  if (warp >= kGatherWarp) {
    // ---- gather producers (NGW warps): cp.async of r, w, s of the coupled
    // blocks and of the own p, x (PRE: p, x, u) and areas, after the pass has
    // been opened; gather thread gl takes the blocks gl, gl + 32 NGW, ...
    constexpr int GT = 32 * NGW;
    const int gl = (warp - kGatherWarp) * 32 + lane;
    constexpr int NBL = (NB + GT - 1) / GT;
    int cn[NBL];
    auto load_cols = [&](unsigned gg, int (&c)[NBL]) {
      const int tri0 = ((int)blockIdx.x + (int)(gg % (unsigned)nq) * (int)nb) * TT;
      const int nt = min(TT, ne - tri0);
#pragma unroll
      for (int j = 0; j < NBL; ++j) {
        const int b = gl + GT * j;
        c[j] = b < 4 * nt ? __ldg(a.cols + (size_t)(b & 3) * a.ne_pad + tri0 + (b >> 2)) : -1;
      }
    };
    bool ok = pro_ok && nq > 0;
    if (ok) load_cols(0u, cn);
    for (unsigned g = 0; ok; ++g) {
      const unsigned q = g % (unsigned)nq;
      const int pass = (int)(g / (unsigned)nq);
      if (q == 0) {
        // The pass may be gathered once every CTA has arrived at the barrier
        // that ends the previous one (the prologue's for pass 0): their vector
        // writes are then complete.  The totals (alpha, beta) are not needed
        // here, so these copies overlap the rest of the reduction.
        int go = 0;  // 1: gather, 0: stop, -1: error
        if (lane == 0) {
          const unsigned long long target = (unsigned long long)(2 + pass) * nb;
          const uint64_t t0 = globaltimer_ns();
          for (unsigned spins = 1;; ++spins) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(&a.bar->count) : "memory");
            if (v >= target) { go = 1; break; }
            if (s_stop) break;
            if (*((volatile int*)&a.bar->status) != kStatusOk) break;
            if ((spins & 63u) == 0u && globaltimer_ns() - t0 > a.timeout_ns) {
              atomicCAS(&a.bar->status, kStatusOk, kStatusTimeout);
              go = -1;
              break;
            }
          }
        }
        go = __shfl_sync(0xffffffffu, go, 0);
        __syncwarp();  // orders the other lanes' copies after lane 0's acquire
        if (go != 1) break;
      }
      const int s = (int)(g % S);
      if (g >= (unsigned)S) {
        const unsigned par = ((g / S) - 1u) & 1u;
        bool got = false;
        const uint64_t t0 = globaltimer_ns();
        for (unsigned spins = 1;; ++spins) {
          if (mbar_try_wait(&empty[s], par)) { got = true; break; }
          if (s_stop) break;
          if ((spins & 63u) == 0u && globaltimer_ns() - t0 > a.timeout_ns) break;
        }
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0 && !s_stop) atomicCAS(&a.bar->status, kStatusOk, kStatusTimeout);
          break;
        }
      }
      int cc[NBL];
#pragma unroll
      for (int j = 0; j < NBL; ++j) cc[j] = cn[j];
      load_cols(g + 1u, cn);  // next tile's indices (the same tiles recur every pass)
      const int tri0 = ((int)blockIdx.x + (int)q * (int)nb) * TT;
      const int nt = min(TT, ne - tri0);
      unsigned char* st = stages + (size_t)s * C::STAGE;
      const V* ro = rbuf(pass);
      const V* wo = wbuf(pass);
      const V* so = sbuf(pass);
#pragma unroll
      for (int j = 0; j < NBL; ++j) {
        if (cc[j] < 0) continue;
        const int b = gl + GT * j;
        const int64_t src = (int64_t)cc[j] * NPAD;
        unsigned char* d = st + C::GATHER + (size_t)b * NPAD * sizeof(V);
#pragma unroll
        for (int c = 0; c < CPB; ++c) {
          cp_async16(d + c * 16, ro + src + c * VPC);
          cp_async16(d + (size_t)NB * NPAD * sizeof(V) + c * 16, wo + src + c * VPC);
          cp_async16(d + (size_t)2 * NB * NPAD * sizeof(V) + c * 16, so + src + c * VPC);
        }
      }
      const int own = nt * CPB;  // 16-byte chunks of one own vector
      for (int c = gl; c < NOWN * own; c += GT) {
        const int v = c >= 2 * own ? 2 : c >= own ? 1 : 0;  // own vector v: p, x, u
        const int cx = c - v * own;
        cp_async16(st + C::OWN + (size_t)v * TT * NPAD * sizeof(V) + cx * 16,
                   a.vec + (int64_t)v * npv + (int64_t)tri0 * NPAD + cx * VPC);
      }
      if (a.coefM != V(0))
        for (int c = gl; c < nt; c += GT) cp_async8_ca(st + C::AREA + c * 8, a.area + tri0 + c);
      cp_async_arrive(&gfull[s]);
    }
    cp_async_wait_all();
    return;
  }

  // ---- consumer warps: one matrix row per thread
  int it = 0;
  double rr = 0.0, rr0 = 0.0;
  bool ok = pro_ok && nq > 0;
  if (threadIdx.x == 0 && !ok) s_stop = 1;
  {
    V alpha = V(0), beta = V(0), muw = V(0), muu = V(0), g_old = V(0), a_old = V(0);
    double stop = 0.0;
    const double inv_n = 1.0 / (double)a.n;
    unsigned g = 0;  // this CTA's tile sequence number (continues across passes)
    for (int pass = 0; ok; ++pass) {
      V* const rn = rbuf(pass + 1);
      V* const wn = wbuf(pass + 1);
      V* const sn = sbuf(pass + 1);
      // partial sums: r.r, w.r, sum w, sum r  (PRE: r.u, w.u, sum w, sum u, r.r, sum r)
      V g0 = V(0), g1 = V(0), g2 = V(0), g3 = V(0), g4 = V(0), g5 = V(0);
      for (int q = 0; q < nq; ++q, ++g) {
        const int s = (int)(g % S);
        const unsigned par = (g / S) & 1u;
        const int tri0 = ((int)blockIdx.x + q * (int)nb) * TT;
        const int nt = min(TT, ne - tri0);
        bool got = mbar_wait_bounded(&full[s], par, a.timeout_ns);
        got = got && mbar_wait_bounded(&gfull[s], par, a.timeout_ns);
        const unsigned char* st = stages + (size_t)s * C::STAGE;
        const V* gr = reinterpret_cast<const V*>(st + C::GATHER);
        const V* gw = gr + NB * NPAD;
        const V* gs = gw + NB * NPAD;
        V* const xs_all = s_rn[g & 1u];
        // new residual of the 4 coupled blocks of every tile triangle
        for (int i = threadIdx.x; i < nt * 4 * NPHI; i += kCgConsumers) {
          const int tb = i / NPHI, kk = i - tb * NPHI;
          const int o = tb * NPAD + kk;
          xs_all[i] = fma(-alpha, fma(beta, gs[o], gw[o] - muw), gr[o]);
        }
        if (!cbar_and(got)) {
          ok = false;
          break;
        }
        if ((int)threadIdx.x < nt * NPHI) {
          const int lt = threadIdx.x / NPHI, k = threadIdx.x - lt * NPHI;
          const V* xs = xs_all + lt * 4 * NPHI;
          const unsigned char* sv = st + (size_t)threadIdx.x * 16;
          // the operator's couplings in difference form (those of A P plainly)
          constexpr bool DIFF = !PRE && DiffForm<T>::value;
          const V xrow = DIFF ? xs[k] : V(0);
          V wv = V(0);
#pragma unroll
          for (int gg = 0; gg < NG; ++gg) {
            typename ValOf<T>::type v[VEC];
            lds_vals<T, VEC>(sv + (size_t)gg * TR * 16, v);
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
              const int c = gg * VEC + u;
              if (c < NC) wv = fma((V)v[u], DIFF ? xs[c] - xrow : xs[c], wv);
            }
          }
          wv *= a.coefK;
          if (a.coefM != V(0)) {
            V mv = V(0);
#pragma unroll
            for (int kk = 0; kk < NPHI; ++kk) mv = fma((V)s_Mref[k * NPHI + kk], xs[kk], mv);
            const double ar = reinterpret_cast<const double*>(st + C::AREA)[lt];
            wv = fma(a.coefM * (V)ar, mv, wv);
          }
          const int o = lt * 4 * NPAD + k;  // own block of triangle lt among the gathered
          const V* own = reinterpret_cast<const V*>(st + C::OWN) + lt * NPAD + k;
          const V w_old = gw[o] - muw;
          const V s_old = gs[o];
          const V p_old = own[0];
          const V x_old = own[TT * NPAD];
          // p = r + beta p  (PRE: p = Pi u + beta p)
          V d_old;
          if constexpr (PRE) d_old = own[2 * TT * NPAD] - muu;
          else d_old = gr[o];
          const V p_new = fma(beta, p_old, d_old);
          const V s_new = fma(beta, s_old, w_old);
          const V r_new = xs[k];
          const int64_t prow = (int64_t)(tri0 + lt) * NPAD + k;
          pp[prow] = p_new;
          xp[prow] = fma(alpha, p_new, x_old);
          sn[prow] = s_new;
          rn[prow] = r_new;
          wn[prow] = wv;
          if constexpr (PRE) {
            // u = P_i r from the streamed rows of P and the own residual block
            const unsigned char* pv = st + C::PBLK + (size_t)threadIdx.x * 16;
            V u = V(0);
#pragma unroll
            for (int gg = 0; gg < NGP; ++gg) {
              V v[VP];
              lds16(pv + (size_t)gg * TR * 16, v);
#pragma unroll
              for (int l4 = 0; l4 < VP; ++l4) {
                const int l = gg * VP + l4;
                if (l < NPHI) u = fma(v[l4], xs[l], u);
              }
            }
            up[prow] = u;
            g0 = fma(r_new, u, g0);
            g1 = fma(wv, u, g1);
            g2 += wv;
            g3 += u;
            g4 = fma(r_new, r_new, g4);
            g5 += r_new;
          } else {
            g0 = fma(r_new, r_new, g0);
            g1 = fma(wv, r_new, g1);
            g2 += wv;
            g3 += r_new;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
      }
      if (!ok) break;
      constexpr int NW = PRE ? 6 : 4;
      V acc[NW];
      acc[0] = g0;
      acc[1] = g1;
      acc[2] = g2;
      acc[3] = g3;
      if constexpr (NW > 4) {
        acc[4] = g4;
        acc[NW - 1] = g5;
      }
      double tot[NW];
      if (!consumer_allreduce<NW, V>(a.bar, a.part, nb, epoch, a.timeout_ns, acc, tot)) {
        ok = false;
        break;
      }
      // scalar recurrences in V: FP64 division is slow on this GPU and the
      // FP32 inner solve carries its scalars in FP32 anyway
      const double mu = a.mean_zero ? tot[2] * inv_n : 0.0;  // mean of w
      // PRE: u enters as Pi u = u - mu_u 1
      const double mu_u = PRE && a.mean_zero ? tot[3] * inv_n : 0.0;
      const double gg = PRE ? tot[0] - mu_u * tot[NW - 1] : tot[0];  // gamma: r.r (PRE: r . Pi u)
      const V gv = (V)gg;
      const V dv = (V)(tot[1] - mu * tot[3]);  // (w - mu 1) . r  (PRE: . Pi u)
      if constexpr (PRE) rr = tot[4];  // r.r
      else rr = gg;
      V an, bn;
      if (pass == 0) {
        rr0 = rr;
        stop = a.stop_rel * a.stop_rel * rr0;
        bn = V(0);
        an = gv / dv;
      } else {
        ++it;
        bn = gv / g_old;
        an = gv / (dv - bn * gv / a_old);
      }
      if (!(rr > stop) || it >= a.max_iters || !(an > V(0)) || !isfinite(an)) break;
      g_old = gv;
      a_old = an;
      alpha = an;
      beta = bn;
      muw = (V)mu;
      muu = (V)mu_u;
    }
  }
  if (threadIdx.x == 0) {
    if (!ok && pro_ok) atomicCAS(&a.bar->status, kStatusOk, kStatusTimeout);
    s_stop = 1;  // the producer warps stop at their next wait
  }
  // the caller's x, unpadded (each thread wrote these rows itself in the last pass)
  for (int q = 0; q < nq; ++q) {
    const int tri0 = ((int)blockIdx.x + q * (int)nb) * TT;
    const int nt = min(TT, ne - tri0);
    if ((int)threadIdx.x < nt * NPHI) {
      const int lt = threadIdx.x / NPHI, k = threadIdx.x - lt * NPHI;
      a.x[(int64_t)tri0 * NPHI + threadIdx.x] = xp[(int64_t)(tri0 + lt) * NPAD + k];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.res->iters = it;
    a.res->rr0 = rr0;
    a.res->rr = rr;
    a.res->status = *((volatile int*)&a.bar->status);
  }
}

template <int NPHI, typename T, typename V, bool PRE, int NGW>
__global__ void __launch_bounds__(CgThreads<NGW>::value, 1) k_cg(CGParams<T, V> a) {
  cg_body<NPHI, T, V, PRE, NGW>(a);
}

// The same kernel with at most 96 registers per thread.  A CTA of 6 warps then
// needs 5 warps' registers per SM sub-partition at 3 CTAs per SM (5 x 32 x 96
// = 15,360 of 16,384); at the uncapped 102 registers (FP32 couplings, p = 2)
// only 2 CTAs fit, although their shared memory would allow 3.
template <int NPHI, typename T, typename V, bool PRE, int NGW>
__global__ void __maxnreg__(96) k_cg_r96(CGParams<T, V> a) {
  cg_body<NPHI, T, V, PRE, NGW>(a);
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

// FMA throughput probe: every thread runs 8 independent chains x <- x a + b
// (no memory traffic inside the loop); the chains' sum is stored so that
// nothing is optimised away.
template <typename V>
__global__ void __launch_bounds__(256) k_fma_rate(V* out, int iters, V a, V b) {
  V x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (V)(threadIdx.x + i) * (V)1e-3;
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  V acc = V(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) acc += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

cudaError_t launch_fma_rate(int fp64, void* out, int blocks, int iters, cudaStream_t s) {
  if (fp64)
    k_fma_rate<double><<<blocks, 256, 0, s>>>(static_cast<double*>(out), iters, 0.999999, 1e-7);
  else
    k_fma_rate<float><<<blocks, 256, 0, s>>>(static_cast<float*>(out), iters, 0.999999f, 1e-7f);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_selftest_wait(GridBarrier* bar, int which, uint64_t timeout_ns, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  if (err != cudaSuccess) return err;
  k_selftest_wait<<<which == 0 ? 2 : 1, 64, 0, s>>>(bar, which, timeout_ns);
  count_launch();
  return cudaGetLastError();
}

// Gather warps per CTA of the persistent CG, by degree and coupling width: a
// table filled from an offline sweep (a deterministic lookup: the choice
// depends on the system only, never on timing at run time, and does not
// change the result's bits: the tiles, the grid and the reduction order are
// the same).
// DGSL_CG_GATHER_WARPS (1 or 2) overrides the table, for sweeps.
int cg_gather_warps(const DevOp& op, size_t coupling_bytes, bool pre) {
  if (const char* e = std::getenv("DGSL_CG_GATHER_WARPS")) {
    const int v = std::atoi(e);
    if (v == 1 || v == 2) return v;
  }
  // swept at 256^2, 512^2, 1024^2 (50-iteration launches): a second gather warp
  // gains 3-6% with plain FP32 couplings at p = 3; at p = 1 and 4 it changes
  // nothing, and with BF16 couplings it costs the third CTA per SM (up to 24%
  // slower).  FP32 at p = 2 keeps one: its register-capped kernel then fits 3
  // CTAs per SM (two gather warps would need 7 warps' registers per CTA).  FP64
  // and block-Jacobi kernels keep one.
  return (coupling_bytes == 4 && !pre && op.nphi == 10) ? 2 : 1;
}

namespace {
// FP32 couplings at p = 2 with one gather warp run the register-capped kernel
// (3 CTAs per SM instead of 2); every other configuration the plain one.  Only
// the kernel selected is instantiated.
template <int NPHI, typename T, typename V, bool PRE, int NGW>
constexpr auto cg_kernel() {
  if constexpr (NPHI == 6 && sizeof(T) == 4 && !PRE && NGW == 1)
    return k_cg_r96<NPHI, T, V, PRE, NGW>;
  else
    return k_cg<NPHI, T, V, PRE, NGW>;
}

template <class KernelT>
int coop_blocks(KernelT kern, int threads, size_t dyn_smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, dyn_smem);
  per = std::max(1, std::min(per, 8));
  return sms * per;
}

template <int NPHI, typename T, typename V, bool PRE, int NGW>
cudaError_t run_cg_ngw(const DevOp& op, const T* vals, const V* pinv, V coefK, V coefM, int mean_zero, V* x, V* r,
                       double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s,
                       int* grid_used) {
  auto kern = cg_kernel<NPHI, T, V, PRE, NGW>();
  constexpr int threads = CgThreads<NGW>::value;
  using Cfg = TileCfg<NPHI, T, V, PRE>;
  const size_t dyn = Cfg::S * (size_t)Cfg::STAGE;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (err != cudaSuccess) return err;
  const int ntiles = (op.ne + Cfg::TT - 1) / Cfg::TT;
  int blocks = std::min(coop_blocks(kern, threads, dyn), w.max_parts);
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
  a.pinv = pinv;
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
  err = cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(threads), args, dyn, s);
  count_launch();
  return err;
}

template <int NPHI, typename T, typename V, bool PRE>
cudaError_t run_cg(const DevOp& op, const T* vals, const V* pinv, V coefK, V coefM, int mean_zero, V* x, V* r,
                   double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns, cudaStream_t s,
                   int* grid_used) {
  // gather warps per CTA from the tuning table (the result does not depend on it:
  // the tile order, the grid and the reduction order are the same)
  if (cg_gather_warps(op, sizeof(T), PRE) == 2)
    return run_cg_ngw<NPHI, T, V, PRE, 2>(op, vals, pinv, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w,
                                          timeout_ns, s, grid_used);
  return run_cg_ngw<NPHI, T, V, PRE, 1>(op, vals, pinv, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w,
                                        timeout_ns, s, grid_used);
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

// Bytes of the persistent CG's vectors: 8 vectors of ne blocks (9 with the
// block-Jacobi preconditioner), each block N_phi values padded to a whole
// number of 16-byte chunks (the larger of the FP32 and FP64 layouts, so one
// buffer serves every precision).
size_t cg_vec_bytes(const DevOp& op, int precond) {
  const size_t pad32 = (size_t)(op.nphi + 3) / 4 * 4 * sizeof(float);
  const size_t pad64 = (size_t)(op.nphi + 1) / 2 * 2 * sizeof(double);
  return (precond ? 9 : 8) * (size_t)op.ne * std::max(pad32, pad64) + 256;
}

#define DGSL_CG_RUN(NPHI, T, V, VALS)                                                                           \
  (pinv ? run_cg<NPHI, T, V, true>(op, VALS, pinv, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w,      \
                                   timeout_ns, s, grid_used)                                                   \
        : run_cg<NPHI, T, V, false>(op, VALS, nullptr, coefK, coefM, mean_zero, x, r, stop_rel, max_iters, w,  \
                                    timeout_ns, s, grid_used))
#define DGSL_CG_CASES(T, V, VALS)          \
  switch (op.p) {                          \
    case 1: return DGSL_CG_RUN(3, T, V, VALS);  \
    case 2: return DGSL_CG_RUN(6, T, V, VALS);  \
    case 3: return DGSL_CG_RUN(10, T, V, VALS); \
    case 4: return DGSL_CG_RUN(15, T, V, VALS); \
  }                                        \
  return cudaErrorInvalidValue;

// With a preconditioned operator the couplings are those of A P, which
// include coefK and the mass term: the kernel then runs with coefK = 1, coefM = 0.
cudaError_t launch_cg_f64(const DevOp& op, double coefK, double coefM, int mean_zero, double* x, double* r,
                          const PrecondOp* pre, double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns,
                          cudaStream_t s, int* grid_used) {
  if (!op.K64 || (pre && (!pre->ap || !pre->pinv))) return cudaErrorInvalidValue;
  const double* pinv = pre ? static_cast<const double*>(pre->pinv) : nullptr;
  const double* vals = pre ? static_cast<const double*>(pre->ap) : op.K64;
  if (pre) {
    coefK = 1.0;
    coefM = 0.0;
  }
  DGSL_CG_CASES(double, double, vals)
}

cudaError_t launch_cg_f32(const DevOp& op, int bf16, float coefK, float coefM, int mean_zero, float* x, float* r,
                          const PrecondOp* pre, double stop_rel, int max_iters, const CGWork& w, uint64_t timeout_ns,
                          cudaStream_t s, int* grid_used) {
  if (pre && (!pre->ap || !pre->pinv)) return cudaErrorInvalidValue;
  const float* pinv = pre ? static_cast<const float*>(pre->pinv) : nullptr;
  if (pre) {
    coefK = 1.0f;
    coefM = 0.0f;
  }
  if (bf16) {
    const uint16_t* vals = pre ? static_cast<const uint16_t*>(pre->ap) : op.K16;
    if (!vals) return cudaErrorInvalidValue;
    DGSL_CG_CASES(uint16_t, float, vals)
  }
  const float* vals = pre ? static_cast<const float*>(pre->ap) : op.K32;
  if (!vals) return cudaErrorInvalidValue;
  DGSL_CG_CASES(float, float, vals)
}

}  // namespace dgsl

