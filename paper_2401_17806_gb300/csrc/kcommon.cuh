// Device helpers shared by the dgsl kernels: L2-coherent loads for data that
// other CTAs write during a persistent launch, a bounded grid barrier and
// deterministic block reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dgsl {

constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 6;  // DGSL_ETIMEOUT

// Loads that bypass L1: L1 is not coherent between SMs, so values written by
// other CTAs of the same persistent launch must be read from L2.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier state in device memory (zeroed before every persistent launch):
// a monotonic arrival counter (alone in its 128-byte line: every CTA adds to
// it), the epoch released by the last arriver of a reducing barrier, the first
// error any CTA recorded, and the reduced totals (polled by every CTA).
struct alignas(128) GridBarrier {
  unsigned long long count;
  unsigned long long pad0[15];
  unsigned long long gen;
  int status;
  int pad;
  double total[4];
  unsigned long long pad1[10];
};
static_assert(sizeof(GridBarrier) == 256, "GridBarrier is two 128-byte lines");

// Sum of v over the block (blockDim.x a multiple of 32, <= 1024).  The
// summation order is fixed by thread index, so it is deterministic.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double s_red[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) s_red[wid][i] = v[i];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = lane < nw ? s_red[lane][i] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[i] = x;
    }
  }
  __syncthreads();
}

// Sum of the per-CTA partials part[0..nparts) (stride NV), computed by every
// CTA in the same fixed order, so all CTAs obtain bit-identical totals.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* part, int nparts, double (&out)[NV]) {
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = 0.0;
  for (int j = threadIdx.x; j < nparts; j += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __ldcg(part + (size_t)j * NV + i);
  block_sum<NV>(v);
  __shared__ double s_tot[NV];
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) s_tot[i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = s_tot[i];
  __syncthreads();
}

// ---- TMA bulk copies (non-tensor) with mbarrier completion, CTA scope.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Orders prior generic-proxy accesses of shared memory before later async-proxy
// (TMA) accesses, and makes mbarrier initialisation visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// L2 policy for data streamed once per use (evicted first, so that data
// reused across CTAs, e.g. the CG vectors, stays resident).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// bulk_g2s with an L2 cache-eviction hint for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for phase `parity` of `bar`; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (unsigned spins = 1;; ++spins) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spins & 255u) == 0u && globaltimer_ns() - t0 > timeout_ns) return false;
  }
}

}  // namespace dgsl
