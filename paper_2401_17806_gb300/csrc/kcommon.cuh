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

// Barrier state in device memory: count of arrivals and a generation word.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int status;      // kStatusOk, or the first error any CTA recorded
  int pad;
};

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The wait
// is bounded: after timeout_ns the CTA records kStatusTimeout and returns
// false; CTAs waiting elsewhere see the status and return false as well.
// Every CTA must call it the same number of times.
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned int nblocks, uint64_t timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &b->gen;
    volatile int* vst = &b->status;
    unsigned int g = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(&b->count, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      uint64_t t0 = globaltimer_ns();
      unsigned int spins = 0;
      while (*vgen == g) {
        if (*vst != kStatusOk) { ok = 0; break; }
        if ((++spins & 255u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
          atomicCAS(&b->status, kStatusOk, kStatusTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*vst != kStatusOk) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

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

}  // namespace dgsl
