// Row kernels of the assembled coupling form, shared by the apply kernels and
// the persistent CG kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kcommon.cuh"

namespace dgsl {

template <typename T>
struct Pack {
  static constexpr int VEC = 16 / (int)sizeof(T);
};

__device__ __forceinline__ void load16(const double* p, double (&v)[2]) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p));
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void load16(const float* p, float (&v)[4]) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void load16(const uint16_t* p, float (&v)[8]) {
  uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
  unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

template <typename T>
struct ValOf {
  using type = T;
};
template <>
struct ValOf<uint16_t> {
  using type = float;
};

// The operator's couplings are applied in difference form: every row of K
// sums to zero (K 1 = 0), so (K x)_row = sum_c a_c (x_c - x_row).  The FP32
// and BF16 copies store the self-coupling slot as 0; the FP64 copy keeps it,
// and a_self (x_row - x_row) adds nothing.  Rounded couplings and rounded
// arithmetic then still annihilate constants exactly, and the smooth
// components (the small eigenvalues) keep a relative error at the rounding
// level instead of one that grows with the condition number.  This also sets
// the accuracy floor of the FP64 refinement residual.  (The couplings of A P
// do not sum to zero and are applied plainly.)
template <typename T>
struct DiffForm {
  static constexpr bool value = true;
};

// Two consecutive values of x (8 bytes for FP32, 16 for FP64) in one load.
__device__ __forceinline__ void ld_pair(const float* p, float& a, float& b) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  a = t.x;
  b = t.y;
}
__device__ __forceinline__ void ld_pair(const double* p, double& a, double& b) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(p));
  a = t.x;
  b = t.y;
}

// Row `row` of K x.  COH: read x from L2 (x is written by other CTAs of a
// persistent launch).  DIFF: couplings in difference form.  PAIR (even N_phi
// only): read the coupled blocks of x two values per load, which needs x
// aligned to two values (the callers' own allocations); the products and
// their order are the same.
template <int NPHI, typename T, typename V, bool COH, bool DIFF = DiffForm<T>::value, bool PAIR = false>
__device__ __forceinline__ V assembled_row(const T* __restrict__ vals, const int32_t* __restrict__ cols,
                                           int ne, int64_t n, int64_t row, const V* x) {
  static_assert(!PAIR || (NPHI % 2 == 0 && !COH), "pair loads need an even block length");
  constexpr int VEC = Pack<T>::VEC;
  constexpr int NC = 4 * NPHI;
  constexpr int NG = (NC + VEC - 1) / VEC;
  const int i = (int)(row / NPHI);
  int col[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) col[b] = __ldg(cols + (size_t)b * ne + i);
  V xr = V(0);
  if (DIFF) xr = COH ? ldcg(x + row) : __ldg(x + row);
  V acc = V(0);
  V xodd = V(0);  // PAIR: the second value of the last pair
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    typename ValOf<T>::type v[VEC];
    load16(vals + ((size_t)g * n + row) * VEC, v);
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
      const int c = g * VEC + u;
      if (c < NC) {
        const int b = c / NPHI, kk = c % NPHI;
        const V* xp = x + (size_t)col[b] * NPHI + kk;
        V xv;
        if constexpr (PAIR) {
          if (kk % 2 == 0)
            ld_pair(xp, xv, xodd);
          else
            xv = xodd;
        } else {
          xv = COH ? ldcg(xp) : __ldg(xp);
        }
        acc = fma((V)v[u], DIFF ? xv - xr : xv, acc);
      }
    }
  }
  return acc;
}

// (Mbar x)_row = A_i sum_kk Mref[k][kk] x_i[kk]   (eq. MassMatrixM)
template <int NPHI, typename V, bool COH>
__device__ __forceinline__ V mass_row(const double* __restrict__ area, const double* __restrict__ Mref,
                                      int64_t row, const V* x) {
  const int i = (int)(row / NPHI), k = (int)(row % NPHI);
  V acc = V(0);
#pragma unroll
  for (int kk = 0; kk < NPHI; ++kk) {
    const V* xp = x + (size_t)i * NPHI + kk;
    acc = fma((V)__ldg(Mref + k * NPHI + kk), COH ? ldcg(xp) : __ldg(xp), acc);
  }
  return (V)__ldg(area + i) * acc;
}


}  // namespace dgsl
