// Internal definition of the operator handle shared by the C-ABI translation
// units (api.cu, server.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "host.h"
#include "kernels.h"

#define DGSL_CUDA(expr)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) throw Error(DGSL_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Sets the thread-local message returned by dgsl_last_error().
void dgsl_set_last_error(const std::string& msg);

using dgsl::CGResult;
using dgsl::DevOp;
using dgsl::Error;
using dgsl::GridBarrier;
using dgsl::HostBlocks;
using dgsl::HostMesh;
using dgsl::RefOps;

// NVTX range around a library phase (build, solve, batch, serving round), for
// Nsight timelines; header-only NVTX 3, inert unless a profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct dgsl_operator {
  HostMesh hm;
  RefOps ro;
  HostBlocks hb;      // kept for host queries (host_only or factored builds)
  bool have_blocks = false;
  int host_only = 0;
  DevOp d;
  std::vector<void*> allocs;
  int64_t device_bytes = 0;
  std::mutex mu;
  // solve workspace (grown on demand)
  struct Work {
    int64_t n = 0;
    double* r64 = nullptr;
    double* d64 = nullptr;
    float* r32 = nullptr;
    float* d32 = nullptr;
    void* vec = nullptr;  // cg_vec_bytes(d): persistent CG vectors
    double* part = nullptr;
    double* part2 = nullptr;
    GridBarrier* bar = nullptr;
    CGResult* res = nullptr;
    double* h_part = nullptr;   // pinned
    CGResult* h_res = nullptr;  // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int max_parts = 0;
  } w;

  template <class T>
  T* dalloc(size_t count) {
    void* p = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) throw Error(DGSL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(p);
    device_bytes += (int64_t)bytes;
    return static_cast<T*>(p);
  }
  template <class T>
  T* upload(const std::vector<T>& v) {
    T* p = dalloc<T>(v.size());
    if (!v.empty()) DGSL_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
  }
  ~dgsl_operator() {
    if (!host_only) {
      cudaSetDevice(d.device);
      for (void* p : allocs) cudaFree(p);
      if (w.h_part) cudaFreeHost(w.h_part);
      if (w.h_res) cudaFreeHost(w.h_res);
      if (w.ev0) cudaEventDestroy(w.ev0);
      if (w.ev1) cudaEventDestroy(w.ev1);
    }
  }
  void ensure_work() {
    if (w.n == d.n && w.r64) return;
    w.n = d.n;
    w.max_parts = cg_max_blocks(d, 0);
    w.r64 = dalloc<double>(d.n);
    w.d64 = dalloc<double>(d.n);
    w.r32 = dalloc<float>(d.n);
    w.d32 = dalloc<float>(d.n);
    w.vec = dalloc<double>((cg_vec_bytes(d) + 7) / 8);
    w.part = dalloc<double>(8 * (size_t)w.max_parts);  // two halves of 4 sums per CTA
    w.part2 = dalloc<double>(2 * (size_t)w.max_parts);
    w.bar = dalloc<GridBarrier>(1);
    w.res = dalloc<CGResult>(1);
    DGSL_CUDA(cudaMallocHost(&w.h_part, 2 * (size_t)w.max_parts * sizeof(double)));
    DGSL_CUDA(cudaMallocHost(&w.h_res, sizeof(CGResult)));
    DGSL_CUDA(cudaEventCreate(&w.ev0));
    DGSL_CUDA(cudaEventCreate(&w.ev1));
  }
};

