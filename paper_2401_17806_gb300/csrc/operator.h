// Internal definition of the operator handle shared by the C-ABI translation
// units (api.cu, server.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "host.h"
#include "kernels.h"
#include "mg.h"

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
  // semi-Lagrangian walk data (built on first use) and its workspace
  struct SL {
    dgsl::SLDev g;
    bool built = false;
    double* vmono = nullptr;
    double* cmono = nullptr;
    size_t cmono_cap = 0;
    int* err = nullptr;
    int* h_err = nullptr;  // pinned
  } sl;
  // workspace of dgsl_ns_step: vbar | c | Mbar c | vbar* (2 n each) | vhat* (2 nd npsi) | b (n) | p_prev (n)
  double* ns = nullptr;
  bool ns_prev_valid = false;  // p_prev holds the pressure of the last step that asked for extrapolation
  // workspace of dgsl_advdiff_step: V (4 stages x 2 per trajectory) | fields (5 n) | ci | rhs | c* (n each)
  double* ad = nullptr;
  // workspace of dgsl_ns_imex_step: V (8 per trajectory) | fields (5 x 2 n) | vI, vst, rhs (2 n each) |
  // b, pr, tmp (n each) | vhs, vIh, vs (2 nd npsi each)
  double* nsi = nullptr;
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
    // block-Jacobi preconditioned operators (A P and P) of recent systems
    // (coefficients and coupling type): up to kKeep kept; an entry in use by a
    // solve, a batch or an admitted server request (refs > 0) is never
    // rebuilt; otherwise the least recently used is replaced first
    struct Precond {
      dgsl::PrecondOp op;
      void* ap = nullptr;
      void* pinv = nullptr;
      size_t ap_bytes = 0, pinv_bytes = 0;
      double coefK = 0.0, coefM = 0.0;
      int type = 0;
      uint64_t used = 0;
      bool valid = false;
      std::atomic<int> refs{0};
    };
    static constexpr size_t kKeep = 4;
    std::vector<std::unique_ptr<Precond>> pj;
    uint64_t pj_clock = 0;
    double* p64 = nullptr;  // FP64 P while building (FP32 / BF16 systems)
    int* pj_bad = nullptr;
    int* h_pj_bad = nullptr;  // pinned
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
  // Stream of host-to-device copies: the build's stream (dgsl_build_opts.stream)
  // while dgsl_build_operators runs, the legacy default stream afterwards.
  cudaStream_t upload_stream = nullptr;
  template <class T>
  T* upload(const std::vector<T>& v) {
    T* p = dalloc<T>(v.size());
    if (!v.empty()) {
      DGSL_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, upload_stream));
      DGSL_CUDA(cudaStreamSynchronize(upload_stream));  // v may be a temporary
    }
    return p;
  }
  ~dgsl_operator() {
    if (!host_only) {
      cudaSetDevice(d.device);
      for (void* p : allocs) cudaFree(p);
      if (w.h_part) cudaFreeHost(w.h_part);
      if (w.h_res) cudaFreeHost(w.h_res);
      if (w.h_pj_bad) cudaFreeHost(w.h_pj_bad);
      if (sl.h_err) cudaFreeHost(sl.h_err);
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
    w.vec = dalloc<double>((cg_vec_bytes(d, 1) + 7) / 8);
    w.part = dalloc<double>(12 * (size_t)w.max_parts);  // two halves of up to 6 sums per CTA
    w.part2 = dalloc<double>(2 * (size_t)w.max_parts);
    w.bar = dalloc<GridBarrier>(1);
    w.res = dalloc<CGResult>(1);
    DGSL_CUDA(cudaMallocHost(&w.h_part, 2 * (size_t)w.max_parts * sizeof(double)));
    DGSL_CUDA(cudaMallocHost(&w.h_res, sizeof(CGResult)));
    DGSL_CUDA(cudaEventCreate(&w.ev0));
    DGSL_CUDA(cudaEventCreate(&w.ev1));
  }
  // Workspace of dgsl_ns_step (caller holds mu).
  double* ensure_ns() {
    if (!ns) ns = dalloc<double>((size_t)10 * d.n + (size_t)2 * d.nd * d.npsi);
    return ns;
  }
  // Workspace of dgsl_advdiff_step (caller holds mu, after ensure_sl).
  double* ensure_advdiff() {
    if (!ad) ad = dalloc<double>((size_t)8 * d.ne * sl.g.ng + (size_t)8 * d.n);
    return ad;
  }
  // Workspace of dgsl_ns_imex_step (caller holds mu, after ensure_sl).
  double* ensure_nsimex() {
    if (!nsi)
      nsi = dalloc<double>((size_t)8 * d.ne * sl.g.ng + (size_t)19 * d.n + (size_t)6 * d.nd * d.npsi);
    return nsi;
  }
  // Semi-Lagrangian walk data and workspace for nf fields (caller holds mu).
  void ensure_sl(int nf) {
    if (!sl.built) {
      dgsl::SLHost h = dgsl::build_sl_host(hm, ro);
      sl.g.p = h.p;
      sl.g.nphi = h.nphi;
      sl.g.ng = h.ng;
      sl.g.ne = d.ne;
      sl.g.tri = upload(h.tri);
      sl.g.nbr = upload(h.nbr);
      sl.g.mono_c = upload(h.mono_c);
      sl.g.pts = upload(h.pts);
      sl.g.q = upload(h.q);
      sl.vmono = dalloc<double>((size_t)d.ne * 2 * d.nphi);
      sl.err = dalloc<int>(1);
      DGSL_CUDA(cudaMallocHost(&sl.h_err, sizeof(int)));
      sl.built = true;
    }
    const size_t need = (size_t)nf * d.ne * d.nphi;
    if (need > sl.cmono_cap) {
      sl.cmono = dalloc<double>(need);  // (a smaller one stays allocated until destroy)
      sl.cmono_cap = need;
    }
  }
  // Block-Jacobi preconditioned operator for A = coefM Mbar + coefK K with
  // couplings of type 0 (FP32), 1 (FP64) or 2 (BF16), built on stream s unless
  // kept from an earlier solve, and held (refs + 1) until release_precond.
  // The caller holds mu and has called ensure_work.
  Work::Precond* acquire_precond(double coefK, double coefM, int type, cudaStream_t s) {
    ++w.pj_clock;
    for (auto& e : w.pj)
      if (e->valid && e->coefK == coefK && e->coefM == coefM && e->type == type) {
        e->used = w.pj_clock;
        e->refs.fetch_add(1);
        return e.get();
      }
    Work::Precond* slot = nullptr;
    if (w.pj.size() >= Work::kKeep)
      for (auto& e : w.pj)
        if (e->refs.load() == 0 && (!slot || (!e->valid && slot->valid) || (e->valid == slot->valid && e->used < slot->used)))
          slot = e.get();
    if (!slot) {
      w.pj.push_back(std::make_unique<Work::Precond>());
      slot = w.pj.back().get();
    }
    Work::Precond& c = *slot;
    c.valid = false;
    // (a buffer too small for a new type is replaced; the old one stays allocated until destroy)
    const size_t need_ap = dgsl::precond_ap_bytes(d, type), need_p = dgsl::precond_pinv_bytes(d, type);
    if (c.ap_bytes < need_ap) {
      c.ap = dalloc<double>((need_ap + 7) / 8);
      c.ap_bytes = need_ap;
    }
    if (c.pinv_bytes < need_p) {
      c.pinv = dalloc<double>((need_p + 7) / 8);
      c.pinv_bytes = need_p;
    }
    if (type != 1 && !w.p64) w.p64 = dalloc<double>((dgsl::precond_pinv_bytes(d, 1) + 7) / 8);
    if (!w.pj_bad) {
      w.pj_bad = dalloc<int>(1);
      DGSL_CUDA(cudaMallocHost(&w.h_pj_bad, sizeof(int)));
    }
    double* p64 = type == 1 ? static_cast<double*>(c.pinv) : w.p64;
    DGSL_CUDA(cudaMemsetAsync(w.pj_bad, 0, sizeof(int), s));
    DGSL_CUDA(dgsl::launch_build_precond(d, coefK, coefM, type, c.ap, c.pinv, p64, w.pj_bad, s));
    DGSL_CUDA(cudaMemcpyAsync(w.h_pj_bad, w.pj_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    if (*w.h_pj_bad) throw Error(DGSL_EINVAL, "block-Jacobi: a diagonal block of A is not positive definite");
    c.op.ap = c.ap;
    c.op.pinv = c.pinv;
    c.coefK = coefK;
    c.coefM = coefM;
    c.type = type;
    c.used = w.pj_clock;
    c.valid = true;
    c.refs.fetch_add(1);
    return &c;
  }
  // Ends a hold taken by acquire_precond (any thread; no lock needed).
  static void release_precond(Work::Precond* c) {
    if (c) c->refs.fetch_sub(1);
  }

  // Two-level multigrid systems (k_mg.cu): the topology once per operator,
  // then one hierarchy and workspace per system (coefficients and type 0 FP32,
  // 1 FP64, 2 BF16 couplings), the last kMGKeep kept like the block-Jacobi
  // systems.  The caller holds mu.
  std::unique_ptr<dgsl::MGTopo> mgtopo;
  struct MGEntry {
    dgsl::MGSysPtr sys;
    double coefK = 0.0, coefM = 0.0;
    int type = 0;
    uint64_t used = 0;
    std::atomic<int> refs{0};
  };
  static constexpr size_t kMGKeep = 4;
  std::vector<std::unique_ptr<MGEntry>> mgs;
  uint64_t mg_clock = 0;
  MGEntry* acquire_mg(double coefK, double coefM, int type, cudaStream_t s) {
    ++mg_clock;
    for (auto& e : mgs)
      if (e->sys && e->coefK == coefK && e->coefM == coefM && e->type == type) {
        e->used = mg_clock;
        e->refs.fetch_add(1);
        return e.get();
      }
    if (!mgtopo) {
      mgtopo = dgsl::mg_topo_build(hm, d, s);
      device_bytes += mgtopo->device_bytes;
    }
    MGEntry* slot = nullptr;
    if (mgs.size() >= kMGKeep)
      for (auto& e : mgs)
        if (e->refs.load() == 0 && (!slot || e->used < slot->used)) slot = e.get();
    if (!slot) {
      mgs.push_back(std::make_unique<MGEntry>());
      slot = mgs.back().get();
    }
    device_bytes -= dgsl::mg_sys_bytes(slot->sys.get());
    slot->sys.reset();
    slot->sys = dgsl::mg_sys_build(*mgtopo, d, coefK, coefM, type, coefM == 0.0, s);
    device_bytes += dgsl::mg_sys_bytes(slot->sys.get());
    slot->coefK = coefK;
    slot->coefM = coefM;
    slot->type = type;
    slot->used = mg_clock;
    slot->refs.fetch_add(1);
    return slot;
  }
  static void release_mg(MGEntry* e) {
    if (e) e->refs.fetch_sub(1);
  }
};

