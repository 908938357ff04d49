// Device side of the two-level multigrid preconditioned CG (k_mg.cu): the
// per-operator topology (vertex numbering, coarse pattern, the reduced
// couplings Lambda^T A_ib Lambda of every triangle block) and the per-system
// hierarchy (A = coefM Mbar + coefK K) with its solve workspace.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <vector>

#include "kernels.h"
#include "mg_host.h"

namespace dgsl {

struct MGTopo {
  MGHost mg;                  // numbering and incidence (levels unused here)
  CsrD pattern, graph;        // pattern of A_0 and the vertex graph
  std::vector<int32_t> nbr;   // [ne][3] internal neighbours
  std::vector<double> Kr;     // [ne][4][3][3] Lambda^T K_(t, b) Lambda
  std::vector<double> Mr;     // [ne][3][3]    A_t Lambda^T Mref Lambda
  int32_t* d_cvid = nullptr;  // [ne][3]
  int32_t* d_v2t_ptr = nullptr;
  int32_t* d_v2t = nullptr;
  int64_t device_bytes = 0;
  ~MGTopo();
};

// Builds the topology of an operator (host mesh plus the device FP64
// couplings, reduced on the device).  Throws Error.
std::unique_ptr<MGTopo> mg_topo_build(const HostMesh& hm, const DevOp& d, cudaStream_t s);

struct MGSys;  // opaque
struct MGSysDeleter {
  void operator()(MGSys* p) const;
};
using MGSysPtr = std::unique_ptr<MGSys, MGSysDeleter>;

// type: 0 FP32 vectors with FP32 couplings, 2 FP32 vectors with BF16
// couplings, 1 FP64.  singular: the pressure operator (mean-zero solves).
MGSysPtr mg_sys_build(const MGTopo& topo, const DevOp& d, double coefK, double coefM, int type, bool singular,
                      cudaStream_t s);
int64_t mg_sys_bytes(const MGSys* m);
int mg_sys_levels(const MGSys* m, std::vector<int>* sizes);
const MGHost& mg_sys_host(const MGSys* m);

struct MGResult {
  int iters = 0;
  int status = 0;     // 0 ok, kStatusTimeout never (no waits), 1: breakdown
  double rr0 = 0.0, rr = 0.0;
  int launches = 0;
};

// Preconditioned CG on A x = b (b, x device vectors of the system's vector
// type, n values; x overwritten), stopping at ||r|| <= stop_rel ||b|| or
// max_iters.  Synchronous.
cudaError_t mg_pcg(MGSys* m, const DevOp& d, const void* b, void* x, double stop_rel, int max_iters, cudaStream_t s,
                   MGResult* res);
// One application z = M r of the preconditioner (asynchronous).
cudaError_t mg_apply(MGSys* m, const DevOp& d, const void* r, void* z, cudaStream_t s);

}  // namespace dgsl
