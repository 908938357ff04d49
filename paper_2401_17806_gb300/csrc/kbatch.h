// Host/device interface of the batched persistent solver engine (k_batch.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dgsl {

constexpr int kMaxSlots = 4096;       // slots per engine (admitted over its lifetime)
constexpr int kMaxRhs = 8;            // right-hand sides per slot
constexpr int kMaxCtas = 2048;        // CTAs of an engine launch (152 SMs x at most 8)
constexpr int kEngineSums = 6 * kMaxRhs;  // partial sums per chunk (up to 6 per right-hand side)

// One request (1..kMaxRhs right-hand sides of one operator), written by the
// host and copied into device memory when the engine admits it.  All pointers
// are device pointers (the inbox itself is mapped host memory).  b, x and r64
// are [nrhs][n] doubles in the operator's order; fvec holds 8 FP32 vectors
// d | p | r0 | r1 | w0 | w1 | s0 | s1 of ne blocks of bl floats (per triangle
// N_phi x rp values, right-hand side innermost), 9 with the block-Jacobi
// preconditioner (u last); part holds kEngineSums doubles per chunk.
struct BSlotDesc {
  int p, ne, ne_pad, mean_zero;
  long long n;
  int nrhs, rp, bl, precond;  // precond: block-Jacobi preconditioned inner CG
  const double* K64;        // FP64 couplings (refinement residual)
  const void* Kin;          // inner couplings, float or bf16 bits (engine type); with
                            // precond those of A P (coefK and the mass term folded in)
  const float* Pin;         // precond: P, FP32, layout of launch_build_precond
  const int32_t* cols;
  const double* area;
  const double* Mref;
  double coefK, coefM;
  const double* b;
  double* x;
  double* r64;
  float* fvec;
  double* part;
  double tol, inner_tol;
  int max_iters, max_refine;
  int nchunk, chunk_tris;
  long long ticket;
};
static_assert(sizeof(BSlotDesc) % 8 == 0, "descriptor is copied in 8-byte words");

// Completion record of a slot (mapped host memory, written once by the engine);
// over the slot's right-hand sides: the first non-OK status, the largest
// iteration and refinement counts and the largest relative residual.
struct BCompletion {
  int done;                 // 0 while pending; 1 when the fields below are final
  int status;               // DGSL_OK / DGSL_ENOTCONV / DGSL_ETIMEOUT
  int iters;
  int refinements;
  double relres;
  long long ticket;
};

// Mapped host inbox: the host writes slots[count .. ] then publishes count
// with a release store; the engine admits them at its next barrier.
struct BInbox {
  int count;
  int stop;                 // host asks a running engine to exit when idle
  int pad[2];
  BSlotDesc slots[kMaxSlots];
};

struct EngineShared;
struct BState;

struct EngineParams {
  BInbox* inbox;            // device view of the mapped inbox
  BCompletion* done;        // device view of the mapped completion records [kMaxSlots]
  BSlotDesc* slots;         // device copies [kMaxSlots]
  BState* state;            // [kMaxSlots]
  EngineShared* sh;
  int* act_slot;            // [kMaxSlots]
  int* act_chunk0;          // [kMaxSlots + 1]
  int* cta_k;               // [kMaxCtas]: index in the active list of each CTA's first chunk
  uint64_t timeout_ns;      // bound of every device wait
  uint64_t idle_ns;         // how long an idle engine waits for new slots before exiting
};

// Triangles per chunk for degree p and ne triangles (a multiple of the CG
// tile, itself a multiple of 4 triangles): 8 tiles.  It depends on the slot
// alone, never on what else is in the engine.  (Fewer tiles per chunk for
// small meshes sped up a batch of 8 small multi-RHS requests by 10% but slowed
// 64 small single-RHS requests by 27%: more chunks, more per-chunk reductions.)
int engine_chunk_tris(int p, int ne);
// Device workspace of one request (r64 | fvec | partials) and the descriptor
// fields that point into it (also sets rp, bl, chunk_tris, nchunk from p, ne,
// n, nrhs and precond).
size_t engine_workspace_bytes(int p, int ne, int nrhs, int precond);
void engine_fill_workspace(BSlotDesc& s, char* ws);
// Device bytes of the engine-owned areas (slot copies, state, shared words,
// lists) and their layout inside one allocation of that size.
size_t engine_state_bytes();
void engine_layout(void* base, EngineParams& P);
// EngineShared (zeroed before every launch) and the fields the host reads back.
size_t engine_shared_bytes();
int engine_shared_status(const void* sh_host_copy);
int engine_shared_admitted(const void* sh_host_copy);
// Launches the engine (cooperative) on `s`; `bf16` selects the inner coupling
// type, `precond` a kernel that also runs block-Jacobi preconditioned slots
// (every slot with precond set needs it).  The caller zeroes EngineShared
// before the launch.
cudaError_t launch_engine(const EngineParams& e, int bf16, int precond, cudaStream_t s, int* grid_used);

}  // namespace dgsl
