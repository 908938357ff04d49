// Batched persistent solver engine: the kernels of launches that also run
// block-Jacobi preconditioned slots (both CG forms in one kernel), compiled
// apart from the plain ones so that the two build in parallel.
#include "kbatch_impl.cuh"

namespace dgsl {

cudaError_t launch_engine_precond(const EngineParams& e, int bf16, cudaStream_t s, int* grid_used) {
  return bf16 ? launch_engine_t<uint16_t, true>(e, s, grid_used) : launch_engine_t<float, true>(e, s, grid_used);
}

}  // namespace dgsl
