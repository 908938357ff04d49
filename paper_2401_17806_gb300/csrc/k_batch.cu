// Batched persistent solver engine: the host side (workspace layout, state
// area, launch) and the kernels for launches of plain CG slots.  The device
// code is in kbatch_impl.cuh.
#include "kbatch_impl.cuh"

namespace dgsl {

// ---------------------------------------------------------------- host side

int engine_chunk_tris(int p, int ne) {
  (void)ne;
  return e_tt(e_nphi(p)) * 8;  // 8 tiles per chunk
}

size_t engine_state_bytes() {
  return sizeof(BSlotDesc) * kMaxSlots + sizeof(BState) * kMaxSlots + 256 + sizeof(int) * (2 * kMaxSlots + 1) +
         sizeof(int) * kMaxCtas + 2048;
}

void engine_layout(void* base, EngineParams& P) {
  char* p = static_cast<char*>(base);
  auto take = [&p](size_t bytes) {
    char* q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  P.slots = reinterpret_cast<BSlotDesc*>(take(sizeof(BSlotDesc) * kMaxSlots));
  P.state = reinterpret_cast<BState*>(take(sizeof(BState) * kMaxSlots));
  P.sh = reinterpret_cast<EngineShared*>(take(sizeof(EngineShared)));
  P.act_slot = reinterpret_cast<int*>(take(sizeof(int) * kMaxSlots));
  P.act_chunk0 = reinterpret_cast<int*>(take(sizeof(int) * (kMaxSlots + 1)));
  P.cta_k = reinterpret_cast<int*>(take(sizeof(int) * kMaxCtas));
}

size_t engine_shared_bytes() { return sizeof(EngineShared); }

int engine_shared_status(const void* sh_host_copy) {
  return static_cast<const EngineShared*>(sh_host_copy)->status;
}
int engine_shared_admitted(const void* sh_host_copy) {
  return static_cast<const EngineShared*>(sh_host_copy)->admitted;
}

size_t engine_workspace_bytes(int p, int ne, int nrhs, int precond) {
  const int nphi = e_nphi(p);
  const int64_t n = (int64_t)ne * nphi;
  const int bl = e_block_len(nphi, e_rp(nrhs));
  const int nchunk = (ne + engine_chunk_tris(p, ne) - 1) / engine_chunk_tris(p, ne);
  auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };
  return a256(8 * (size_t)n * nrhs) + a256(4 * (precond ? 9 : 8) * (size_t)ne * bl) +
         a256(8 * (size_t)e_part_stride(precond) * nchunk);
}

void engine_fill_workspace(BSlotDesc& s, char* ws) {
  const int nphi = e_nphi(s.p);
  auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };
  s.rp = e_rp(s.nrhs);
  s.bl = e_block_len(nphi, s.rp);
  s.chunk_tris = engine_chunk_tris(s.p, s.ne);
  s.nchunk = (s.ne + s.chunk_tris - 1) / s.chunk_tris;
  s.r64 = reinterpret_cast<double*>(ws);
  ws += a256(8 * (size_t)s.n * s.nrhs);
  s.fvec = reinterpret_cast<float*>(ws);
  ws += a256(4 * (s.precond ? 9 : 8) * (size_t)s.ne * s.bl);
  s.part = reinterpret_cast<double*>(ws);
}

cudaError_t launch_engine(const EngineParams& e, int bf16, int precond, cudaStream_t s, int* grid_used) {
  if (precond) return launch_engine_precond(e, bf16, s, grid_used);
  return bf16 ? launch_engine_t<uint16_t, false>(e, s, grid_used) : launch_engine_t<float, false>(e, s, grid_used);
}

}  // namespace dgsl
