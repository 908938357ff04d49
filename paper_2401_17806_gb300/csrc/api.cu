// C-ABI of dgsl: operator build and upload, applies, and the CG solve driver
// (FP64 iterative refinement around the persistent CG kernels).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"
#include "host.h"
#include "kernels.h"
#include "operator.h"

using namespace dgsl;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace dgsl_api {
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

const dgsl_operator* check_dev(const dgsl_operator* op) {
  if (!op) throw Error(DGSL_EINVAL, "operator is NULL");
  if (op->host_only) throw Error(DGSL_ENODEVICE, "operator was built host-only");
  return op;
}
}  // namespace dgsl_api

using namespace dgsl_api;

void dgsl_set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {

uint16_t f32_to_bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;  // round to nearest even
  return (uint16_t)(u >> 16);
}
}  // namespace

namespace {

// Couplings in the interleaved row layout.  Every row of K sums to zero
// (K 1 = 0: the nodal basis is a partition of unity and G 1 = 0 on the
// torus), so (K x)_row = sum_{c != row} a_c (x_c - x_row): the kernels form
// a_c (x_c - x_row), and diff stores the self-coupling slot as 0 (the FP32 and
// BF16 copies; the FP64 copy keeps it, where it multiplies x_row - x_row).
// Rounded couplings then still annihilate constants, and the relative error of
// the smooth (small-eigenvalue) components stays at the rounding level instead
// of growing with the condition number.
template <class T>
std::vector<T> to_ell(const HostBlocks& hb, int64_t n, T (*cvt)(double), bool diff) {
  const int N = hb.nphi, NC = 4 * N;
  const int VEC = 16 / (int)sizeof(T);
  const int NG = (NC + VEC - 1) / VEC;
  std::vector<T> out((size_t)NG * n * VEC, cvt(0.0));
  for (int i = 0; i < hb.ne; ++i)
    for (int k = 0; k < N; ++k) {
      const int64_t row = (int64_t)i * N + k;
      for (int c = 0; c < NC; ++c) {
        const int b = c / N, kk = c % N;
        double v = b == 0 ? hb.Kd[((size_t)i * N + k) * N + kk] : hb.Ko[(((size_t)i * 3 + (b - 1)) * N + k) * N + kk];
        if (diff && b == 0 && kk == k) v = 0.0;
        out[((size_t)(c / VEC) * n + row) * VEC + c % VEC] = cvt(v);
      }
    }
  return out;
}
double cvt_d(double v) { return v; }
float cvt_f(double v) { return (float)v; }
uint16_t cvt_b(double v) { return f32_to_bf16_bits((float)v); }

}  // namespace

extern "C" {

const char* dgsl_last_error(void) { return g_last_error.c_str(); }
const char* dgsl_version(void) { return "dgsl 0.1 (sm_103a)"; }
uint64_t dgsl_launch_count(void) { return launch_count(); }

void dgsl_default_solve_opts(dgsl_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-10;
  o->max_iters = 200000;
  o->precision = DGSL_PREC_F64;
  o->use_x0 = 0;
  o->inner_tol = 1e-3;
  o->max_refine = 30;
  o->form = DGSL_FORM_ASSEMBLED;
  o->precond = DGSL_PRECOND_NONE;
  o->pad = 0;
}

int dgsl_build_operators(const dgsl_mesh* mesh, int p, const dgsl_build_opts* opts, dgsl_operator** out) {
  NvtxRange nvtx("dgsl_build_operators");
  if (!mesh || !out) return fail(DGSL_EINVAL, "mesh and out must be non-NULL");
  *out = nullptr;
  dgsl_build_opts o{0, 0, 0, 0, nullptr};
  if (opts) o = *opts;
  if (o.store == 0) o.store = DGSL_STORE_F64 | DGSL_STORE_F32;
  try {
    auto op = std::make_unique<dgsl_operator>();
    op->host_only = o.host_only;
    op->ro = build_reference_operators(p);
    op->hm = build_mesh(*mesh);
    HostBlocks hb = build_blocks(op->hm, op->ro);
    DevOp& d = op->d;
    d.p = p;
    d.nphi = op->ro.nphi;
    d.npsi = op->ro.npsi;
    d.ne = op->hm.ne;
    d.nd = op->hm.nd;
    d.ncol = op->hm.n_colours();
    d.n = (int64_t)d.ne * d.nphi;
    d.device = o.device;
    if (d.ncol > 8) throw Error(DGSL_EMESH, "edge colouring needs more than 8 colours");
    for (int c = 0; c <= d.ncol; ++c) d.colour_offsets[c] = op->hm.colour_offsets[c];
    if (!o.host_only) {
      DGSL_CUDA(cudaSetDevice(o.device));
      op->upload_stream = (cudaStream_t)o.stream;
      upload_dual_tables(o.device);
      // column rows padded to a multiple of 4 triangles: every 4-triangle group of
      // a row starts on a 16-byte boundary (bulk copies of tile indices)
      d.ne_pad = (d.ne + 3) / 4 * 4;
      std::vector<int32_t> cols((size_t)4 * d.ne_pad, 0);
      for (int i = 0; i < d.ne; ++i) {
        cols[i] = i;
        for (int b = 1; b < 4; ++b) cols[(size_t)b * d.ne_pad + i] = hb.nbr[(size_t)i * 3 + b - 1];
      }
      d.cols = op->upload(cols);
      {
        // two trailing zeros: the engine copies a tile's areas in whole 16-byte units
        std::vector<double> a = hb.area;
        a.resize(a.size() + 2, 0.0);
        d.area = op->upload(a);
      }
      d.Mref = op->upload(op->ro.Mref);
      d.Mrefinv = op->upload(dgsl::mref_inverse(op->ro));
      if (o.store & DGSL_STORE_F64) d.K64 = op->upload(to_ell<double>(hb, d.n, cvt_d, false));
      if (o.store & DGSL_STORE_F32) d.K32 = op->upload(to_ell<float>(hb, d.n, cvt_f, true));
      if (o.store & DGSL_STORE_BF16) d.K16 = op->upload(to_ell<uint16_t>(hb, d.n, cvt_b, true));
      if (o.factored) {
        d.G = op->upload(hb.G);
        d.Minv = op->upload(hb.Minv);
        d.Uloc = op->upload(hb.Uloc);
        d.elr = op->upload(hb.elr);
        std::vector<int32_t> tedge((size_t)3 * d.ne, -1);
        for (int e = 0; e < d.nd; ++e)
          for (int s = 0; s < 2; ++s) tedge[(size_t)hb.elr[2 * e + s] * 3 + hb.eloc[2 * e + s]] = 2 * e + s;
        d.tedge = op->upload(tedge);
      }
      DGSL_CUDA(cudaStreamSynchronize(op->upload_stream));
      op->upload_stream = nullptr;  // later uploads (first-use data) use the legacy default stream
    }
    if (o.host_only || o.factored) {
      op->hb = std::move(hb);
      op->have_blocks = true;
    }
    *out = op.release();
    return DGSL_OK;
  } catch (const Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(DGSL_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(DGSL_EINVAL, e.what());
  }
}

void dgsl_destroy_operator(dgsl_operator* op) { delete op; }

int dgsl_operator_info(const dgsl_operator* op, dgsl_info* out) {
  if (!op || !out) return fail(DGSL_EINVAL, "NULL argument");
  out->p = op->d.p;
  out->n_phi = op->d.nphi;
  out->n_psi = op->d.npsi;
  out->n_tri = op->d.ne;
  out->n_edge = op->d.nd;
  out->n_colours = op->d.ncol;
  out->n_dof = op->d.n;
  out->n_dual = (int64_t)op->d.nd * op->d.npsi;
  out->device_bytes = op->device_bytes;
  out->host_only = op->host_only;
  out->device = op->d.device;
  return DGSL_OK;
}

int dgsl_query_maps(const dgsl_operator* op, dgsl_maps* m) {
  if (!op || !m) return fail(DGSL_EINVAL, "NULL argument");
  const HostMesh& h = op->hm;
  auto cp = [](void* dst, const void* src, size_t bytes) {
    if (dst) std::memcpy(dst, src, bytes);
  };
  cp(m->edge_vtx, h.edge_vtx.data(), h.edge_vtx.size() * 4);
  cp(m->lr, h.lr.data(), h.lr.size() * 4);
  cp(m->loc, h.loc.data(), h.loc.size());
  cp(m->shift, h.shift.data(), h.shift.size());
  cp(m->tri_edge, h.tri_edge.data(), h.tri_edge.size() * 4);
  cp(m->perm, h.perm.data(), h.perm.size() * 4);
  cp(m->edge_perm, h.edge_perm.data(), h.edge_perm.size() * 4);
  cp(m->colour, h.colour.data(), h.colour.size());
  cp(m->colour_offsets, h.colour_offsets.data(), h.colour_offsets.size() * 4);
  return DGSL_OK;
}

int dgsl_query_sl_tables(const dgsl_operator* op, int32_t* nbr, double* trans) {
  if (!op) return fail(DGSL_EINVAL, "NULL argument");
  DGSL_TRY({
    const dgsl::SLHost h = dgsl::build_sl_host(op->hm, op->ro);
    if (nbr) std::memcpy(nbr, h.nbr.data(), h.nbr.size() * sizeof(int32_t));
    if (trans)
      for (int i = 0; i < op->hm.ne; ++i)
        for (int k = 0; k < 6; ++k) trans[(size_t)i * 6 + k] = h.tri[(size_t)i * 16 + 10 + k];
    return DGSL_OK;
  });
}

int dgsl_node_coords(const dgsl_operator* op, int grid, double* xy) {
  if (!op || !xy) return fail(DGSL_EINVAL, "NULL argument");
  if (grid != DGSL_MAIN && grid != DGSL_DUAL) return fail(DGSL_EINVAL, "grid must be DGSL_MAIN or DGSL_DUAL");
  node_coords(op->hm, op->ro, grid, xy);
  return DGSL_OK;
}

int dgsl_query_blocks(const dgsl_operator* op, double* G, double* Minv, double* Mref, double* area) {
  if (!op) return fail(DGSL_EINVAL, "NULL operator");
  if ((G || Minv) && !op->have_blocks) return fail(DGSL_EINVAL, "blocks kept only for host_only or factored builds");
  if (G) std::memcpy(G, op->hb.G.data(), op->hb.G.size() * sizeof(double));
  if (Minv) std::memcpy(Minv, op->hb.Minv.data(), op->hb.Minv.size() * sizeof(double));
  if (Mref) std::memcpy(Mref, op->ro.Mref.data(), op->ro.Mref.size() * sizeof(double));
  if (area) {
    for (int i = 0; i < op->hm.ne; ++i) {
      const double* P = &op->hm.txy[(size_t)op->hm.perm[i] * 6];
      area[i] = (P[2] - P[0]) * (P[5] - P[1]) - (P[3] - P[1]) * (P[4] - P[0]);
    }
  }
  return DGSL_OK;
}

int dgsl_query_couplings(const dgsl_operator* op, double* Kd, double* Ko, int32_t* nbr) {
  if (!op) return fail(DGSL_EINVAL, "NULL operator");
  if (!op->have_blocks) return fail(DGSL_EINVAL, "couplings kept only for host_only or factored builds");
  if (Kd) std::memcpy(Kd, op->hb.Kd.data(), op->hb.Kd.size() * sizeof(double));
  if (Ko) std::memcpy(Ko, op->hb.Ko.data(), op->hb.Ko.size() * sizeof(double));
  if (nbr) std::memcpy(nbr, op->hb.nbr.data(), op->hb.nbr.size() * sizeof(int32_t));
  return DGSL_OK;
}

static int check_vec_args(const void* a, const void* b, int n_rhs) {
  if (!a || !b) return fail(DGSL_EINVAL, "vector pointers must be non-NULL");
  if (n_rhs < 1) return fail(DGSL_EINVAL, "n_rhs must be >= 1");
  return DGSL_OK;
}

int dgsl_apply_schur(const dgsl_operator* op, int form, double dt, const double* x, double* y, int n_rhs,
                     void* stream) {
  DGSL_TRY({
    check_dev(op);
    if (int e = check_vec_args(x, y, n_rhs)) return e;
    if (form != DGSL_FORM_ASSEMBLED && form != DGSL_FORM_FACTORED) return fail(DGSL_EINVAL, "unknown form");
    if (form == DGSL_FORM_FACTORED && !op->d.G) return fail(DGSL_EINVAL, "factored form needs opts.factored");
    if (form == DGSL_FORM_ASSEMBLED && !op->d.K64) return fail(DGSL_EINVAL, "FP64 couplings not stored");
    DGSL_CUDA(cudaSetDevice(op->d.device));
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < n_rhs; ++k) {
      const double* xk = x + (size_t)k * op->d.n;
      double* yk = y + (size_t)k * op->d.n;
      if (form == DGSL_FORM_ASSEMBLED) DGSL_CUDA(launch_apply_assembled_f64(op->d, dt * dt, 0.0, xk, yk, s));
      else DGSL_CUDA(launch_apply_factored_f64(op->d, dt * dt, 0.0, xk, yk, s));
    }
    return DGSL_OK;
  });
}

int dgsl_apply_schur_f32(const dgsl_operator* op, float dt, const float* x, float* y, int n_rhs, void* stream) {
  DGSL_TRY({
    check_dev(op);
    if (int e = check_vec_args(x, y, n_rhs)) return e;
    if (!op->d.K32) return fail(DGSL_EINVAL, "FP32 couplings not stored");
    DGSL_CUDA(cudaSetDevice(op->d.device));
    for (int k = 0; k < n_rhs; ++k)
      DGSL_CUDA(launch_apply_assembled_f32(op->d, dt * dt, x + (size_t)k * op->d.n, y + (size_t)k * op->d.n,
                                           (cudaStream_t)stream));
    return DGSL_OK;
  });
}

int dgsl_apply_helmholtz(const dgsl_operator* op, double nu_dt, const double* x, double* y, int n_rhs,
                         void* stream) {
  DGSL_TRY({
    check_dev(op);
    if (int e = check_vec_args(x, y, n_rhs)) return e;
    if (!op->d.K64) return fail(DGSL_EINVAL, "FP64 couplings not stored");
    DGSL_CUDA(cudaSetDevice(op->d.device));
    for (int k = 0; k < n_rhs; ++k)
      DGSL_CUDA(launch_apply_assembled_f64(op->d, nu_dt, 1.0, x + (size_t)k * op->d.n, y + (size_t)k * op->d.n,
                                           (cudaStream_t)stream));
    return DGSL_OK;
  });
}

int dgsl_project_d2m_rhs(const dgsl_operator* op, const double* vhat, double* b, int n_rhs, void* stream) {
  DGSL_TRY({
    check_dev(op);
    if (int e = check_vec_args(vhat, b, n_rhs)) return e;
    if (!op->d.Uloc) return fail(DGSL_EINVAL, "projections need opts.factored");
    DGSL_CUDA(cudaSetDevice(op->d.device));
    const size_t nv = (size_t)op->d.nd * op->d.npsi;
    for (int k = 0; k < n_rhs; ++k)
      DGSL_CUDA(launch_d2m_rhs(op->d, vhat + k * nv, b + (size_t)k * op->d.n, (cudaStream_t)stream));
    return DGSL_OK;
  });
}

int dgsl_project_m2d(const dgsl_operator* op, const double* vbar, double* vhat, int n_rhs, void* stream) {
  DGSL_TRY({
    check_dev(op);
    if (int e = check_vec_args(vbar, vhat, n_rhs)) return e;
    if (!op->d.Uloc) return fail(DGSL_EINVAL, "projections need opts.factored");
    DGSL_CUDA(cudaSetDevice(op->d.device));
    const size_t nv = (size_t)op->d.nd * op->d.npsi;
    for (int k = 0; k < n_rhs; ++k)
      DGSL_CUDA(launch_m2d(op->d, vbar + (size_t)k * op->d.n, vhat + k * nv, (cudaStream_t)stream));
    return DGSL_OK;
  });
}

int dgsl_apply_div(const dgsl_operator* op, const double* vhat, double* y, int n_rhs, void* stream) {
  DGSL_TRY({
    check_dev(op);
    if (int e = check_vec_args(vhat, y, n_rhs)) return e;
    if (!op->d.G) return fail(DGSL_EINVAL, "divergence needs opts.factored");
    DGSL_CUDA(cudaSetDevice(op->d.device));
    const size_t nv = (size_t)2 * op->d.nd * op->d.npsi;
    for (int k = 0; k < n_rhs; ++k)
      DGSL_CUDA(launch_div(op->d, vhat + k * nv, y + (size_t)k * op->d.n, (cudaStream_t)stream));
    return DGSL_OK;
  });
}

int dgsl_velocity_update(const dgsl_operator* op, double coef, const double* F, const double* p, double* v,
                         int n_rhs, void* stream) {
  DGSL_TRY({
    check_dev(op);
    if (int e = check_vec_args(F, v, n_rhs)) return e;
    if (!p) return fail(DGSL_EINVAL, "p must be non-NULL");
    if (!std::isfinite(coef)) return fail(DGSL_EINVAL, "coef must be finite");
    if (!op->d.G || !op->d.Minv) return fail(DGSL_EINVAL, "the velocity update needs opts.factored");
    DGSL_CUDA(cudaSetDevice(op->d.device));
    const size_t nv = (size_t)2 * op->d.nd * op->d.npsi;
    for (int k = 0; k < n_rhs; ++k)
      DGSL_CUDA(launch_velocity_update(op->d, coef, F + k * nv, p + (size_t)k * op->d.n, v + k * nv,
                                       (cudaStream_t)stream));
    return DGSL_OK;
  });
}

int dgsl_sl_quadrature(int p, double* pts, double* w, int32_t* n_g) {
  if (p < 1 || p > 4) return fail(DGSL_EINVAL, "p must be 1..4");
  std::vector<double> q, qw;
  dgsl::sl_rule(p, q, qw);
  if (n_g) *n_g = (int32_t)qw.size();
  if (pts) std::copy(q.begin(), q.end(), pts);
  if (w) std::copy(qw.begin(), qw.end(), w);
  return DGSL_OK;
}

int dgsl_sl_transport(const dgsl_operator* cop, double dt, const double* vbar, const double* c, double* cstar,
                      int n_fields, double* foot, int32_t* cell, int32_t* steps, void* stream) {
  NvtxRange nvtx("dgsl_sl_transport");
  DGSL_TRY({
    check_dev(cop);
    if (!vbar) return fail(DGSL_EINVAL, "vbar must be non-NULL");
    if (!std::isfinite(dt)) return fail(DGSL_EINVAL, "dt must be finite");
    if (n_fields < 0 || n_fields > dgsl::kSLMaxFields) return fail(DGSL_EINVAL, "n_fields must be 0..8");
    if (n_fields > 0 && (!c || !cstar)) return fail(DGSL_EINVAL, "c and cstar must be non-NULL");
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    op->ensure_sl(n_fields);
    cudaStream_t s = (cudaStream_t)stream;
    DGSL_CUDA(cudaMemsetAsync(op->sl.err, 0, sizeof(int), s));
    DGSL_CUDA(dgsl::launch_sl_transport(op->sl.g, op->d.n, dt, vbar, c, n_fields, cstar, foot, cell, steps,
                                        kSLMaxSteps, op->sl.vmono, op->sl.cmono, op->sl.err, s));
    DGSL_CUDA(cudaMemcpyAsync(op->sl.h_err, op->sl.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    if (*op->sl.h_err)
      return fail(DGSL_ENOTCONV, "a trajectory crossed more than " + std::to_string(kSLMaxSteps) + " cells");
    return DGSL_OK;
  });
}

int dgsl_sl_transport_imex(const dgsl_operator* cop, int R, double dt, const double* vbar, const double* c,
                           double* cstar, int n_fields, double* foot, int32_t* cell, int32_t* steps, void* stream) {
  NvtxRange nvtx("dgsl_sl_transport_imex");
  DGSL_TRY({
    check_dev(cop);
    dgsl::SLTableau tab;
    if (!dgsl::sl_tableau(R, tab)) return fail(DGSL_EINVAL, "R must be 0, 1 or 2");
    if (!vbar) return fail(DGSL_EINVAL, "vbar must be non-NULL");
    if (!std::isfinite(dt)) return fail(DGSL_EINVAL, "dt must be finite");
    if (n_fields < 0 || n_fields > dgsl::kSLMaxFields) return fail(DGSL_EINVAL, "n_fields must be 0..8");
    if (n_fields > 0 && (!c || !cstar)) return fail(DGSL_EINVAL, "c and cstar must be non-NULL");
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    op->ensure_sl(n_fields);
    cudaStream_t s = (cudaStream_t)stream;
    DGSL_CUDA(cudaMemsetAsync(op->sl.err, 0, sizeof(int), s));
    DGSL_CUDA(dgsl::launch_sl_stages(op->sl.g, op->d.n, dt, tab, vbar, c, n_fields, cstar, foot, cell, steps,
                                     kSLMaxSteps, op->sl.vmono, op->sl.cmono, op->sl.err, s));
    DGSL_CUDA(cudaMemcpyAsync(op->sl.h_err, op->sl.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    if (*op->sl.h_err)
      return fail(DGSL_ENOTCONV, "a segment crossed more than " + std::to_string(kSLMaxSteps) + " cells");
    return DGSL_OK;
  });
}

}  // extern "C"

// ------------------------------------------------------------ solve driver
namespace dgsl_api {

struct Sums {
  double s, ss;
};

Sums read_sums(dgsl_operator* op, const double* dev_part, int nparts, cudaStream_t s) {
  DGSL_CUDA(cudaMemcpyAsync(op->w.h_part, dev_part, 2 * (size_t)nparts * sizeof(double), cudaMemcpyDeviceToHost, s));
  DGSL_CUDA(cudaStreamSynchronize(s));
  Sums r{0.0, 0.0};
  for (int j = 0; j < nparts; ++j) {
    r.s += op->w.h_part[2 * j];
    r.ss += op->w.h_part[2 * j + 1];
  }
  return r;
}

// One right-hand side.  Outer loop: r = b - A x in FP64 (assembled FP64
// couplings); inner: CG on A d = r in FP64 (PREC_F64) or on the FP32 / BF16
// couplings with FP32 vectors; x += d in FP64.
// Solve options with the defaults filled in for NULL, checked, and checked
// against the couplings the operator stores.  Returns DGSL_OK or the error.
int resolve_solve_opts(const dgsl_operator* op, const dgsl_solve_opts* opts, dgsl_solve_opts& o) {
  dgsl_default_solve_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol > 0.0) || o.max_iters < 1 || o.max_refine < 1) return fail(DGSL_EINVAL, "bad solve options");
  if (o.precision < DGSL_PREC_F64 || o.precision > DGSL_PREC_BF16_IR) return fail(DGSL_EINVAL, "bad precision");
  if (o.precond != DGSL_PRECOND_NONE && o.precond != DGSL_PRECOND_BLOCK_JACOBI && o.precond != DGSL_PRECOND_MULTIGRID)
    return fail(DGSL_EINVAL, "precond must be DGSL_PRECOND_NONE, DGSL_PRECOND_BLOCK_JACOBI or DGSL_PRECOND_MULTIGRID");
  if (!op->d.K64) return fail(DGSL_EINVAL, "FP64 couplings are needed for the refinement residual");
  if (o.precision == DGSL_PREC_F32_IR && !op->d.K32) return fail(DGSL_EINVAL, "FP32 couplings not stored");
  if (o.precision == DGSL_PREC_BF16_IR && !op->d.K16) return fail(DGSL_EINVAL, "BF16 couplings not stored");
  if (o.precision == DGSL_PREC_BF16_IR && o.precond == DGSL_PRECOND_MULTIGRID && !op->d.K32)
    return fail(DGSL_EINVAL, "the multigrid solve with BF16 couplings also needs the FP32 couplings");
  return DGSL_OK;
}

// Iterations of one multigrid inner solve (a converging one needs tens).
constexpr int kMGInnerCap = 2000;

int solve_one(dgsl_operator* op, int kind, double coef, const double* b, double* x, const dgsl_solve_opts& o,
              dgsl_solve_info* info, cudaStream_t s) {
  NvtxRange nvtx(kind == DGSL_SCHUR ? "dgsl_cg_solve Schur" : "dgsl_cg_solve Helmholtz");
  DevOp& d = op->d;
  auto& w = op->w;
  const int64_t n = d.n;
  const int mean_zero = kind == DGSL_SCHUR ? 1 : 0;
  const double coefK = kind == DGSL_SCHUR ? coef * coef : coef;
  const double coefM = kind == DGSL_SCHUR ? 0.0 : 1.0;
  const uint64_t timeout_ns = 10ull * 1000 * 1000 * 1000;
  int nparts = 0;
  DGSL_CUDA(launch_sum2(b, n, w.part2, w.max_parts, &nparts, s));
  Sums sb = read_sums(op, w.part2, nparts, s);
  const double b_mean = mean_zero ? sb.s / (double)n : 0.0;
  double bnorm2 = mean_zero ? std::max(0.0, sb.ss - (double)n * b_mean * b_mean) : sb.ss;
  if (!o.use_x0) DGSL_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  int iters = 0, refinements = 0, status = DGSL_OK, launches = 0, grid_used = 0;
  double kernel_ms = 0.0;
  double relres = 0.0, best = INFINITY;
  int stall = 0;
  CGWork cw;
  cw.vec = w.vec;
  cw.part = w.part;
  cw.bar = w.bar;
  cw.res = w.res;
  cw.max_parts = w.max_parts;
  const int ptype = o.precision == DGSL_PREC_F64 ? 1 : o.precision == DGSL_PREC_BF16_IR ? 2 : 0;
  auto* held = o.precond == DGSL_PRECOND_BLOCK_JACOBI ? op->acquire_precond(coefK, coefM, ptype, s) : nullptr;
  std::unique_ptr<dgsl_operator::Work::Precond, void (*)(dgsl_operator::Work::Precond*)> hold(
      held, dgsl_operator::release_precond);
  const dgsl::PrecondOp* pre = held ? &held->op : nullptr;
  auto* mgh = o.precond == DGSL_PRECOND_MULTIGRID ? op->acquire_mg(coefK, coefM, ptype, s) : nullptr;
  std::unique_ptr<dgsl_operator::MGEntry, void (*)(dgsl_operator::MGEntry*)> hold_mg(mgh, dgsl_operator::release_mg);
  for (;;) {
    DGSL_CUDA(launch_residual_f64(d, coefK, coefM, mean_zero, b, x, b_mean, w.r64, w.part2, w.max_parts, &nparts, s));
    Sums sr = read_sums(op, w.part2, nparts, s);
    // the exact projection keeps sum(r) at rounding level; the norm uses all of r
    const double rnorm = std::sqrt(sr.ss);
    bnorm2 = bnorm2 > 0.0 ? bnorm2 : 0.0;
    const double bnorm = std::sqrt(bnorm2);
    relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    if (bnorm == 0.0 || relres <= o.tol) break;
    if (iters >= o.max_iters || refinements >= o.max_refine) {
      status = DGSL_ENOTCONV;
      break;
    }
    if (relres < 0.9 * best) {
      best = relres;
      stall = 0;
    } else if (++stall >= 3) {
      status = DGSL_ENOTCONV;
      break;
    }
    const int budget = o.max_iters - iters;
    // aim the inner solve a little below what the outer target still needs
    const double need = 0.5 * o.tol / relres;
    int grid = 0;
    DGSL_CUDA(cudaEventRecord(w.ev0, s));
    if (mgh) {
      // multigrid PCG: FP64 on the FP64 couplings, else FP32 vectors on the
      // FP32 or BF16 couplings of a scaled residual
      // (an inner solve that stalls, e.g. on BF16 couplings, ends after
      // kMGInnerCap iterations and leaves the decision to the refinement rule)
      dgsl::MGResult mr;
      const int mg_budget = std::min(budget, kMGInnerCap);
      if (o.precision == DGSL_PREC_F64) {
        DGSL_CUDA(dgsl::mg_pcg(mgh->sys.get(), d, w.r64, w.d64, std::max(need, 1e-15), mg_budget, s, &mr));
      } else {
        DGSL_CUDA(launch_scale_to_f32(w.r64, 1.0 / rnorm, w.r32, n, s));
        DGSL_CUDA(dgsl::mg_pcg(mgh->sys.get(), d, w.r32, w.d32, std::min(1.0, std::max(o.inner_tol, need)),
                               mg_budget, s, &mr));
      }
      w.h_res->iters = mr.iters;
      w.h_res->status = 0;
      w.h_res->rr0 = mr.rr0;
      w.h_res->rr = mr.rr;
    } else if (o.precision == DGSL_PREC_F64) {
      const double stop_rel = std::max(need, 1e-15);
      DGSL_CUDA(launch_cg_f64(d, coefK, coefM, mean_zero, w.d64, w.r64, pre, stop_rel, budget, cw, timeout_ns, s,
                              &grid));
    } else {
      const int bf16 = o.precision == DGSL_PREC_BF16_IR;
      const double stop_rel = std::min(1.0, std::max(o.inner_tol, need));
      DGSL_CUDA(launch_scale_to_f32(w.r64, 1.0 / rnorm, w.r32, n, s));
      DGSL_CUDA(launch_cg_f32(d, bf16, (float)coefK, (float)coefM, mean_zero, w.d32, w.r32, pre, stop_rel, budget,
                              cw, timeout_ns, s, &grid));
    }
    DGSL_CUDA(cudaEventRecord(w.ev1, s));
    if (!mgh) DGSL_CUDA(cudaMemcpyAsync(w.h_res, w.res, sizeof(CGResult), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    const CGResult cr = *w.h_res;
    {
      float ms = 0.f;
      DGSL_CUDA(cudaEventElapsedTime(&ms, w.ev0, w.ev1));
      kernel_ms += ms;
      ++launches;
      grid_used = grid;
    }
    if (cr.status != 0) {
      status = DGSL_ETIMEOUT;
      break;
    }
    iters += cr.iters;
    ++refinements;
    if (o.precision == DGSL_PREC_F64) {
      DGSL_CUDA(launch_axpy_f64(1.0, w.d64, x, n, s));
    } else {
      DGSL_CUDA(launch_axpy_f32_to_f64(rnorm, w.d32, x, n, s));
    }
    if (cr.iters == 0) {
      status = DGSL_ENOTCONV;
      break;
    }
  }
  if (mean_zero) {
    DGSL_CUDA(launch_sum2(x, n, w.part2, w.max_parts, &nparts, s));
    DGSL_CUDA(launch_sum_to_first(w.part2, nparts, s));
    DGSL_CUDA(launch_remove_mean_f64(x, w.part2, n, s));
  }
  // a solve that stopped short of the tolerance reports the FP64 rounding
  // floor of its residual: the relative residual of the returned x's exact
  // counterpart rounded to FP64 (expected value; see k_residual_floor_f64)
  double floor_rel = 0.0;
  if (status == DGSL_ENOTCONV && bnorm2 > 0.0) {
    DGSL_CUDA(launch_residual_floor_f64(d, coefK, coefM, x, w.part2, w.max_parts, &nparts, s));
    const Sums sf = read_sums(op, w.part2, nparts, s);
    floor_rel = std::sqrt(sf.s / 3.0) * std::ldexp(1.0, -53) / std::sqrt(bnorm2);
  }
  DGSL_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->status = status;
    info->iters = iters;
    info->refinements = refinements;
    info->cg_launches = launches;
    info->relres = relres;
    info->cg_kernel_ms = kernel_ms;
    info->grid = grid_used;
    info->pad = 0;
    info->relres_floor = floor_rel;
  }
  return status;
}

}  // namespace dgsl_api

extern "C" int dgsl_cg_solve(const dgsl_operator* cop, int kind, double coef, const double* b, double* x, int n_rhs,
                             const dgsl_solve_opts* opts, dgsl_solve_info* info, void* stream) {
  DGSL_TRY({
    check_dev(cop);
    if (int e = check_vec_args(b, x, n_rhs)) return e;
    if (kind != DGSL_SCHUR && kind != DGSL_HELMHOLTZ) return fail(DGSL_EINVAL, "kind must be DGSL_SCHUR or DGSL_HELMHOLTZ");
    if (!(coef >= 0.0) || !std::isfinite(coef)) return fail(DGSL_EINVAL, "coef must be finite and >= 0");
    dgsl_solve_opts o;
    if (int e = resolve_solve_opts(cop, opts, o)) return e;
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    op->ensure_work();
    int worst = DGSL_OK;
    for (int k = 0; k < n_rhs; ++k) {
      int st = solve_one(op, kind, coef, b + (size_t)k * op->d.n, x + (size_t)k * op->d.n, o, info ? info + k : nullptr,
                         (cudaStream_t)stream);
      if (st != DGSL_OK && worst == DGSL_OK) worst = st;
    }
    if (worst != DGSL_OK) g_last_error = worst == DGSL_ENOTCONV ? "not converged within max_iters" : "device wait timed out";
    return worst;
  });
}

// ------------------------------------------------------------ multigrid preconditioner
namespace {
int mg_kind_coefs(int kind, double coef, double& coefK, double& coefM) {
  if (kind != DGSL_SCHUR && kind != DGSL_HELMHOLTZ) return fail(DGSL_EINVAL, "kind must be DGSL_SCHUR or DGSL_HELMHOLTZ");
  if (!(coef >= 0.0) || !std::isfinite(coef)) return fail(DGSL_EINVAL, "coef must be finite and >= 0");
  coefK = kind == DGSL_SCHUR ? coef * coef : coef;
  coefM = kind == DGSL_SCHUR ? 0.0 : 1.0;
  if (kind == DGSL_SCHUR && coefK == 0.0) return fail(DGSL_EINVAL, "the Schur operator needs dt > 0");
  return DGSL_OK;
}
using MGHold = std::unique_ptr<dgsl_operator::MGEntry, void (*)(dgsl_operator::MGEntry*)>;
}  // namespace

extern "C" int dgsl_apply_multigrid(const dgsl_operator* cop, int kind, double coef, int precision, const void* r,
                                    void* z, void* stream) {
  DGSL_TRY({
    check_dev(cop);
    if (!r || !z) return fail(DGSL_EINVAL, "r and z must be non-NULL");
    double coefK = 0.0;
    double coefM = 0.0;
    if (int e = mg_kind_coefs(kind, coef, coefK, coefM)) return e;
    if (precision < DGSL_PREC_F64 || precision > DGSL_PREC_BF16_IR) return fail(DGSL_EINVAL, "bad precision");
    const int type = precision == DGSL_PREC_F64 ? 1 : precision == DGSL_PREC_BF16_IR ? 2 : 0;
    if (!cop->d.K64) return fail(DGSL_EINVAL, "the multigrid setup needs the FP64 couplings");
    if ((type == 0 && !cop->d.K32) || (type == 2 && (!cop->d.K16 || !cop->d.K32)))
      return fail(DGSL_EINVAL, "the operator lacks the couplings of this precision");
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    auto* e = op->acquire_mg(coefK, coefM, type, (cudaStream_t)stream);
    MGHold hold(e, dgsl_operator::release_mg);
    DGSL_CUDA(dgsl::mg_apply(e->sys.get(), op->d, r, z, (cudaStream_t)stream));
    return DGSL_OK;
  });
}

extern "C" int dgsl_query_multigrid(const dgsl_operator* cop, int kind, double coef, dgsl_mg_info* info,
                                    int32_t* cvid, int32_t* agg) {
  DGSL_TRY({
    check_dev(cop);
    double coefK = 0.0;
    double coefM = 0.0;
    if (int e = mg_kind_coefs(kind, coef, coefK, coefM)) return e;
    if (!cop->d.K64) return fail(DGSL_EINVAL, "the multigrid setup needs the FP64 couplings");
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    auto* e = op->acquire_mg(coefK, coefM, 1, nullptr);
    MGHold hold(e, dgsl_operator::release_mg);
    const dgsl::MGHost& h = dgsl::mg_sys_host(e->sys.get());
    if ((int)h.lv.size() > 16) return fail(DGSL_EINVAL, "more than 16 levels");
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->n_levels = (int32_t)h.lv.size();
      info->n_vertices = h.nv;
      for (size_t l = 0; l < h.lv.size(); ++l) info->sizes[l] = h.lv[l].A.n;
    }
    if (cvid)
      for (int t = 0; t < op->d.ne; ++t)
        for (int m = 0; m < 3; ++m) cvid[(size_t)op->hm.perm[t] * 3 + m] = h.cvid[(size_t)t * 3 + m];
    if (agg) {
      size_t o = 0;
      for (size_t l = 0; l + 1 < h.lv.size(); ++l)
        for (int32_t a : h.lv[l].agg) agg[o++] = a;
    }
    return DGSL_OK;
  });
}

// ------------------------------------------------------------ Navier-Stokes step
// ------------------------------------------------------------ solve without allocation
//
// dgsl_cg_solve_noalloc: the same refinement + persistent-CG solve as
// dgsl_cg_solve, for callers that must not allocate device memory at solve
// time.  Its scratch (residual, correction, search directions, matvec output,
// per-CTA partial sums, barrier and result words) lives in one file-scope
// device array of fixed size.  The array belongs to this file's device code:
// it is reserved on a device when that code is loaded there (with CUDA's lazy
// module loading, the default, at the first call of this entry point on the
// device) and stays reserved until the process exits.
namespace {

constexpr int64_t kNoAllocMaxDof = int64_t(1) << 18;   // 262,144 DOFs per right-hand side
// Per-CTA partial-sum slots: room for the grids dgsl_cg_solve uses (at most
// 8 CTAs per SM) on a device of up to 256 SMs, so both entry points launch the
// same grids and reduce in the same order.
constexpr int kNoAllocMaxParts = 2048;
constexpr size_t kNoAllocVecBytes = (size_t)kNoAllocMaxDof * sizeof(double);
// CG vectors (cg_vec_bytes: 8 per-triangle padded vectors; at most 32/3 n doubles, for p = 1)
constexpr size_t kNoAllocCgSlots = 11;
// r64 | d64 (also r32 + d32) | CG vectors | part (2 x 4 slots) | part2 (2) | barrier | result
constexpr size_t kNoAllocBytes =
    (2 + kNoAllocCgSlots) * kNoAllocVecBytes + 10 * (size_t)kNoAllocMaxParts * sizeof(double) + 256 + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};

// Device address of the array on `device` (current).  In host code the
// array's name is only a host-side stand-in; the address must come from
// cudaGetSymbolAddress, once per device.
void* noalloc_scratch(int device) {
  if (device < 0 || device >= 64) throw Error(DGSL_EINVAL, "device ordinal out of range");
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) throw Error(DGSL_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = p;
  }
  return g_noalloc_ptr[device];
}

int solve_one_noalloc(const DevOp& d, unsigned char* base, int max_parts, int kind, double coef, const double* b,
                      double* x, const dgsl_solve_opts& o, dgsl_solve_info* info, cudaStream_t s) {
  const int64_t n = d.n;
  double* r64 = reinterpret_cast<double*>(base);
  double* d64 = reinterpret_cast<double*>(base + kNoAllocVecBytes);
  float* r32 = reinterpret_cast<float*>(base + kNoAllocVecBytes);
  float* d32 = r32 + kNoAllocMaxDof;
  void* vbuf = base + 2 * kNoAllocVecBytes;
  double* part = reinterpret_cast<double*>(base + (2 + kNoAllocCgSlots) * kNoAllocVecBytes);
  double* part2 = part + 8 * kNoAllocMaxParts;  // fixed offsets; max_parts <= kNoAllocMaxParts slots used
  unsigned char* tail = reinterpret_cast<unsigned char*>(part2 + 2 * kNoAllocMaxParts);
  GridBarrier* bar = reinterpret_cast<GridBarrier*>(tail);
  CGResult* res = reinterpret_cast<CGResult*>(tail + 256);
  double h_part[2 * kNoAllocMaxParts];
  CGResult h_res;
  auto sums = [&](const double* dev_part, int np) {
    DGSL_CUDA(cudaMemcpyAsync(h_part, dev_part, 2 * (size_t)np * sizeof(double), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    double a = 0.0, q = 0.0;
    for (int j = 0; j < np; ++j) {
      a += h_part[2 * j];
      q += h_part[2 * j + 1];
    }
    return std::make_pair(a, q);
  };
  const int mean_zero = kind == DGSL_SCHUR ? 1 : 0;
  const double coefK = kind == DGSL_SCHUR ? coef * coef : coef;
  const double coefM = kind == DGSL_SCHUR ? 0.0 : 1.0;
  const uint64_t timeout_ns = 10ull * 1000 * 1000 * 1000;
  int np = 0;
  DGSL_CUDA(launch_sum2(b, n, part2, max_parts, &np, s));
  auto sb = sums(part2, np);
  const double b_mean = mean_zero ? sb.first / (double)n : 0.0;
  const double bnorm2 = mean_zero ? std::max(0.0, sb.second - (double)n * b_mean * b_mean) : sb.second;
  const double bnorm = std::sqrt(bnorm2);
  if (!o.use_x0) DGSL_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  int iters = 0, refinements = 0, status = DGSL_OK, launches = 0, grid_used = 0, stall = 0;
  double relres = 0.0, best = INFINITY;
  CGWork cw;
  cw.vec = vbuf;
  cw.part = part;
  cw.bar = bar;
  cw.res = res;
  cw.max_parts = max_parts;
  for (;;) {
    DGSL_CUDA(launch_residual_f64(d, coefK, coefM, mean_zero, b, x, b_mean, r64, part2, max_parts, &np, s));
    const double rnorm = std::sqrt(sums(part2, np).second);
    relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    if (bnorm == 0.0 || relres <= o.tol) break;
    if (iters >= o.max_iters || refinements >= o.max_refine) {
      status = DGSL_ENOTCONV;
      break;
    }
    if (relres < 0.9 * best) {
      best = relres;
      stall = 0;
    } else if (++stall >= 3) {
      status = DGSL_ENOTCONV;
      break;
    }
    const int budget = o.max_iters - iters;
    const double need = 0.5 * o.tol / relres;
    int grid = 0;
    if (o.precision == DGSL_PREC_F64) {
      DGSL_CUDA(launch_cg_f64(d, coefK, coefM, mean_zero, d64, r64, nullptr, std::max(need, 1e-15), budget, cw,
                              timeout_ns, s, &grid));
    } else {
      DGSL_CUDA(launch_scale_to_f32(r64, 1.0 / rnorm, r32, n, s));
      DGSL_CUDA(launch_cg_f32(d, o.precision == DGSL_PREC_BF16_IR, (float)coefK, (float)coefM, mean_zero, d32, r32,
                              nullptr, std::min(1.0, std::max(o.inner_tol, need)), budget, cw, timeout_ns, s, &grid));
    }
    DGSL_CUDA(cudaMemcpyAsync(&h_res, res, sizeof(CGResult), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    ++launches;
    grid_used = grid;
    if (h_res.status != 0) {
      status = DGSL_ETIMEOUT;
      break;
    }
    iters += h_res.iters;
    ++refinements;
    if (o.precision == DGSL_PREC_F64) DGSL_CUDA(launch_axpy_f64(1.0, d64, x, n, s));
    else DGSL_CUDA(launch_axpy_f32_to_f64(rnorm, d32, x, n, s));
    if (h_res.iters == 0) {
      status = DGSL_ENOTCONV;
      break;
    }
  }
  if (mean_zero) {
    DGSL_CUDA(launch_sum2(x, n, part2, max_parts, &np, s));
    DGSL_CUDA(launch_sum_to_first(part2, np, s));
    DGSL_CUDA(launch_remove_mean_f64(x, part2, n, s));
  }
  DGSL_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->status = status;
    info->iters = iters;
    info->refinements = refinements;
    info->cg_launches = launches;
    info->relres = relres;
    info->cg_kernel_ms = 0.0;
    info->grid = grid_used;
    info->pad = 0;
    info->relres_floor = 0.0;
  }
  return status;
}

}  // namespace

extern "C" int dgsl_cg_solve_noalloc(const dgsl_operator* cop, int kind, double coef, const double* b, double* x,
                                     int n_rhs, const dgsl_solve_opts* opts, dgsl_solve_info* info, void* stream) {
  DGSL_TRY({
    check_dev(cop);
    if (int e = check_vec_args(b, x, n_rhs)) return e;
    if (kind != DGSL_SCHUR && kind != DGSL_HELMHOLTZ) return fail(DGSL_EINVAL, "kind must be DGSL_SCHUR or DGSL_HELMHOLTZ");
    if (!(coef >= 0.0) || !std::isfinite(coef)) return fail(DGSL_EINVAL, "coef must be finite and >= 0");
    if (cop->d.n > kNoAllocMaxDof || cg_vec_bytes(cop->d, 0) > kNoAllocCgSlots * kNoAllocVecBytes)
      return fail(DGSL_EINVAL, "dgsl_cg_solve_noalloc: operator has " + std::to_string(cop->d.n) +
                                   " DOFs, above the fixed scratch limit of " + std::to_string(kNoAllocMaxDof));
    dgsl_solve_opts o;
    if (int e = resolve_solve_opts(cop, opts, o)) return e;
    if (o.precond != DGSL_PRECOND_NONE)
      return fail(DGSL_EINVAL, "dgsl_cg_solve_noalloc: no preconditioner (its blocks do not fit the fixed scratch)");
    // The refinement loop reads the residual norm back to the host after every
    // step, which a stream that is being captured cannot do: refuse before
    // anything is enqueued, so the caller's capture stays intact.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      return fail(DGSL_EINVAL,
                  "dgsl_cg_solve_noalloc: the stream is being captured (or the capture state cannot be read); "
                  "this solve synchronises with the host every refinement step and cannot be captured");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    DGSL_CUDA(cudaSetDevice(cop->d.device));
    const int max_parts = cg_max_blocks(cop->d, 0);
    if (max_parts > kNoAllocMaxParts)
      return fail(DGSL_EINVAL, "dgsl_cg_solve_noalloc: the device has more SMs than the fixed scratch serves");
    unsigned char* base = static_cast<unsigned char*>(noalloc_scratch(cop->d.device));
    int worst = DGSL_OK;
    for (int k = 0; k < n_rhs; ++k) {
      int st = solve_one_noalloc(cop->d, base, max_parts, kind, coef, b + (size_t)k * cop->d.n,
                                 x + (size_t)k * cop->d.n, o, info ? info + k : nullptr, (cudaStream_t)stream);
      if (st != DGSL_OK && worst == DGSL_OK) worst = st;
    }
    if (worst != DGSL_OK) g_last_error = worst == DGSL_ENOTCONV ? "not converged within max_iters" : "device wait timed out";
    return worst;
  });
}

// ------------------------------------------------------------ FMA rate probe
extern "C" int dgsl_measure_fma_rate(int device, int fp64, double* flops_per_s) {
  if (!flops_per_s || (fp64 != 0 && fp64 != 1)) return fail(DGSL_EINVAL, "fp64 must be 0 or 1 and the output given");
  try {
    DGSL_CUDA(cudaSetDevice(device));
    int sms = 0;
    DGSL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = sms * 8, iters = fp64 ? 4096 : 65536, reps = 10;
    void* out = nullptr;
    DGSL_CUDA(cudaMalloc(&out, (size_t)blocks * 256 * 8));
    std::unique_ptr<void, void (*)(void*)> guard(out, [](void* q) { cudaFree(q); });
    cudaStream_t st = nullptr;
    DGSL_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    std::unique_ptr<CUstream_st, void (*)(cudaStream_t)> sguard(st, [](cudaStream_t q) { cudaStreamDestroy(q); });
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DGSL_CUDA(cudaEventCreate(&e0));
    std::unique_ptr<CUevent_st, void (*)(cudaEvent_t)> g0(e0, [](cudaEvent_t q) { cudaEventDestroy(q); });
    DGSL_CUDA(cudaEventCreate(&e1));
    std::unique_ptr<CUevent_st, void (*)(cudaEvent_t)> g1(e1, [](cudaEvent_t q) { cudaEventDestroy(q); });
    for (int r = 0; r < 3; ++r) DGSL_CUDA(launch_fma_rate(fp64, out, blocks, iters, st));  // warm-up
    DGSL_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) DGSL_CUDA(launch_fma_rate(fp64, out, blocks, iters, st));
    DGSL_CUDA(cudaEventRecord(e1, st));
    DGSL_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    DGSL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *flops_per_s = 2.0 * (double)blocks * 256.0 * 8.0 * (double)iters * reps / (ms * 1e-3);
    return DGSL_OK;
  } catch (const Error& e) {
    return fail(e.code, e.what());
  }
}

// ------------------------------------------------------------ failure-detection self-test
extern "C" int dgsl_selftest_wait_timeout(int device, int which, double timeout_s, int* status) {
  if (!status || (which != 0 && which != 1) || !(timeout_s > 0.0) || timeout_s > 5.0)
    return fail(DGSL_EINVAL, "which must be 0 or 1 and 0 < timeout_s <= 5");
  try {
    DGSL_CUDA(cudaSetDevice(device));
    GridBarrier* bar = nullptr;
    DGSL_CUDA(cudaMalloc(&bar, sizeof(GridBarrier)));
    std::unique_ptr<GridBarrier, void (*)(GridBarrier*)> guard(bar, [](GridBarrier* b) { cudaFree(b); });
    DGSL_CUDA(launch_selftest_wait(bar, which, (uint64_t)(timeout_s * 1e9), nullptr));
    DGSL_CUDA(cudaDeviceSynchronize());
    GridBarrier h;
    DGSL_CUDA(cudaMemcpy(&h, bar, sizeof(GridBarrier), cudaMemcpyDeviceToHost));
    *status = h.status == kStatusTimeout ? DGSL_ETIMEOUT : DGSL_OK;
    return DGSL_OK;
  } catch (const Error& e) {
    return fail(e.code, e.what());
  }
}
