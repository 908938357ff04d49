// C-ABI of dgsl: the time steps built from the semi-Lagrangian transport and
// the solves -- the first-order Navier-Stokes step, the SL-IMEX
// advection-diffusion step and the SL-IMEX Navier-Stokes stages (Sec. 3 and
// App. A).  Each composes the kernels of k_apply.cu and k_sl.cu with the CG
// solve driver of api.cu on the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "api_internal.h"
#include "kernels.h"
#include "operator.h"

using namespace dgsl;
using namespace dgsl_api;

extern "C" int dgsl_ns_step(const dgsl_operator* cop, double dt, double nu, const double* vhat_in, double* vhat_out,
                            double* p_out, const dgsl_solve_opts* opts, dgsl_solve_info* info, void* stream) {
  NvtxRange nvtx("dgsl_ns_step");
  DGSL_TRY({
    check_dev(cop);
    if (!vhat_in || !vhat_out) return fail(DGSL_EINVAL, "vhat_in and vhat_out must be non-NULL");
    if (!(dt > 0.0) || !std::isfinite(dt) || !(nu >= 0.0) || !std::isfinite(nu))
      return fail(DGSL_EINVAL, "dt must be finite and > 0, nu finite and >= 0");
    if (!cop->d.G || !cop->d.Minv || !cop->d.Uloc) return fail(DGSL_EINVAL, "the step needs opts.factored");
    dgsl_solve_opts o;
    if (int e = resolve_solve_opts(cop, opts, o)) return e;
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    op->ensure_work();
    op->ensure_sl(2);
    const DevOp& d = op->d;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = d.n;
    const size_t nv = (size_t)d.nd * d.npsi;
    double* w = op->ensure_ns();
    double* vbar = w;               // [2][n] main-grid velocity (eq. d2m)
    double* c = vbar + 2 * n;       // [2][n] transported (Sec. 2.5)
    double* mc = c + 2 * n;         // [2][n] Mbar c
    double* vst = mc + 2 * n;       // [2][n] after the viscous solve (eq. ad5)
    double* vhs = vst + 2 * n;      // [2][nd][npsi] on the dual grid (eq. m2d)
    double* b = vhs + 2 * nv;       // [n] divergence
    // (the d2m right-hand side goes to c first: the inverse mass is not applied in place)
    for (int k = 0; k < 2; ++k) DGSL_CUDA(launch_d2m_rhs(d, vhat_in + k * nv, c + k * n, s));
    DGSL_CUDA(launch_mass_inv(d, c, vbar, 2, s));
    DGSL_CUDA(cudaMemsetAsync(op->sl.err, 0, sizeof(int), s));
    DGSL_CUDA(dgsl::launch_sl_transport(op->sl.g, n, dt, vbar, vbar, 2, c, nullptr, nullptr, nullptr, kSLMaxSteps,
                                        op->sl.vmono, op->sl.cmono, op->sl.err, s));
    DGSL_CUDA(cudaMemcpyAsync(op->sl.h_err, op->sl.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    for (int k = 0; k < 2; ++k) DGSL_CUDA(launch_apply_assembled_f64(d, 0.0, 1.0, c + k * n, mc + k * n, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    if (*op->sl.h_err)
      return fail(DGSL_ENOTCONV, "a trajectory crossed more than " + std::to_string(kSLMaxSteps) + " cells");
    int worst = DGSL_OK;
    dgsl_solve_info inf[3];
    // the viscous solves start from the transported velocity (H = Mbar + nu dt K)
    DGSL_CUDA(cudaMemcpyAsync(vst, c, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    dgsl_solve_opts oh = o;
    oh.use_x0 = 1;
    for (int k = 0; k < 2; ++k) {
      const int st = solve_one(op, DGSL_HELMHOLTZ, nu * dt, mc + k * n, vst + k * n, oh, &inf[k], s);
      if (st != DGSL_OK && worst == DGSL_OK) worst = st;
    }
    for (int k = 0; k < 2; ++k) DGSL_CUDA(launch_m2d(d, vst + k * n, vhs + k * nv, s));
    DGSL_CUDA(launch_div(d, vhs, b, s));
    double* pr = p_out ? p_out : vbar;  // (vbar is free again)
    dgsl_solve_opts osch = o;
    osch.use_x0 = o.use_x0 && p_out ? 1 : 0;  // warm start from the caller's last pressure
    double* p_prev = b + n;
    const bool extrap = o.use_x0 == 2 && p_out;
    if (extrap && op->ns_prev_valid) DGSL_CUDA(launch_extrapolate(p_out, p_prev, p_out, n, s));  // 2 p^n - p^{n-1}
    const int st = solve_one(op, DGSL_SCHUR, dt, b, pr, osch, &inf[2], s);
    if (extrap && !op->ns_prev_valid) {
      DGSL_CUDA(cudaMemcpyAsync(p_prev, p_out, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      op->ns_prev_valid = true;
    }
    if (st != DGSL_OK && worst == DGSL_OK) worst = st;
    DGSL_CUDA(launch_velocity_update(d, dt * dt, vhs, pr, vhat_out, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    if (info)
      for (int k = 0; k < 3; ++k) info[k] = inf[k];
    if (worst != DGSL_OK)
      dgsl_set_last_error(worst == DGSL_ENOTCONV ? "a solve did not converge" : "device wait timed out");
    return worst;
  });
}

extern "C" int dgsl_advdiff_step(const dgsl_operator* cop, int R, double dt, double alpha, const double* vbar,
                      const double* c_in, double* c_out, const dgsl_solve_opts* opts, dgsl_solve_info* info,
                      void* stream) {
  NvtxRange nvtx("dgsl_advdiff_step");
  DGSL_TRY({
    check_dev(cop);
    dgsl::SLTableau tab;
    if (!dgsl::sl_tableau(R, tab)) return fail(DGSL_EINVAL, "R must be 0, 1 or 2");
    if (!vbar || !c_in || !c_out) return fail(DGSL_EINVAL, "vbar, c_in and c_out must be non-NULL");
    if (!(dt > 0.0) || !std::isfinite(dt) || !(alpha >= 0.0) || !std::isfinite(alpha))
      return fail(DGSL_EINVAL, "dt must be finite and > 0, alpha finite and >= 0");
    dgsl_solve_opts o;
    if (int e = resolve_solve_opts(cop, opts, o)) return e;
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    op->ensure_work();
    op->ensure_sl(1 + tab.ns);
    const DevOp& d = op->d;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = d.n;
    const int64_t nt = (int64_t)d.ne * op->sl.g.ng;
    double* V = op->ensure_advdiff();         // [ns][nt][2] stage velocities
    double* F = V + 8 * nt;                   // [1 + ns][n]: C^n, H_0, ..., H_{ns-1}
    double* ci = F + 5 * n;                   // stage value C^I_s
    double* rhs = ci + n;                     // Mbar C^I_s
    double* cst = rhs + n;                    // C*_s
    DGSL_CUDA(cudaMemcpyAsync(F, c_in, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DGSL_CUDA(cudaMemsetAsync(op->sl.err, 0, sizeof(int), s));
    DGSL_CUDA(dgsl::launch_sl_stage_velocities(op->sl.g, n, dt, tab, vbar, V, op->sl.vmono, kSLMaxSteps, op->sl.err,
                                               s));
    dgsl_solve_opts oh = o;
    oh.use_x0 = 1;  // each diffusion solve starts from its stage value
    int worst = DGSL_OK;
    dgsl_solve_info inf[4];
    // implicit c_s = sum_j a_{s,j}
    double c[4] = {};
    for (int i = 0; i < tab.ns; ++i)
      for (int j = 0; j <= i; ++j) c[i] += tab.ai[i][j];
    for (int st = 0; st < tab.ns; ++st) {
      dgsl::SLStage sg;
      sg.s = st;
      for (int j = 0; j <= st; ++j) {
        sg.a[j] = tab.ai[st][j];
        sg.shift[j] = c[st] - c[j];
      }
      DGSL_CUDA(dgsl::launch_sl_advdiff_stage(op->sl.g, n, n, dt, sg, V, F, op->sl.cmono, ci, kSLMaxSteps,
                                              op->sl.err, s));
      DGSL_CUDA(launch_apply_assembled_f64(d, 0.0, 1.0, ci, rhs, s));
      DGSL_CUDA(cudaMemcpyAsync(cst, ci, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      const double add = tab.ai[st][st] * dt;
      const int r = solve_one(op, DGSL_HELMHOLTZ, add * alpha, rhs, cst, oh, &inf[st], s);
      if (r != DGSL_OK && worst == DGSL_OK) worst = r;
      if (st + 1 < tab.ns) DGSL_CUDA(dgsl::launch_sl_flux(cst, ci, 1.0 / add, F + (int64_t)(1 + st) * n, n, s));
    }
    DGSL_CUDA(cudaMemcpyAsync(c_out, cst, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DGSL_CUDA(cudaMemcpyAsync(op->sl.h_err, op->sl.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    if (*op->sl.h_err)
      return fail(DGSL_ENOTCONV, "a segment crossed more than " + std::to_string(kSLMaxSteps) + " cells");
    if (info)
      for (int k = 0; k < tab.ns; ++k) info[k] = inf[k];
    if (worst != DGSL_OK)
      dgsl_set_last_error(worst == DGSL_ENOTCONV ? "a solve did not converge" : "device wait timed out");
    return worst;
  });
}

extern "C" int dgsl_ns_imex_step(const dgsl_operator* cop, int R, double dt, double nu, const double* vhat_in,
                                 double* vhat_out, double* p_out, const dgsl_solve_opts* opts, dgsl_solve_info* info,
                                 void* stream) {
  NvtxRange nvtx("dgsl_ns_imex_step");
  DGSL_TRY({
    check_dev(cop);
    dgsl::SLTableau tab;
    if (!dgsl::sl_tableau(R, tab)) return fail(DGSL_EINVAL, "R must be 0, 1 or 2");
    if (!vhat_in || !vhat_out) return fail(DGSL_EINVAL, "vhat_in and vhat_out must be non-NULL");
    if (!(dt > 0.0) || !std::isfinite(dt) || !(nu >= 0.0) || !std::isfinite(nu))
      return fail(DGSL_EINVAL, "dt must be finite and > 0, nu finite and >= 0");
    if (!cop->d.G || !cop->d.Minv || !cop->d.Uloc) return fail(DGSL_EINVAL, "the step needs opts.factored");
    dgsl_solve_opts o;
    if (int e = resolve_solve_opts(cop, opts, o)) return e;
    dgsl_operator* op = const_cast<dgsl_operator*>(cop);
    std::lock_guard<std::mutex> lock(op->mu);
    DGSL_CUDA(cudaSetDevice(op->d.device));
    op->ensure_work();
    op->ensure_sl(5);
    const DevOp& d = op->d;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = d.n;
    const int64_t nv = (int64_t)d.nd * d.npsi;
    const int64_t nt = (int64_t)d.ne * op->sl.g.ng;
    double* V = op->ensure_nsimex();  // [ns][nt][2] stage velocities
    double* F = V + 8 * nt;           // [1 + ns][2][n]: vbar^n, Hbar_0, ..., Hbar_{ns-1}
    double* vI = F + 10 * n;          // [2][n] stage value (also the explicit stage field)
    double* vst = vI + 2 * n;         // [2][n] after the viscous solve
    double* rhs = vst + 2 * n;        // [2][n]
    double* b = rhs + 2 * n;          // [n] divergence
    double* prs = b + n;              // [n] pressure scratch
    double* tmp = prs + n;            // [n]
    double* vhs = tmp + n;            // [2][nv] vhat*
    double* vIh = vhs + 2 * nv;       // [2][nv] L_md(vI), then the stage flux Hhat
    double* vs = vIh + 2 * nv;        // [2][nv] stage velocity vhat_s
    double* pr = p_out ? p_out : prs;
    DGSL_CUDA(cudaMemsetAsync(V, 0, (size_t)8 * nt * sizeof(double), s));
    DGSL_CUDA(cudaMemsetAsync(op->sl.err, 0, sizeof(int), s));
    // vbar^n = L_dm(vhat^n) (eq. d2m)
    for (int k = 0; k < 2; ++k) {
      DGSL_CUDA(launch_d2m_rhs(d, vhat_in + k * nv, tmp, s));
      DGSL_CUDA(launch_mass_inv(d, tmp, F + k * n, 1, s));
    }
    double c[4] = {};
    double ct[4] = {};
    for (int i = 0; i < tab.ns; ++i)
      for (int j = 0; j < 4; ++j) {
        c[i] += tab.ai[i][j];
        ct[i] += tab.at[i][j];
      }
    dgsl_solve_opts oh = o;
    oh.use_x0 = 1;
    dgsl_solve_opts osch = o;
    osch.use_x0 = o.use_x0 && p_out ? 1 : 0;
    int worst = DGSL_OK;
    dgsl_solve_info inf[12];
    for (int st = 0; st < tab.ns; ++st) {
      // the stage velocity of every trajectory
      dgsl::SLStage se;
      se.s = st;
      for (int j = 0; j < st; ++j) {
        se.a[j] = tab.at[st][j];
        se.shift[j] = ct[st] - c[j];
      }
      const double* field = F;  // vbar^n for the first stage
      if (st > 0) {
        for (int k = 0; k < 2; ++k)
          DGSL_CUDA(dgsl::launch_sl_advdiff_stage(op->sl.g, n, 2 * n, dt, se, V, F + k * n, op->sl.cmono, vI + k * n,
                                                  kSLMaxSteps, op->sl.err, s));
        field = vI;
      }
      // (the two components are n apart in both F and vI)
      DGSL_CUDA(dgsl::launch_sl_stage_velocity(op->sl.g, n, dt, se, field, V, op->sl.vmono, kSLMaxSteps, op->sl.err,
                                               s));
      // the implicit stage value
      dgsl::SLStage si;
      si.s = st;
      for (int j = 0; j <= st; ++j) {
        si.a[j] = tab.ai[st][j];
        si.shift[j] = c[st] - c[j];
      }
      for (int k = 0; k < 2; ++k)
        DGSL_CUDA(dgsl::launch_sl_advdiff_stage(op->sl.g, n, 2 * n, dt, si, V, F + k * n, op->sl.cmono, vI + k * n,
                                                kSLMaxSteps, op->sl.err, s));
      const double h = tab.ai[st][st] * dt;
      // viscous solves (eq. ad5), back to the dual grid (eq. m2d), pressure (eq. pressure_final), update (eq. nc.2)
      for (int k = 0; k < 2; ++k) {
        DGSL_CUDA(launch_apply_assembled_f64(d, 0.0, 1.0, vI + k * n, rhs + k * n, s));
        DGSL_CUDA(cudaMemcpyAsync(vst + k * n, vI + k * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        const int r = solve_one(op, DGSL_HELMHOLTZ, nu * h, rhs + k * n, vst + k * n, oh, &inf[3 * st + k], s);
        if (r != DGSL_OK && worst == DGSL_OK) worst = r;
        DGSL_CUDA(launch_m2d(d, vst + k * n, vhs + k * nv, s));
      }
      DGSL_CUDA(launch_div(d, vhs, b, s));
      const int r = solve_one(op, DGSL_SCHUR, h, b, pr, osch, &inf[3 * st + 2], s);
      if (r != DGSL_OK && worst == DGSL_OK) worst = r;
      osch.use_x0 = 1;  // later stages start from the last stage's pressure
      DGSL_CUDA(launch_velocity_update(d, h * h, vhs, pr, vs, s));
      if (st + 1 < tab.ns) {
        // the stage flux Hhat_s = (vhat_s - L_md(vI)) / h and its main-grid copy Hbar_s = L_dm(Hhat_s)
        for (int k = 0; k < 2; ++k) DGSL_CUDA(launch_m2d(d, vI + k * n, vIh + k * nv, s));
        DGSL_CUDA(dgsl::launch_sl_flux(vs, vIh, 1.0 / h, vIh, 2 * nv, s));
        for (int k = 0; k < 2; ++k) {
          DGSL_CUDA(launch_d2m_rhs(d, vIh + k * nv, tmp, s));
          DGSL_CUDA(launch_mass_inv(d, tmp, F + (int64_t)(1 + st) * 2 * n + k * n, 1, s));
        }
      }
    }
    DGSL_CUDA(cudaMemcpyAsync(vhat_out, vs, 2 * (size_t)nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DGSL_CUDA(cudaMemcpyAsync(op->sl.h_err, op->sl.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DGSL_CUDA(cudaStreamSynchronize(s));
    if (*op->sl.h_err)
      return fail(DGSL_ENOTCONV, "a segment crossed more than " + std::to_string(kSLMaxSteps) + " cells");
    if (info)
      for (int k = 0; k < 3 * tab.ns; ++k) info[k] = inf[k];
    if (worst != DGSL_OK)
      dgsl_set_last_error(worst == DGSL_ENOTCONV ? "a solve did not converge" : "device wait timed out");
    return worst;
  });
}
