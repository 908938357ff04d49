// Helpers shared by the C-ABI translation units (api.cu, steps.cu).
#pragma once

#include <cuda_runtime.h>

#include <exception>
#include <string>

#include "operator.h"

namespace dgsl_api {

// Sets the thread-local message of dgsl_last_error() and returns code.
int fail(int code, const std::string& msg);
// The operator, or throws (NULL: DGSL_EINVAL; host-only: DGSL_ENODEVICE).
const dgsl_operator* check_dev(const dgsl_operator* op);
// Solve options with the defaults filled in for NULL, checked, and checked
// against the couplings the operator stores.  Returns DGSL_OK or the error.
int resolve_solve_opts(const dgsl_operator* op, const dgsl_solve_opts* opts, dgsl_solve_opts& o);
// One FP64-refined CG solve of kind DGSL_SCHUR (coef = dt) or DGSL_HELMHOLTZ
// (coef = nu dt) on stream s; the caller holds op->mu and has called
// op->ensure_work().  Returns the solve's status and fills *info.
int solve_one(dgsl_operator* op, int kind, double coef, const double* b, double* x, const dgsl_solve_opts& o,
              dgsl_solve_info* info, cudaStream_t s);
// Cells one semi-Lagrangian trajectory (or segment) may cross before the walk
// gives up and the call returns DGSL_ENOTCONV.
constexpr int kSLMaxSteps = 1 << 16;

}  // namespace dgsl_api

// Runs body; a dgsl::Error or std::exception becomes a status code and the
// message of dgsl_last_error().
#define DGSL_TRY(body)                              \
  try {                                             \
    body;                                           \
  } catch (const dgsl::Error& e) {                  \
    return dgsl_api::fail(e.code, e.what());        \
  } catch (const std::exception& e) {               \
    return dgsl_api::fail(DGSL_EINVAL, e.what());   \
  }
