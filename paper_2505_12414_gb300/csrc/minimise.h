// minimise.h -- host quasi-Newton minimiser used by fit_minimise / fit_minimise_fcn.
#pragma once

#include <functional>

#include "../../include/gbnll.h"

namespace gbnll {

// Objective: fills f and g (full external parameter vector) at theta; returns an
// nll_status (NLL_OK on success; any other value rejects the point).
using Objective = std::function<int(const double* theta, double* f, double* g)>;

// Analytic second derivatives at theta (full external parameter vector) from one pass: the
// objective f, its gradient g (n), H (n x n, row-major) and, when W is not null, the
// squared-weight score matrix; returns an nll_status.
using HessianFn = std::function<int(const double* theta, double* f, double* g, double* H, double* W)>;

// strategy 2 and 4 and hessian 2/3 of fit_options need `hess`; without it they are rejected.
// strategy 4 minimises by damped Newton steps with the analytic Hessian at every iterate.
int bfgs_minimise(const Objective& fn, int n, const double* theta0, const double* lo, const double* hi,
                  const double* step, const int* fixed, const fit_options* opt, fit_result* out,
                  const HessianFn* hess = nullptr);

// Dense symmetric positive-definite inverse by Cholesky; false if not positive definite.
bool spd_inverse(int n, const double* a, double* inv);

}  // namespace gbnll
