// gp_mixed.cuh -- entry points of the split-precision (GP_MIXED) path.
#pragma once

#include "gp_internal.cuh"

struct gp_ctx;

namespace gp {

// -2logL over T candidates with the split-precision factorisation.
int mixed_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                    const double* theta, double p, double delta, double* nll, double* mu_hat,
                    double* sigma2_hat, double* logdet, int* status);

// Assemble and factor one instance (b.count == 1) with the split-precision
// path and leave [a | b] = L^-1 [1 | Y] (refined) in Z, ready for finalize.
int mixed_fit_factor(gp_ctx* ctx, const Batch& b, double* Z, size_t zs);

}  // namespace gp
