// k_mixed.cu -- split-precision (GP_MIXED) factorisation path.
#include "gp_mixed.cuh"

namespace gp {

int mixed_nll_batch(gp_ctx*, int, int, const double*, const double*, int, const double*, double,
                    double, double*, double*, double*, double*, int*) {
    return GP_ENOTSUP;
}

int mixed_fit_factor(gp_ctx*, const Batch&, double*, size_t) { return GP_ENOTSUP; }

}  // namespace gp
