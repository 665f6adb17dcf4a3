// corr.cuh -- the correlation families of gp_correlation on the device.
//
// Power-exponential (eq. 2):  rho = exp(-S),  S = sum_k theta_k |dx_k|^p.
// Matern, nu = 1/2, 3/2, 5/2, in the same product form over dimensions: with
// h_k = c theta_k |dx_k| (c = 1, sqrt 3, sqrt 5),
//   rho = exp(-sum_k h_k) prod_k q(h_k),  q(h) = 1, 1 + h, 1 + h + h^2 / 3,
// so one exponential per entry remains and the theta-independent part of each
// term (|dx_k|^p, or |dx_k|) is shared by every candidate, as the assembly
// kernels arrange.  The kernels therefore take theta pre-multiplied by c and
// the powers with p = 1 for the Matern families.
#pragma once

#include "df.cuh"
#include "gp_internal.cuh"

namespace gp {

// c of h = c theta |dx| (1 for the power-exponential family)
__host__ __device__ __forceinline__ double corr_theta_scale(int corr) {
    return corr == GP_CORR_MATERN32 ? 1.7320508075688772935 : (corr == GP_CORR_MATERN52 ? 2.2360679774997896964 : 1.0);
}

__host__ __device__ __forceinline__ bool corr_is_matern(int corr) { return corr != GP_CORR_POWEXP; }

// q(h) in double
__device__ __forceinline__ double matern_q(double h, int corr) {
    if (corr == GP_CORR_MATERN32) return 1.0 + h;
    if (corr == GP_CORR_MATERN52) return 1.0 + h + h * h / 3.0;
    return 1.0;
}

// q(h) in double-float (h >= 0); third = 1/3 as double-float
__device__ __forceinline__ dfl matern_q_df(dfl h, int corr, dfl third) {
    if (corr == GP_CORR_MATERN32) return df_add(dfl{1.f, 0.f}, h);
    if (corr == GP_CORR_MATERN52) return df_add(dfl{1.f, 0.f}, df_fma(df_mul(h, h), third, h));
    return dfl{1.f, 0.f};
}

}  // namespace gp
