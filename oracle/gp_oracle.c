/*
 * gp_oracle.c -- CPU FP64 oracle for the Gaussian-process likelihood and
 * kriging path of Franey, Ranjan & Chipman, "A Short Note on Gaussian Process
 * Modeling for Large Datasets using Graphics Processing Units".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA path, and the CUDA
 * path never calls it.
 *
 * Everything is IEEE double, accumulated left to right in the order the
 * definitions are written.  No blocking, no reordering, no BLAS/LAPACK.
 *
 * Matrices are dense row-major n x n: A[i*n + j].
 *
 * Readings of the paper where it is silent (each also listed in the design
 * notes):
 *   - nugget: R_delta = R + delta*I (the diagonal becomes 1 + delta); the
 *     cross-correlation r(x*) used for prediction carries no delta.
 *   - -2 log L is eq. (4) taken literally:  log|R| + n log Q  with
 *     Q = (Y - 1 mu)' R^-1 (Y - 1 mu)  (not divided by n).  The full Gaussian
 *     form log|R| + n log sigma2 + n (1 + log 2 pi) is returned beside it.
 *   - Q == 0 (n = 1, or Y constant) gives -2logL = -inf and status DEGENERATE.
 *   - a Cholesky pivot <= 0 (or not finite) gives status NOTPD and
 *     -2logL = +inf; no pivoting, no jitter.
 *   - the kriging variance is the ordinary-kriging mean squared error
 *     sigma2 [ c0 - r'R^-1 r + (1 - 1'R^-1 r)^2 / (1'R^-1 1) ] with
 *     c0 = 1 + delta (nugget counted in the process variance) or c0 = 1.
 */
#include <float.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

/* The arithmetic type.  The oracle proper is built in IEEE double.  Built
 * with -DGPO_EXTENDED the same definitions run in long double (64-bit
 * significand on x86_64, 113-bit on aarch64): that build exists only to
 * bound the double build's own rounding error on small cases.  The math
 * calls are type-generic (tgmath.h), so each runs in the arithmetic type. */
#ifdef GPO_EXTENDED
typedef long double real;
#define GPO_UNIT_ROUNDOFF (LDBL_EPSILON / 2)
#else
typedef double real;
#define GPO_UNIT_ROUNDOFF (DBL_EPSILON / 2)
#endif
#define GPO_PI ((real)3.141592653589793238462643383279502884L)

#define GPO_OK 0
#define GPO_NOTPD (-3)
#define GPO_DEGENERATE (-6)
#define GPO_ENOMEM (-2)

/* Correlation families (argument fam of every function below).
 *   GPO_POWEXP:   eq. (2) of Section 2, exp(-theta_k |x_ik - x_jk|^p) per
 *                 input dimension.
 *   GPO_MATERN*:  the Matern family Section 2 names as an alternative (it
 *                 cites Stein 1999 and Santner et al. 2003 and gives no
 *                 formula), read in the same product form over dimensions,
 *                 with h = theta_k |x_ik - x_jk| and the closed forms of the
 *                 Matern correlation for half-integer smoothness nu:
 *                   nu = 1/2: exp(-h)
 *                   nu = 3/2: (1 + sqrt(3) h) exp(-sqrt(3) h)
 *                   nu = 5/2: (1 + sqrt(5) h + 5 h^2 / 3) exp(-sqrt(5) h)
 *                 p is not used. */
#define GPO_POWEXP 0
#define GPO_MATERN12 1
#define GPO_MATERN32 2
#define GPO_MATERN52 3

/* One dimension's factor of the correlation. */
static real gpo_corr_1d(real diff, real theta, real p, int fam) {
    real a = fabs(diff);
    if (fam == GPO_MATERN12) return exp(-theta * a);
    if (fam == GPO_MATERN32) {
        real h = sqrt((real)3) * theta * a;
        return (1.0 + h) * exp(-h);
    }
    if (fam == GPO_MATERN52) {
        real h = sqrt((real)5) * theta * a;
        return (1.0 + h + h * h / 3.0) * exp(-h);
    }
    return exp(-theta * pow(a, p));
}

/* Correlation between two points: the product over the d input dimensions
 * (eq. 2 for the power-exponential family). */
static real gpo_corr_pair(int d, const real* xi, const real* xj,
                            const real* theta, real p, int fam) {
    real r = 1.0;
    for (int k = 0; k < d; ++k) r *= gpo_corr_1d(xi[k] - xj[k], theta[k], p, fam);
    return r;
}

/* R(theta), full n x n, plus the nugget delta on the diagonal. */
void gpo_corr_matrix(int n, int d, const real* x, const real* theta,
                     real p, int fam, real delta, real* R) {
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            real v = gpo_corr_pair(d, x + (size_t)i * d, x + (size_t)j * d, theta, p, fam);
            if (i == j) v += delta;
            R[(size_t)i * n + j] = v;
        }
    }
}

/* Cross-correlations r_i(x*) = corr(z(x*), z(x_i)) by eq. (2); no nugget. */
void gpo_cross_corr(int n, int d, const real* x, const real* xs,
                    const real* theta, real p, int fam, real* r) {
    for (int i = 0; i < n; ++i)
        r[i] = gpo_corr_pair(d, xs, x + (size_t)i * d, theta, p, fam);
}

/* Unblocked Cholesky (Cholesky-Banachiewicz, row by row): R = L L'.
 * L is written to the lower triangle of L (upper set to zero).  The paper's
 * CPU path factors R by Cholesky (Section 3).  Returns 0, or (k+1) where k
 * is the first column whose pivot is not positive and finite. */
int gpo_cholesky(int n, const real* R, real* L) {
    memset(L, 0, sizeof(real) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            real s = R[(size_t)i * n + j];
            for (int k = 0; k < j; ++k)
                s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            if (i == j) {
                if (!(s > 0.0) || !isfinite(s)) return i + 1;
                L[(size_t)i * n + i] = sqrt(s);
            } else {
                L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
            }
        }
    }
    return 0;
}

/* Forward substitution L z = b. */
void gpo_forward(int n, const real* L, const real* b, real* z) {
    for (int i = 0; i < n; ++i) {
        real s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * z[k];
        z[i] = s / L[(size_t)i * n + i];
    }
}

/* Back substitution L' w = e. */
void gpo_backward(int n, const real* L, const real* e, real* w) {
    for (int i = n - 1; i >= 0; --i) {
        real s = e[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * w[k];
        w[i] = s / L[(size_t)i * n + i];
    }
}

/* 1-norm condition estimate kappa_1(A) = ||A||_1 * est(||A^-1||_1) for
 * symmetric positive definite A = L L', with est(.) Hager's iteration
 * (W. W. Hager, "Condition estimates", SIAM J. Sci. Stat. Comput. 5, 1984),
 * at most 5 steps, using solves with L only.  The estimate is a lower bound
 * of the true condition number. */
real gpo_cond1_est(int n, const real* A, const real* L) {
    real* work = (real*)malloc(sizeof(real) * 5 * (size_t)n);
    if (!work) return NAN;
    real* v = work;
    real* yv = work + n;
    real* z = work + 2 * n;
    real* t = work + 3 * n;
    real* sg = work + 4 * n;
    real anorm = 0.0;
    for (int j = 0; j < n; ++j) {
        real c = 0.0;
        for (int i = 0; i < n; ++i) c += fabs(A[(size_t)i * n + j]);
        if (c > anorm) anorm = c;
    }
    for (int i = 0; i < n; ++i) v[i] = 1.0 / n;
    real est = 0.0;
    int jprev = -1;
    for (int iter = 0; iter < 5; ++iter) {
        gpo_forward(n, L, v, t);
        gpo_backward(n, L, t, yv);          /* yv = A^-1 v */
        est = 0.0;
        for (int i = 0; i < n; ++i) est += fabs(yv[i]);
        for (int i = 0; i < n; ++i) sg[i] = (yv[i] >= 0.0) ? 1.0 : -1.0;
        gpo_forward(n, L, sg, t);
        gpo_backward(n, L, t, z);           /* z = A^-T sign(yv), A symmetric */
        int jmax = 0;
        real zmax = fabs(z[0]);
        for (int i = 1; i < n; ++i)
            if (fabs(z[i]) > zmax) { zmax = fabs(z[i]); jmax = i; }
        real ztv = 0.0;
        for (int i = 0; i < n; ++i) ztv += z[i] * v[i];
        if (zmax <= ztv || jmax == jprev) break;
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        v[jmax] = 1.0;
        jprev = jmax;
    }
    free(work);
    return anorm * est;
}

/* Q = e'e is zero in exact arithmetic when Y lies in the span of 1 (always
 * so for n = 1).  In floating point e = b - mu a then holds only rounding
 * noise of size ~u |b|, so Q is taken as zero when it is no larger than
 * 16 n u^2 b'b (u the unit roundoff: 2^-53 in double), which includes
 * Q == 0 exactly. */
static int gpo_q_is_zero(int n, real Q, real bb) {
    const real u = GPO_UNIT_ROUNDOFF;
    return Q <= 16.0 * n * u * u * bb;
}

/* Profile -2 log-likelihood at one theta, eqs. (3)-(4) of Section 2.
 *
 * out[0] = -2logL = log|R| + n log Q            (eq. 4, literal)
 * out[1] = mu_hat = (1'R^-1 1)^-1 1'R^-1 Y       (eq. 3)
 * out[2] = sigma2_hat = Q / n                     (eq. 3)
 * out[3] = log|R| = 2 sum log L_ii
 * out[4] = Q = (Y - 1 mu_hat)' R^-1 (Y - 1 mu_hat)
 * out[5] = full Gaussian form log|R| + n log sigma2_hat + n (1 + log 2 pi)
 * out[6] = 1-norm condition estimate of R (0 if not requested)
 * Returns the status (0, NOTPD, DEGENERATE, ENOMEM).
 *
 * Route: R by eq. (2) -> Cholesky R = L L' -> a = L^-1 1, b = L^-1 Y, so that
 * 1'R^-1 1 = a'a and 1'R^-1 Y = a'b; e = b - mu a = L^-1 (Y - 1 mu) and
 * Q = e'e. */
int gpo_nll(int n, int d, const real* x, const real* y, const real* theta,
            real p, int fam, real delta, int want_cond, real* out) {
    const real nan = NAN;
    for (int i = 0; i < 7; ++i) out[i] = nan;
    out[6] = 0.0;
    real* R = (real*)malloc(sizeof(real) * (size_t)n * n);
    real* L = (real*)malloc(sizeof(real) * (size_t)n * n);
    real* ones = (real*)malloc(sizeof(real) * (size_t)n);
    real* a = (real*)malloc(sizeof(real) * (size_t)n);
    real* b = (real*)malloc(sizeof(real) * (size_t)n);
    real* e = (real*)malloc(sizeof(real) * (size_t)n);
    int status = GPO_OK;
    if (!R || !L || !ones || !a || !b || !e) { status = GPO_ENOMEM; goto done; }

    gpo_corr_matrix(n, d, x, theta, p, fam, delta, R);
    if (gpo_cholesky(n, R, L) != 0) {
        status = GPO_NOTPD;
        out[0] = INFINITY;
        out[5] = INFINITY;
        goto done;
    }
    for (int i = 0; i < n; ++i) ones[i] = 1.0;
    gpo_forward(n, L, ones, a);
    gpo_forward(n, L, y, b);
    real aa = 0.0, ab = 0.0;
    for (int i = 0; i < n; ++i) { aa += a[i] * a[i]; ab += a[i] * b[i]; }
    real mu = ab / aa;
    real Q = 0.0, bb = 0.0;
    for (int i = 0; i < n; ++i) { e[i] = b[i] - mu * a[i]; Q += e[i] * e[i]; bb += b[i] * b[i]; }
    real logdet = 0.0;
    for (int i = 0; i < n; ++i) logdet += log(L[(size_t)i * n + i]);
    logdet *= 2.0;
    real sigma2 = Q / n;
    out[1] = mu;
    out[2] = sigma2;
    out[3] = logdet;
    out[4] = Q;
    if (gpo_q_is_zero(n, Q, bb)) {
        status = GPO_DEGENERATE;
        out[0] = -INFINITY;
        out[5] = -INFINITY;
    } else {
        out[0] = logdet + n * log(Q);
        out[5] = logdet + n * log(sigma2) + n * (1.0 + log(2 * GPO_PI));
    }
    if (want_cond) out[6] = gpo_cond1_est(n, R, L);
done:
    free(R); free(L); free(ones); free(a); free(b); free(e);
    return status;
}

/* -2 log L at T candidate theta vectors (theta is T x d row-major); the
 * candidates are independent, so they are spread over host threads.  Each
 * evaluation is the single-threaded gpo_nll above.  out is T x 7. */
void gpo_nll_batch(int n, int d, const real* x, const real* y, int T,
                   const real* theta, real p, int fam, real delta, int want_cond,
                   real* out, int* status) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t)
        status[t] = gpo_nll(n, d, x, y, theta + (size_t)t * d, p, fam, delta,
                            want_cond, out + (size_t)t * 7);
}

/* Kriging prediction at N points xs (N x d) with the fit at theta.
 * yhat[m] = mu_hat + r' R^-1 (Y - 1 mu_hat)            (w = L^-T e)
 * s2[m]   = sigma2_hat [ c0 - r'R^-1 r + (1 - 1'R^-1 r)^2 / (1'R^-1 1) ]
 * where v = L^-1 r gives r'R^-1 r = v'v and 1'R^-1 r = a'v, and
 * c0 = 1 + delta if nugget_in_var else 1.  s2 may be NULL.
 * Returns the status of the fit. */
int gpo_predict(int n, int d, const real* x, const real* y, const real* theta,
                real p, int fam, real delta, int N, const real* xs, int nugget_in_var,
                real* yhat, real* s2) {
    real* R = (real*)malloc(sizeof(real) * (size_t)n * n);
    real* L = (real*)malloc(sizeof(real) * (size_t)n * n);
    real* ones = (real*)malloc(sizeof(real) * (size_t)n);
    real* a = (real*)malloc(sizeof(real) * (size_t)n);
    real* b = (real*)malloc(sizeof(real) * (size_t)n);
    real* e = (real*)malloc(sizeof(real) * (size_t)n);
    real* w = (real*)malloc(sizeof(real) * (size_t)n);
    int status = GPO_OK;
    if (!R || !L || !ones || !a || !b || !e || !w) { status = GPO_ENOMEM; goto done; }
    gpo_corr_matrix(n, d, x, theta, p, fam, delta, R);
    if (gpo_cholesky(n, R, L) != 0) {
        status = GPO_NOTPD;
        for (int m = 0; m < N; ++m) { yhat[m] = NAN; if (s2) s2[m] = NAN; }
        goto done;
    }
    for (int i = 0; i < n; ++i) ones[i] = 1.0;
    gpo_forward(n, L, ones, a);
    gpo_forward(n, L, y, b);
    real aa = 0.0, ab = 0.0;
    for (int i = 0; i < n; ++i) { aa += a[i] * a[i]; ab += a[i] * b[i]; }
    real mu = ab / aa;
    real Q = 0.0;
    for (int i = 0; i < n; ++i) { e[i] = b[i] - mu * a[i]; Q += e[i] * e[i]; }
    real sigma2 = Q / n;
    gpo_backward(n, L, e, w);
    real c0 = nugget_in_var ? 1.0 + delta : 1.0;
#pragma omp parallel
    {
        real* r = (real*)malloc(sizeof(real) * (size_t)n);
        real* v = (real*)malloc(sizeof(real) * (size_t)n);
#pragma omp for schedule(static)
        for (int m = 0; m < N; ++m) {
            if (!r || !v) { yhat[m] = NAN; if (s2) s2[m] = NAN; continue; }
            gpo_cross_corr(n, d, x, xs + (size_t)m * d, theta, p, fam, r);
            real yh = 0.0;
            for (int i = 0; i < n; ++i) yh += r[i] * w[i];
            yhat[m] = mu + yh;
            if (s2) {
                gpo_forward(n, L, r, v);
                real vv = 0.0, av = 0.0;
                for (int i = 0; i < n; ++i) { vv += v[i] * v[i]; av += a[i] * v[i]; }
                real g = 1.0 - av;
                s2[m] = sigma2 * (c0 - vv + g * g / aa);
            }
        }
        free(r); free(v);
    }
done:
    free(R); free(L); free(ones); free(a); free(b); free(e); free(w);
    return status;
}

/* The factor and the solve vectors of one fit, for tests that check the
 * intermediate quantities: L (n x n), a = L^-1 1, b = L^-1 Y, w = R^-1(Y-1mu).
 * Returns the status. */
int gpo_fit_parts(int n, int d, const real* x, const real* y, const real* theta,
                  real p, int fam, real delta, real* R, real* L, real* a, real* b,
                  real* w) {
    gpo_corr_matrix(n, d, x, theta, p, fam, delta, R);
    if (gpo_cholesky(n, R, L) != 0) return GPO_NOTPD;
    real* ones = (real*)malloc(sizeof(real) * (size_t)n);
    real* e = (real*)malloc(sizeof(real) * (size_t)n);
    if (!ones || !e) { free(ones); free(e); return GPO_ENOMEM; }
    for (int i = 0; i < n; ++i) ones[i] = 1.0;
    gpo_forward(n, L, ones, a);
    gpo_forward(n, L, y, b);
    real aa = 0.0, ab = 0.0;
    for (int i = 0; i < n; ++i) { aa += a[i] * a[i]; ab += a[i] * b[i]; }
    real mu = ab / aa;
    for (int i = 0; i < n; ++i) e[i] = b[i] - mu * a[i];
    gpo_backward(n, L, e, w);
    free(ones); free(e);
    return GPO_OK;
}

/* d/dtheta_k of one dimension's factor, divided by the factor itself:
 * dlog rho / dtheta for the family (h = c theta |dx| for the Matern forms):
 *   power-exponential: -|dx|^p
 *   nu = 1/2:  -|dx|
 *   nu = 3/2:  rho' / rho = -h / (1 + h) * sqrt(3) |dx|
 *   nu = 5/2:  rho' / rho = -h (1 + h) / (3 (1 + h + h^2/3)) * sqrt(5) |dx| */
static real gpo_dlog_corr_1d(real diff, real theta, real p, int fam) {
    real a = fabs(diff);
    if (fam == GPO_MATERN12) return -a;
    if (fam == GPO_MATERN32) {
        real h = sqrt((real)3) * theta * a;
        return -h / (1.0 + h) * sqrt((real)3) * a;
    }
    if (fam == GPO_MATERN52) {
        real h = sqrt((real)5) * theta * a;
        return -h * (1.0 + h) / (3.0 * (1.0 + h + h * h / 3.0)) * sqrt((real)5) * a;
    }
    return -pow(a, p);
}

/* Gradient of -2 log L (eq. 4) with respect to theta at one theta:
 *   d(-2logL)/dtheta_k = tr(R^-1 dR_k) - (n / Q) w' dR_k w,
 * from d log|R| = tr(R^-1 dR) and, mu_hat being the minimiser of Q over mu,
 * dQ = -w' dR w with w = R^-1 (Y - 1 mu_hat).  dR_k = dR/dtheta_k is
 * R_ij dlog rho(x_ik - x_jk)/dtheta_k off the diagonal and 0 on it (the
 * nugget and the unit diagonal do not depend on theta).  R^-1 is formed
 * column by column by two triangular solves of e_j.  grad has d entries;
 * out is filled as by gpo_nll.  Returns the status (grad NaN if not OK). */
int gpo_nll_grad(int n, int d, const real* x, const real* y, const real* theta,
                 real p, int fam, real delta, real* grad, real* out) {
    int status = gpo_nll(n, d, x, y, theta, p, fam, delta, 0, out);
    for (int k = 0; k < d; ++k) grad[k] = NAN;
    if (status != GPO_OK) return status;
    real* R = (real*)malloc(sizeof(real) * (size_t)n * n);
    real* L = (real*)malloc(sizeof(real) * (size_t)n * n);
    real* Ri = (real*)malloc(sizeof(real) * (size_t)n * n);
    real* a = (real*)malloc(sizeof(real) * (size_t)n);
    real* b = (real*)malloc(sizeof(real) * (size_t)n);
    real* w = (real*)malloc(sizeof(real) * (size_t)n);
    real* col = (real*)malloc(sizeof(real) * (size_t)n);
    real* tmp = (real*)malloc(sizeof(real) * (size_t)n);
    if (!R || !L || !Ri || !a || !b || !w || !col || !tmp) {
        status = GPO_ENOMEM;
        goto done;
    }
    status = gpo_fit_parts(n, d, x, y, theta, p, fam, delta, R, L, a, b, w);
    if (status != GPO_OK) goto done;
    for (int j = 0; j < n; ++j) {          /* column j of R^-1 = L^-T L^-1 e_j */
        for (int i = 0; i < n; ++i) col[i] = (i == j) ? 1.0 : 0.0;
        gpo_forward(n, L, col, tmp);
        gpo_backward(n, L, tmp, col);
        for (int i = 0; i < n; ++i) Ri[(size_t)i * n + j] = col[i];
    }
    {
        const real Q = out[4];
        for (int k = 0; k < d; ++k) {
            real tr = 0.0, quad = 0.0;
            for (int i = 0; i < n; ++i) {
                for (int j = 0; j < n; ++j) {
                    if (i == j) continue;
                    const real* xi = x + (size_t)i * d;
                    const real* xj = x + (size_t)j * d;
                    const real dR = R[(size_t)i * n + j] * gpo_dlog_corr_1d(xi[k] - xj[k], theta[k], p, fam);
                    tr += Ri[(size_t)j * n + i] * dR;
                    quad += w[i] * dR * w[j];
                }
            }
            grad[k] = tr - n / Q * quad;
        }
    }
done:
    free(R); free(L); free(Ri); free(a); free(b); free(w); free(col); free(tmp);
    return status;
}

int gpo_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
