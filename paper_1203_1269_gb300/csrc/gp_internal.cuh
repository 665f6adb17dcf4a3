// gp_internal.cuh -- shared definitions of libgp's CUDA sources.
//
// Storage of R and of its Cholesky factor (per instance): the lower
// triangle in NB x NB tiles.  Tile (I, J), I >= J, starts at tile index
// J*nt - J*(J-1)/2 + (I - J) (tile columns packed one after another), and
// is column-major inside (element (r, c) at r + NB*c).  Rows/columns >= n
// hold the identity so that the padded factor is block-diag(L, I).
// Diagonal tiles hold both triangles of R; after factorisation their
// lower triangle holds L.
#pragma once

#include <atomic>
#include <mutex>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <cuda_bf16.h>

#include "../../include/gp.h"

#define GP_NB 128
#define GP_TILE_ELEMS (GP_NB * GP_NB)
#define GP_MAX_D 64
#define GP_MAX_SLICES 7
#define GP_PANEL_SLICES 7

namespace gp {

// Candidates one call takes: the chunk loops over them stay in int.
constexpr int kMaxCandidates = 1 << 30;

__host__ __device__ inline int num_tiles(int n) { return (n + GP_NB - 1) / GP_NB; }

__host__ __device__ inline long long tile_index(int I, int J, int nt) {
    return (long long)J * nt - (long long)J * (J - 1) / 2 + (I - J);
}

__host__ __device__ inline long long packed_tiles(int nt) {
    return (long long)nt * (nt + 1) / 2;
}

__host__ __device__ inline size_t packed_elems(int n) {
    int nt = num_tiles(n);
    return (size_t)packed_tiles(nt) * GP_TILE_ELEMS;
}

// lower-triangle linear index q -> (i, k), k <= i, over an m x m triangle
// (a float square root seeds r, the integer loops make it exact: FP64 is
// scarce on this GPU and this runs once per work item in every warp role)
__device__ inline void tri_decode(int q, int& i, int& k) {
    int r = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
    while ((long long)(r + 1) * (r + 2) / 2 <= q) ++r;
    while ((long long)r * (r + 1) / 2 > q) --r;
    i = r;
    k = q - r * (r + 1) / 2;
}

// Per-instance record written by the factorisation and solve kernels.
struct InstState {
    double logdet;
    double aa;      // 1'R^-1 1
    double ab;      // 1'R^-1 Y
    double mu;
    double Q;
    double bb;
    int status;
    int fail_col;
    // 1-norm condition estimate (split path, k_cond.cu): ||R||_1, Hager's
    // estimate of ||R^-1||_1 and the iteration's state
    double anorm;
    double est;
    int hager_iter;
    int hager_jprev;
    int hager_done;   // 1: the estimate has stopped; the solve kernels skip the instance
    // iterative refinement of the split path (k_mixed.cu)
    double piv_inv;   // sum_i 1 / L_ii^2 over the factor's pivots
    double dq_prev;   // change of n log Q made by the previous refinement step
    int refine_done;  // 1: the refinement has stopped; the solve kernels skip the instance
};

// Batched problem description handed to the kernels (by value).
struct Batch {
    int n, d, nt, count;          // count = instances in this launch chunk
    double p, delta;
    const double* x;              // n x d
    const double* y;              // n
    const double* theta;          // count x d (already offset to the chunk)
    double* A;                    // count * packed_elems(n)   (double tiles), or
    float2* Adf;                  // double-float tiles (split path; A unused then)
    float2* Rdf;                  // double-float copy of R (split path)
    size_t inst_stride;           // elements between instances in A / Adf / Rdf
    InstState* st;                // count
    int asm_cols;                 // double-float assembly: tile columns per CTA (16 or 32)
    int corr;                     // gp_correlation
};

// Split-precision path: per-instance buffers (double-float tiles, bf16
// slice images of the current panel and of W = L_JJ^-1, solve vectors).
struct MixedBatch {
    int n, d, nt, count;
    double delta;                 // the nugget (the refinement's log-det error estimate)
    int s;                        // slices of the trailing update operands
    int ps;                       // slices of the panel solve operands (GP_PANEL_SLICES)
    int ug;                       // accumulator groups of the trailing update (3, 4 or 7)
    int inject_timeout;           // test hook: one split-GEMM CTA waits on a barrier nothing signals
    int update_tile;              // columns of a trailing-update output tile (128 or 64)
    int sp;                       // slice slots per row block in PS (max(s, ps))
    float2* A;                    // working matrix -> factor (double-float tiles)
    float2* Rc;                   // copy of R (double-float tiles), for residuals
    size_t inst_stride;
    __nv_bfloat16* PS;            // panel slices: [row block][slice][4 chunks][128 x 32]
    int* PE;                      // panel row exponents: [row block][128]
    __nv_bfloat16* WS;            // slices of W's rows: [slice][4 chunks][128 x 32]
    int* WE;                      // [128]
    __nv_bfloat16* PF;            // two-panel slices for the fused update: [row block][slice][8 chunks][128 x 32]
    int* FE;                      // their row exponents: [row block][128]
    size_t pf_stride, fe_stride;
    int fuse;                     // 1: trailing updates of panel pairs fused (K = 256)
    int fwd;                      // 1: the forward solve L [x_1 x_y] = [1 Y] runs inside the
                                  // factorisation (diagonal blocks and panel slicing)
    float2* WT;                   // L_JJ^-1 per diagonal block, double-float tiles: [J][128 x 128]
    float2* WR;                   // the same, row-major (its transpose column-major), stride wt_stride
    size_t wt_stride;
    size_t ps_stride, pe_stride, ws_stride, we_stride;
    float2* Z;                    // 10 columns of npad double-float values: x_1, x_y, two
                                  // residual / correction columns, 1 / L_ii, two
                                  // condition-estimate columns, |R| row sums, and
                                  // a = L^-1 1, b = L^-1 Y (kept from the forward solve)
    size_t z_stride;
    float2* RP;                   // per-tile partial sums of the tile-parallel solves and residual
    size_t rp_stride;
    int* SC;                      // per-block counters of the tile-parallel substitutions
    size_t sc_stride;
    const double* y;
    InstState* st;
    int* err;                     // set when a bounded device wait gave up
};

constexpr int kZCols = 10;
// kernel launches of one forward or backward substitution pass (the first
// block's diagonal step, then a tile step per further block column that
// also finishes the next block)
inline int subst_launches(int nt) { return nt; }
// partial sums of the tile-parallel residual per lower tile: row products
// [2 column halves][2 right-hand sides][128], then column products [2][2][64]
constexpr int kRpTile = 2 * 2 * GP_NB + 2 * 2 * (GP_NB / 2);

// A kernel's dynamic shared-memory limit is a per-device attribute: each
// launcher keeps the largest size it has set on every device ordinal and
// raises the limit once per device (and again when it needs more).  Threads
// that launch the same kernel with different sizes (contexts on several
// streams) take a lock around the check and the attribute call, so the
// attribute only ever grows: without it, a thread setting a smaller size
// after another set a larger one would leave the larger launches refused.
constexpr int kMaxDevices = 64;
inline std::mutex& smem_limit_mutex() {
    static std::mutex m;
    return m;
}
template <typename Kernel>
inline cudaError_t raise_smem_limit(Kernel* kernel, size_t bytes, std::atomic<size_t> (&done)[kMaxDevices]) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kMaxDevices;
    if (cached && bytes <= done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(smem_limit_mutex());
    if (cached && bytes <= done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && cached) done[dev].store(bytes, std::memory_order_release);
    return e;
}

// ---- context accessors (gp_capi.cu) ----------------------------------------
int ctx_fail(gp_ctx* ctx, int code, const char* fmt, ...);
int ctx_device(const gp_ctx* ctx);
// the argument checks every entry point shares: n, d, p (for eq. 2's family), delta
int ctx_check_common(gp_ctx* ctx, int n, int d, double p, double delta);
int ctx_correlation(const gp_ctx* ctx);
cudaStream_t ctx_stream(const gp_ctx* ctx);

// ---- kernels (launch helpers, all on `stream`) ----------------------------
cudaError_t launch_validate_theta(const Batch& b, cudaStream_t s);
cudaError_t launch_assemble_tiles(const Batch& b, cudaStream_t s);
cudaError_t launch_assemble_dense(int n, int d, const double* x, const double* theta, double p, int corr,
                                  double delta, double* R, cudaStream_t s);
cudaError_t launch_potrf_f64(const Batch& b, int J, cudaStream_t s);
cudaError_t launch_trsm_f64(const Batch& b, int J, cudaStream_t s);
// the tiles of a trailing update: all, column J + 1 only, or the others
enum : int { kUpdateAll = 0, kUpdateColumn = 1, kUpdateRest = 2 };
cudaError_t launch_update_f64(const Batch& b, int J, cudaStream_t s, int which = kUpdateAll);
cudaError_t launch_forward_solve(const Batch& b, double* Z, size_t z_stride, cudaStream_t s);
cudaError_t launch_finalize(const Batch& b, const double* Z, size_t z_stride, double* nll,
                            double* mu, double* sigma2, double* logdet, int* status,
                            cudaStream_t s);
cudaError_t launch_fit_finish(const Batch& b, double* Z, size_t z_stride, double* scalars,
                              cudaStream_t s);
cudaError_t launch_backward_solve(const Batch& b, double* Z, size_t z_stride, int col,
                                  cudaStream_t s);
// kernels that launch_forward_solve (backward = false) or launch_backward_solve launch
int solve_f64_launches(int nt, bool backward);
// Kriging with the variance's solve on the tensor cores (k_var_tc.cu).
struct VarTables {
    __nv_bfloat16* LS;            // slices of the rows of L left of the diagonal blocks
    __nv_bfloat16* WS;            // slices of the rows of W_J = L_JJ^-1
    int* LE;                      // npad row exponents of LS
    int* WE;                      // npad row exponents of WS
    int* lbits;                   // npad scratch: row maxima as float bits
};
struct VarCall {
    int n, d, nt, N, corr;
    double p, c0;
    int ev;                       // fixed exponent of the slices of v = L^-1 r
    int inject_timeout;
    const float2* x;              // n x d design points (double-float)
    const double* theta;
    const float2* w;              // npad: R^-1 (Y - 1 mu_hat)
    const float2* a;              // npad: L^-1 1
    const double* sc;             // model scalars
    const double* xs;             // N x d
    double* yhat;
    double* s2;                   // null: means only
    VarTables t;
    int* err;
    float2* rtab;                 // var_rhs_tab_bytes(): the r kernel's tables
};
size_t var_table_bytes(int nt);
size_t var_rx_bytes(int nt);      // per point block
size_t var_mp_bytes(int nt);      // per point block
size_t var_vs_bytes(int nt);      // per CTA: the slices of V
size_t var_cta_bytes(int nt);     // per CTA of the tensor-core pass: V's and C_J's slices
size_t var_rhs_tab_bytes();
VarTables var_tables_at(void* base, int nt);
cudaError_t launch_var_rhs_tables(const VarCall& c, cudaStream_t s, int* kernels);
cudaError_t launch_var_tables(const float2* L, int nt, const VarTables& t, cudaStream_t s, int* kernels);
cudaError_t launch_var_points(const VarCall& c, int m0, int npb, float2* RX, float2* MP, cudaStream_t s,
                              int* kernels);
cudaError_t launch_var_pass(const VarCall& c, int m0, int npb, const float2* RX, __nv_bfloat16* VS,
                            __nv_bfloat16* CS, int grid, cudaStream_t s, int* kernels);
cudaError_t launch_predict(int n, int d, int nt, const float2* x, const double* theta, double p, int corr, double c0,
                           const float2* L, const float2* w, const float2* a, const double* scalars, int N,
                           const double* xs, double* yhat, double* s2, float2* work, int chunk, int nr,
                           cudaStream_t s);
cudaError_t launch_to_df_inplace(double* p, size_t count, cudaStream_t s);
size_t predict_work_per_cta(int nt, int nr);
// test points per CTA for N points on a device of `sms` SMs (8 or 16)
int predict_points_per_cta(int N, int sms);

cudaError_t launch_diag_mixed(const MixedBatch& b, int J, cudaStream_t s);
cudaError_t launch_split_panel(const MixedBatch& b, int J, int ns, int gemv, cudaStream_t s);
cudaError_t launch_gemm_panel(const MixedBatch& b, int J, cudaStream_t s);
cudaError_t launch_gemm_update(const MixedBatch& b, int J, cudaStream_t s);
cudaError_t launch_gemm_update_column(const MixedBatch& b, int J, cudaStream_t s);
cudaError_t launch_gemm_update_fused(const MixedBatch& b, int J, cudaStream_t s);
cudaError_t launch_split_fused(const MixedBatch& b, int J, cudaStream_t s);
cudaError_t launch_df_forward(const MixedBatch& b, int c0, int init, cudaStream_t s);
cudaError_t launch_rhs_init(const MixedBatch& b, cudaStream_t s);
cudaError_t launch_df_backward(const MixedBatch& b, int c0, int add_to, cudaStream_t s);
cudaError_t launch_df_residual(const MixedBatch& b, cudaStream_t s);
cudaError_t launch_grad(const Batch& b, double* Z, size_t zs, double* X, double* Ri, double* partial,
                        const int* status, double* grad, cudaStream_t s, int* kernels);
cudaError_t launch_norm1(const MixedBatch& b, cudaStream_t s);
cudaError_t launch_hager(const MixedBatch& b, int phase, double* cond, cudaStream_t s);
cudaError_t launch_fill_int(int* dst, int count, int value, cudaStream_t s);
cudaError_t launch_scatter(int m, const int* idx, const double* src, double* dst, cudaStream_t s);
cudaError_t launch_scatter_int(int m, const int* idx, const int* src, int* dst, cudaStream_t s);
cudaError_t launch_df_finalize(const MixedBatch& b, double* nll, double* mu, double* sigma2,
                               double* logdet, int* status, cudaStream_t s);
cudaError_t launch_keep_forward(const MixedBatch& b, cudaStream_t s);
cudaError_t launch_refine_check(const MixedBatch& b, int step, cudaStream_t s);
cudaError_t launch_split_model(const MixedBatch& v, float2* Zm, double* scalars, const double* nll,
                               const int* status, int* status_out, cudaStream_t s);
cudaError_t launch_df_to_double(const float2* src, double* dst, size_t count, cudaStream_t s);

}  // namespace gp
