// gp_capi.cu -- the C ABI of libgp (declared in include/gp.h): contexts,
// argument checks, the device workspace, batching of theta candidates and
// the sequence of kernel launches for each call.
#include <algorithm>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "gp_internal.cuh"

struct gp_ctx {
    int device = 0;
    int sms = 1;                // streaming multiprocessors of the device
    cudaStream_t stream = nullptr;
    size_t budget = 0;          // bytes the context and its models may hold
    size_t models_bytes = 0;    // held by live models
    gp_options opt;
    void* ws = nullptr;         // workspace arena
    size_t ws_bytes = 0;
    std::string err;
    // phase timers (CUDA events on the context's stream) and launch counter
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_open;
    double phase_ms[GP_NUM_PHASES] = {0};
    std::vector<gp_model*> models;   // live models (detached when the context goes first)
    std::vector<gp_plan*> plans;     // live plans (likewise)
    long long phase_launches[GP_NUM_PHASES] = {0};
    long long launches = 0;
    // a second stream for work that overlaps the main stream inside a call
    // (forked from and joined back to it with the two events)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the FP64 factorisation's look-ahead: a high-priority stream
    cudaStream_t la = nullptr;
    cudaEvent_t ev_la0 = nullptr, ev_la1 = nullptr;
};

struct gp_model {
    gp_ctx* ctx = nullptr;
    int n = 0, d = 0, nt = 0, prec = 0;
    int corr = 0;               // gp_correlation the fit was made with
    double p = 0.0, delta = 0.0;
    void* mem = nullptr;        // one allocation holding everything below
    size_t bytes = 0;
    double* L = nullptr;        // packed factor tiles
    double* Z = nullptr;        // [a | w], 2 * npad
    double* x = nullptr;        // n x d
    double* theta = nullptr;    // d
    double* scalars = nullptr;  // nll, mu, sigma2, logdet, Q, aa (+2 spare)
    int* status = nullptr;
    gp::InstState* st = nullptr;
    double host_scalars[6];
};

struct gp_plan {
    gp_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* ws = nullptr;         // the plan's own workspace
    size_t ws_bytes = 0;
    long long kernels = 0;
};

namespace {

cudaEvent_t take_event(gp_ctx* ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket a group of launches of one phase with events (when timing is on)
// and count the kernels it launched.
struct PhaseScope {
    gp_ctx* ctx;
    int phase;
    int kernels;
    cudaEvent_t e0 = nullptr;
    cudaStream_t st;
    PhaseScope(gp_ctx* c, int ph, int k, cudaStream_t on = nullptr)
        : ctx(c), phase(ph), kernels(k), st(on ? on : c->stream) {
        if (ctx->timing) {
            e0 = take_event(ctx);
            cudaEventRecord(e0, st);
        }
    }
    ~PhaseScope() {
        ctx->launches += kernels;
        ctx->phase_launches[phase] += kernels;
        if (ctx->timing) {
            cudaEvent_t e1 = take_event(ctx);
            cudaEventRecord(e1, st);
            ctx->ev_open.push_back({phase, {e0, e1}});
        }
    }
};

int fail(gp_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

#define GP_CUDA(ctx, call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail((ctx), GP_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                            \
    } while (0)

int check_common(gp_ctx* ctx, int n, int d, double p, double delta) {
    if (!ctx) return GP_EINVAL;
    if (n < 1 || n > (1 << 20)) return fail(ctx, GP_EINVAL, "n = %d out of range [1, 2^20]", n);
    if (d < 1 || d > GP_MAX_D) return fail(ctx, GP_EINVAL, "d = %d out of range [1, %d]", d, GP_MAX_D);
    if (ctx->opt.correlation == GP_CORR_POWEXP && !(p > 0.0 && p <= 2.0))
        return fail(ctx, GP_EINVAL, "p = %g outside (0, 2]", p);
    if (!(delta >= 0.0) || !std::isfinite(delta))
        return fail(ctx, GP_EINVAL, "delta = %g must be finite and >= 0", delta);
    return GP_OK;
}

// Make the workspace at least `bytes` large, within the budget.
int ensure_ws(gp_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return GP_OK;
    if (bytes + ctx->models_bytes > ctx->budget)
        return fail(ctx, GP_ENOMEM, "workspace of %zu bytes exceeds the HBM budget (%zu, %zu held by models)",
                    bytes, ctx->budget, ctx->models_bytes);
    // stream-ordered: no device-wide synchronisation, so contexts on other
    // streams keep running while this one grows its workspace
    if (ctx->ws) {
        cudaFreeAsync(ctx->ws, ctx->stream);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    cudaError_t e = cudaMallocAsync(&ctx->ws, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return fail(ctx, GP_ENOMEM, "workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->ws_bytes = bytes;
    return GP_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Bytes of workspace per instance of the FP64 path.
size_t per_instance_bytes_f64(int n) {
    const int nt = gp::num_tiles(n);
    return align256(gp::packed_elems(n) * sizeof(double)) +
           align256((size_t)2 * nt * GP_NB * sizeof(double)) + align256(sizeof(gp::InstState));
}

// Candidates per chunk of a batched call and the workspace it grows to:
// `per` bytes per candidate plus `extra`, within the budget left next to the
// models, the max_batch option and the grid.y bound (65535) of the
// per-candidate launches.  False when not even one candidate fits.
struct Chunking {
    int Tc = 0;
    size_t bytes = 0;
};

bool chunk_batch(const gp_options& opt, size_t budget, size_t held, size_t per, size_t extra, int T,
                 Chunking* out) {
    const size_t avail = budget > held ? budget - held : 0;
    long long cap = (long long)((avail > extra ? avail - extra : 0) / per);
    if (opt.max_batch > 0 && cap > opt.max_batch) cap = opt.max_batch;
    if (cap > 65535) cap = 65535;
    if (cap < 1) return false;
    out->Tc = (int)(cap < T ? cap : T);
    out->bytes = per * (size_t)out->Tc + extra;
    return true;
}

int ensure_la(gp_ctx* ctx) {
    if (ctx->la) return GP_OK;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&ctx->la, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_la0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_la1, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GP_ECUDA, "creating the look-ahead stream failed");
    }
    return GP_OK;
}

// Batches of at most this many instances factor with a look-ahead.
constexpr int kLookaheadMax = 16;

// Factor `b.count` instances already assembled in b.A.  A small batch (a
// fit's one instance) cannot fill the GPU with the serial diagonal step and
// the panel of a block column, so it looks ahead by one: after the update
// of column J + 1 (its tiles only), the diagonal step and panel of J + 1 run
// on a high-priority stream beside the rest of update J (their CTAs fit on
// an SM beside an update CTA).  Every tile still takes its updates in
// block-column order on the main stream: the same bits as without.
int run_factor_f64(gp_ctx* ctx, const gp::Batch& b) {
    const int nt = b.nt;
    if (b.count <= kLookaheadMax && nt > 1) {
        int rc = ensure_la(ctx);
        if (rc) return rc;
        {
            PhaseScope ps(ctx, GP_PHASE_POTRF, 1);
            GP_CUDA(ctx, gp::launch_potrf_f64(b, 0, ctx->stream));
        }
        {
            PhaseScope ps(ctx, GP_PHASE_TRSM, 1);
            GP_CUDA(ctx, gp::launch_trsm_f64(b, 0, ctx->stream));
        }
        for (int J = 0; J + 1 < nt; ++J) {
            {
                PhaseScope ps(ctx, GP_PHASE_UPDATE, 1);
                GP_CUDA(ctx, gp::launch_update_f64(b, J, ctx->stream, gp::kUpdateColumn));
            }
            GP_CUDA(ctx, cudaEventRecord(ctx->ev_la0, ctx->stream));
            GP_CUDA(ctx, cudaStreamWaitEvent(ctx->la, ctx->ev_la0, 0));
            {
                PhaseScope ps(ctx, GP_PHASE_POTRF, 1, ctx->la);
                GP_CUDA(ctx, gp::launch_potrf_f64(b, J + 1, ctx->la));
            }
            if (J + 2 < nt) {
                PhaseScope ps(ctx, GP_PHASE_TRSM, 1, ctx->la);
                GP_CUDA(ctx, gp::launch_trsm_f64(b, J + 1, ctx->la));
            }
            GP_CUDA(ctx, cudaEventRecord(ctx->ev_la1, ctx->la));
            if (J + 2 < nt) {
                PhaseScope ps(ctx, GP_PHASE_UPDATE, 1);
                GP_CUDA(ctx, gp::launch_update_f64(b, J, ctx->stream, gp::kUpdateRest));
            }
            GP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_la1, 0));
        }
        return GP_OK;
    }
    for (int J = 0; J < b.nt; ++J) {
        const int more = (J + 1 < b.nt) ? 1 : 0;
        {
            PhaseScope ps(ctx, GP_PHASE_POTRF, 1);
            GP_CUDA(ctx, gp::launch_potrf_f64(b, J, ctx->stream));
        }
        if (more) {
            PhaseScope ps(ctx, GP_PHASE_TRSM, 1);
            GP_CUDA(ctx, gp::launch_trsm_f64(b, J, ctx->stream));
        }
        if (more) {
            PhaseScope ps(ctx, GP_PHASE_UPDATE, 1);
            GP_CUDA(ctx, gp::launch_update_f64(b, J, ctx->stream));
        }
    }
    return GP_OK;
}

// Bytes of workspace per instance of the split-precision path.
struct MixedSizes {
    size_t A, PS, PE, WS, WE, PF, FE, WT, Z, RP, SC, st, per;   // WT also sizes WR
};

// Bytes after the instances of a split-precision batch: its error flag.
constexpr size_t kMixedTail = 256;

MixedSizes mixed_sizes(int n, int s) {
    const int nt = gp::num_tiles(n);
    const int ps = GP_PANEL_SLICES;
    const int sp = s > ps ? s : ps;
    MixedSizes z;
    z.A = align256(gp::packed_elems(n) * sizeof(float2));
    z.PS = align256((size_t)nt * sp * GP_TILE_ELEMS * sizeof(__nv_bfloat16));
    z.PE = align256((size_t)nt * GP_NB * sizeof(int));
    z.WS = align256((size_t)ps * GP_TILE_ELEMS * sizeof(__nv_bfloat16));
    z.WE = align256((size_t)GP_NB * sizeof(int));
    z.PF = align256((size_t)nt * s * 2 * GP_TILE_ELEMS * sizeof(__nv_bfloat16));
    z.FE = align256((size_t)nt * GP_NB * sizeof(int));
    z.WT = align256((size_t)nt * GP_TILE_ELEMS * sizeof(float2));
    z.Z = align256((size_t)gp::kZCols * nt * GP_NB * sizeof(float2));
    z.RP = align256((size_t)gp::packed_tiles(nt) * gp::kRpTile * sizeof(float2));
    z.SC = align256((size_t)nt * sizeof(int));
    z.st = align256(sizeof(gp::InstState));
    z.per = 2 * z.A + z.PS + z.PE + z.WS + z.WE + z.PF + z.FE + 2 * z.WT + z.Z + z.RP + z.SC + z.st;
    return z;
}

// Carve the split-precision buffers of `cnt` instances out of `base`.
gp::MixedBatch mixed_layout(gp_ctx* ctx, int n, int cnt, const double* y, char* base, const MixedSizes& z,
                            int Tc, int slices) {
    gp::MixedBatch mb{};
    char* c = base;
    mb.A = (float2*)c; c += z.A * Tc;
    mb.Rc = (float2*)c; c += z.A * Tc;
    mb.PS = (__nv_bfloat16*)c; c += z.PS * Tc;
    mb.PE = (int*)c; c += z.PE * Tc;
    mb.WS = (__nv_bfloat16*)c; c += z.WS * Tc;
    mb.WE = (int*)c; c += z.WE * Tc;
    mb.PF = (__nv_bfloat16*)c; c += z.PF * Tc;
    mb.FE = (int*)c; c += z.FE * Tc;
    mb.WT = (float2*)c; c += z.WT * Tc;
    mb.WR = (float2*)c; c += z.WT * Tc;
    mb.Z = (float2*)c; c += z.Z * Tc;
    mb.RP = (float2*)c; c += z.RP * Tc;
    mb.SC = (int*)c; c += z.SC * Tc;
    mb.st = (gp::InstState*)c; c += z.st * Tc;
    mb.err = (int*)c;
    mb.n = n; mb.nt = gp::num_tiles(n); mb.count = cnt; mb.s = slices;
    mb.ps = GP_PANEL_SLICES;
    mb.ug = ctx->opt.update_groups;
    mb.inject_timeout = ctx->opt.inject_timeout & 1;
    mb.update_tile = ctx->opt.update_tile;
    mb.sp = mb.s > mb.ps ? mb.s : mb.ps;
    mb.inst_stride = z.A / sizeof(float2);
    mb.ps_stride = z.PS / sizeof(__nv_bfloat16);
    mb.pe_stride = z.PE / sizeof(int);
    mb.ws_stride = z.WS / sizeof(__nv_bfloat16);
    mb.we_stride = z.WE / sizeof(int);
    mb.pf_stride = z.PF / sizeof(__nv_bfloat16);
    mb.fe_stride = z.FE / sizeof(int);
    mb.wt_stride = z.WT / sizeof(float2);
    mb.fuse = ctx->opt.fuse_panels;
    mb.fwd = y != nullptr;
    mb.z_stride = z.Z / sizeof(float2);
    mb.rp_stride = z.RP / sizeof(float2);
    mb.sc_stride = z.SC / sizeof(int);
    mb.y = y;
    return mb;
}

// The context's second stream and its fork / join events (made on first use).
int ensure_aux(gp_ctx* ctx) {
    if (ctx->aux) return GP_OK;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GP_ECUDA, "creating the auxiliary stream failed");
    }
    return GP_OK;
}

// Assemble and factor (split precision) the instances of `mb`.
int run_mixed_factor(gp_ctx* ctx, gp::MixedBatch& mb, int d, const double* x, const double* theta, double p,
                     double delta) {
    gp::Batch b{};
    b.n = mb.n; b.d = d; b.nt = mb.nt; b.count = mb.count; b.p = p; b.delta = delta;
    b.corr = ctx->opt.correlation;
    b.x = x; b.y = mb.y; b.theta = theta; b.A = nullptr; b.Adf = mb.A; b.Rdf = mb.Rc;
    b.inst_stride = mb.inst_stride; b.st = mb.st;
    b.asm_cols = ctx->opt.assemble_cols;
    mb.d = d;
    mb.delta = delta;
    GP_CUDA(ctx, cudaMemsetAsync(mb.err, 0, sizeof(int), ctx->stream));
    {
        PhaseScope ps(ctx, GP_PHASE_ASSEMBLE, mb.fwd ? 3 : 2);
        GP_CUDA(ctx, gp::launch_validate_theta(b, ctx->stream));
        GP_CUDA(ctx, gp::launch_assemble_tiles(b, ctx->stream));
        if (mb.fwd) GP_CUDA(ctx, gp::launch_rhs_init(mb, ctx->stream));
    }
    const int nt = mb.nt;
    int rc = ensure_aux(ctx);
    if (rc) return rc;
    // Diagonal block J and the slices of panel J's tiles for the panel solve
    // touch disjoint buffers: the slicing runs on the second stream while
    // the diagonal kernel (latency-bound, about one CTA per SM) runs on the
    // main one, and the panel solve waits for both.
    auto diag_and_slices = [&](int J) -> int {
        const bool slices = J + 1 < nt;
        if (slices) GP_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
        {
            PhaseScope ps(ctx, GP_PHASE_POTRF, 1);
            GP_CUDA(ctx, gp::launch_diag_mixed(mb, J, ctx->stream));
        }
        if (slices) {
            GP_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
            ctx->launches += 1;
            ctx->phase_launches[GP_PHASE_SPLIT] += 1;
            GP_CUDA(ctx, gp::launch_split_panel(mb, J, mb.ps, 0, ctx->aux));
            GP_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->aux));
            // the time the main stream waits here is the slicing left exposed
            PhaseScope ps(ctx, GP_PHASE_SPLIT, 0);
            GP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
        }
        return GP_OK;
    };
    auto panel = [&](int J) -> int {
        PhaseScope ps(ctx, GP_PHASE_TRSM, 1);
        GP_CUDA(ctx, gp::launch_gemm_panel(mb, J, ctx->stream));
        return GP_OK;
    };
    int J = 0;
    while (J < nt) {
        rc = diag_and_slices(J);
        if (rc) return rc;
        if (J + 1 == nt) break;
        rc = panel(J);
        if (rc) return rc;
        {
            PhaseScope ps(ctx, GP_PHASE_SPLIT, 1);
            GP_CUDA(ctx, gp::launch_split_panel(mb, J, mb.s, 1, ctx->stream));
        }
        if (mb.fuse && J + 2 < nt) {
            // panel pair (J, J + 1): update column J + 1 from panel J, factor and
            // solve panel J + 1, then apply both panels to the trailing tiles in
            // one K = 256 pass
            {
                PhaseScope ps(ctx, GP_PHASE_UPDATE, 1);
                GP_CUDA(ctx, gp::launch_gemm_update_column(mb, J, ctx->stream));
            }
            rc = diag_and_slices(J + 1);
            if (rc) return rc;
            rc = panel(J + 1);
            if (rc) return rc;
            {
                PhaseScope ps(ctx, GP_PHASE_SPLIT, 1);
                GP_CUDA(ctx, gp::launch_split_fused(mb, J, ctx->stream));
            }
            {
                PhaseScope ps(ctx, GP_PHASE_UPDATE, 1);
                GP_CUDA(ctx, gp::launch_gemm_update_fused(mb, J, ctx->stream));
            }
            J += 2;
        } else {
            PhaseScope ps(ctx, GP_PHASE_UPDATE, 1);
            GP_CUDA(ctx, gp::launch_gemm_update(mb, J, ctx->stream));
            J += 1;
        }
    }
    return GP_OK;
}

// Solves with refinement and the likelihood for the factored instances: the
// backward substitution x = L^-T [a b] of the forward solve's results, then
// up to refine_iters refinement steps (residual and forward correction; the
// correction's backward substitution only when another step follows), each
// closed by k_refine_check, which forms the sums of eq. 3 and stops the
// candidates whose -2logL no further step can improve (k_mixed.cu).
int run_mixed_solve(gp_ctx* ctx, const gp::MixedBatch& mb, double* nll, double* mu, double* sigma2,
                    double* logdet, int* status) {
    const int sp = gp::subst_launches(mb.nt);
    const int steps = ctx->opt.refine_iters;
    PhaseScope ps(ctx, GP_PHASE_SOLVE, (mb.fwd ? 0 : 1 + sp) + 1 + sp + 1 + steps * (sp + 3) +
                                           (steps > 1 ? (steps - 1) * sp : 0) + 1);
    // with mb.fwd the factorisation has already done the first forward solve
    if (!mb.fwd) GP_CUDA(ctx, gp::launch_df_forward(mb, 0, 1, ctx->stream));
    GP_CUDA(ctx, gp::launch_keep_forward(mb, ctx->stream));
    GP_CUDA(ctx, gp::launch_df_backward(mb, 0, -1, ctx->stream));
    GP_CUDA(ctx, gp::launch_refine_check(mb, 0, ctx->stream));
    for (int k = 1; k <= steps; ++k) {
        if (k > 1) GP_CUDA(ctx, gp::launch_df_backward(mb, 2, 0, ctx->stream));   // x += L^-T z
        GP_CUDA(ctx, gp::launch_df_residual(mb, ctx->stream));
        GP_CUDA(ctx, gp::launch_df_forward(mb, 2, 0, ctx->stream));
        GP_CUDA(ctx, gp::launch_refine_check(mb, k, ctx->stream));
    }
    GP_CUDA(ctx, gp::launch_df_finalize(mb, nll, mu, sigma2, logdet, status, ctx->stream));
    return GP_OK;
}

// 1-norm condition estimates of the factored instances (k_cond.cu): ||R||_1,
// then Hager's iteration, all instances in step, at most five rounds.
int run_mixed_cond(gp_ctx* ctx, const gp::MixedBatch& mb, double* cond) {
    constexpr int kRounds = 5;
    const int sp = gp::subst_launches(mb.nt);
    PhaseScope ps(ctx, GP_PHASE_SOLVE, 3 + kRounds * (1 + 2 * sp) + (kRounds - 1) * (1 + 2 * sp));
    GP_CUDA(ctx, gp::launch_norm1(mb, ctx->stream));
    GP_CUDA(ctx, gp::launch_hager(mb, 0, nullptr, ctx->stream));
    for (int it = 0; it < kRounds; ++it) {
        GP_CUDA(ctx, gp::launch_df_forward(mb, 5, 0, ctx->stream));      // z = R^-1 sign(y)
        GP_CUDA(ctx, gp::launch_df_backward(mb, 5, -1, ctx->stream));
        GP_CUDA(ctx, gp::launch_hager(mb, 2, nullptr, ctx->stream));
        if (it + 1 == kRounds) break;
        GP_CUDA(ctx, gp::launch_df_forward(mb, 5, 0, ctx->stream));      // y = R^-1 e_j
        GP_CUDA(ctx, gp::launch_df_backward(mb, 5, -1, ctx->stream));
        GP_CUDA(ctx, gp::launch_hager(mb, 1, nullptr, ctx->stream));
    }
    GP_CUDA(ctx, gp::launch_hager(mb, 3, cond, ctx->stream));
    return GP_OK;
}

// Where the last chunk of a batched call left its candidates in the
// workspace: gp_fit_batch builds a model from one of them.
struct LastChunk {
    int c0 = 0, cnt = 0;
    bool split = false;
    gp::MixedBatch mb{};          // split path
    double* A = nullptr;          // FP64 path: factors, [a | b] solve vectors, records
    double* Z = nullptr;
    gp::InstState* st = nullptr;
    size_t a_stride = 0, z_stride = 0;
};

int mixed_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                    const double* theta, double p, double delta, double* nll, double* mu,
                    double* sigma2, double* logdet, int* status, int slices, double* cond,
                    LastChunk* last = nullptr) {
    const MixedSizes z = mixed_sizes(n, slices);
    Chunking ch;
    if (!chunk_batch(ctx->opt, ctx->budget, ctx->models_bytes, z.per, kMixedTail, T, &ch))
        return fail(ctx, GP_ENOMEM, "one instance (%zu bytes) exceeds the HBM budget", z.per);
    const int Tc = ch.Tc;
    int rc = ensure_ws(ctx, ch.bytes);
    if (rc) return rc;
    for (int c0 = 0; c0 < T; c0 += Tc) {
        const int cnt = (T - c0 < Tc) ? (T - c0) : Tc;
        gp::MixedBatch mb = mixed_layout(ctx, n, cnt, y, (char*)ctx->ws, z, Tc, slices);
        rc = run_mixed_factor(ctx, mb, d, x, theta + (size_t)c0 * d, p, delta);
        if (rc) return rc;
        rc = run_mixed_solve(ctx, mb, nll + c0, mu + c0, sigma2 + c0, logdet ? logdet + c0 : nullptr,
                             status + c0);
        if (rc) return rc;
        if (cond) {
            rc = run_mixed_cond(ctx, mb, cond + c0);
            if (rc) return rc;
        }
        if (last) {
            last->c0 = c0;
            last->cnt = cnt;
            last->split = true;
            last->mb = mb;
        }
    }
    return GP_OK;
}

// -2logL in IEEE double for T candidates (batches sized by the budget).
int fp64_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                   const double* theta, double p, double delta, double* nll, double* mu_hat,
                   double* sigma2_hat, double* logdet, int* status, LastChunk* last = nullptr) {
    const int nt = gp::num_tiles(n);
    const size_t per = per_instance_bytes_f64(n);
    Chunking ch;
    if (!chunk_batch(ctx->opt, ctx->budget, ctx->models_bytes, per, 0, T, &ch))
        return fail(ctx, GP_ENOMEM, "one instance (%zu bytes) exceeds the HBM budget", per);
    const int Tc = ch.Tc;
    int rc = ensure_ws(ctx, ch.bytes);
    if (rc) return rc;
    char* base = (char*)ctx->ws;
    const size_t a_bytes = align256(gp::packed_elems(n) * sizeof(double));
    const size_t z_bytes = align256((size_t)2 * nt * GP_NB * sizeof(double));
    double* A = (double*)base;
    double* Z = (double*)(base + a_bytes * Tc);
    gp::InstState* st = (gp::InstState*)(base + (a_bytes + z_bytes) * Tc);
    for (int c0 = 0; c0 < T; c0 += Tc) {
        const int cnt = (T - c0 < Tc) ? (T - c0) : Tc;
        gp::Batch b{};
        b.n = n; b.d = d; b.nt = nt; b.count = cnt; b.corr = ctx->opt.correlation;
        b.p = p; b.delta = delta; b.x = x; b.y = y; b.theta = theta + (size_t)c0 * d;
        b.A = A; b.inst_stride = a_bytes / sizeof(double); b.st = st;
        {
            PhaseScope ps(ctx, GP_PHASE_ASSEMBLE, 2);
            GP_CUDA(ctx, gp::launch_validate_theta(b, ctx->stream));
            GP_CUDA(ctx, gp::launch_assemble_tiles(b, ctx->stream));
        }
        rc = run_factor_f64(ctx, b);
        if (rc) return rc;
        const size_t zs = z_bytes / sizeof(double);
        PhaseScope ps(ctx, GP_PHASE_SOLVE, gp::solve_f64_launches(b.nt, false) + 1);
        GP_CUDA(ctx, gp::launch_forward_solve(b, Z, zs, ctx->stream));
        GP_CUDA(ctx, gp::launch_finalize(b, Z, zs, nll + c0, mu_hat + c0, sigma2_hat + c0,
                                         logdet ? logdet + c0 : nullptr, status + c0, ctx->stream));
        if (last) {
            last->c0 = c0;
            last->cnt = cnt;
            last->split = false;
            last->A = A;
            last->Z = Z;
            last->st = st;
            last->a_stride = a_bytes / sizeof(double);
            last->z_stride = zs;
        }
    }
    return GP_OK;
}

// Error of -2logL per unit of cond_1(R) allowed for a split factorisation
// with s slices in the trailing updates: 2^-(8 s + 6).  The largest ratio
// measured on the 256 candidates of the n = 4000 benchmark batch (cond_1
// from 2e7 to 4e11) was 9.5e-11 with 3 slices and 5.4e-16 with 5; the
// bound leaves a margin of 10 or more.
double split_error_per_cond(int s) { return std::ldexp(1.0, -(8 * s + 6)); }

// GP_AUTO's routing buffers (allocated beside the workspace): compacted theta
// and the outputs of a re-evaluated subset, indices, and cond / prec_used when
// the caller passed none.
size_t auto_staging_bytes(int T, int d) {
    const size_t bT = align256((size_t)T * sizeof(double));
    const size_t bI = align256((size_t)T * sizeof(int));
    return align256((size_t)T * d * sizeof(double)) + 6 * bT + 4 * bI;
}

// GP_AUTO: route every candidate to the cheapest arithmetic whose bound
// meets auto_tol (GP_FP32, then GP_MIXED, then GP_FP64); see gp.h.
int auto_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                   const double* theta, double p, double delta, double* nll, double* mu,
                   double* sigma2, double* logdet, int* status, double* cond, int* prec_used) {
    const double tol = ctx->opt.auto_tol;
    const size_t bT = align256((size_t)T * sizeof(double));
    const size_t bI = align256((size_t)T * sizeof(int));
    const size_t total = auto_staging_bytes(T, d);
    void* dev = nullptr;
    if (cudaMallocAsync(&dev, total, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GP_ENOMEM, "GP_AUTO staging allocation of %zu bytes failed", total);
    }
    char* c = (char*)dev;
    double* th_c = (double*)c; c += align256((size_t)T * d * sizeof(double));
    double* nll_c = (double*)c; c += bT;
    double* mu_c = (double*)c; c += bT;
    double* s2_c = (double*)c; c += bT;
    double* ld_c = (double*)c; c += bT;
    double* cond_c = (double*)c; c += bT;
    double* cond_all = cond ? cond : (double*)c; c += bT;
    int* st_c = (int*)c; c += bI;
    int* idx_d = (int*)c; c += bI;
    int* pu = prec_used ? prec_used : (int*)c; c += bI;
    auto done = [&](int rc) {
        cudaFreeAsync(dev, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (rc == GP_OK && e != cudaSuccess) return fail(ctx, GP_ECUDA, "GP_AUTO: %s", cudaGetErrorString(e));
        return rc;
    };
    int rc = mixed_nll_batch(ctx, n, d, x, y, T, theta, p, delta, nll, mu, sigma2, logdet, status, 3, cond_all);
    if (rc) return done(rc);
    if (gp::launch_fill_int(pu, T, GP_FP32, ctx->stream) != cudaSuccess)
        return done(fail(ctx, GP_ECUDA, "GP_AUTO: fill launch failed"));
    std::vector<int> hst(T);
    std::vector<double> hc(T), hth((size_t)T * d);
    if (cudaMemcpyAsync(hst.data(), status, (size_t)T * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) ||
        cudaMemcpyAsync(hc.data(), cond_all, (size_t)T * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) ||
        cudaMemcpyAsync(hth.data(), theta, (size_t)T * d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) ||
        cudaStreamSynchronize(ctx->stream))
        return done(fail(ctx, GP_ECUDA, "GP_AUTO: reading the estimates failed"));
    // a candidate moves on unless it factored and its bound meets the tolerance
    auto needs_more = [&](int st, double cnd, int s) {
        if (st == GP_EINVAL || st == GP_ETIMEOUT) return false;
        if (st != GP_OK) return true;
        return !(cnd * split_error_per_cond(s) <= tol);
    };
    std::vector<int> idx;
    for (int t = 0; t < T; ++t)
        if (needs_more(hst[t], hc[t], 3)) idx.push_back(t);
    for (int tier = 0; tier < 2 && !idx.empty(); ++tier) {
        const int m = (int)idx.size();
        const int prec = tier == 0 ? GP_MIXED : GP_FP64;
        std::vector<double> thc((size_t)m * d);
        for (int i = 0; i < m; ++i)
            std::memcpy(&thc[(size_t)i * d], &hth[(size_t)idx[i] * d], d * sizeof(double));
        if (cudaMemcpyAsync(th_c, thc.data(), thc.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) ||
            cudaMemcpyAsync(idx_d, idx.data(), (size_t)m * sizeof(int), cudaMemcpyHostToDevice, ctx->stream))
            return done(fail(ctx, GP_ECUDA, "GP_AUTO: staging copy failed"));
        if (prec == GP_MIXED)
            rc = mixed_nll_batch(ctx, n, d, x, y, m, th_c, p, delta, nll_c, mu_c, s2_c, ld_c, st_c,
                                 ctx->opt.slices, cond_c);
        else
            rc = fp64_nll_batch(ctx, n, d, x, y, m, th_c, p, delta, nll_c, mu_c, s2_c, ld_c, st_c);
        if (rc) return done(rc);
        cudaStream_t s = ctx->stream;
        if (gp::launch_scatter(m, idx_d, nll_c, nll, s) || gp::launch_scatter(m, idx_d, mu_c, mu, s) ||
            gp::launch_scatter(m, idx_d, s2_c, sigma2, s) ||
            (logdet && gp::launch_scatter(m, idx_d, ld_c, logdet, s)) ||
            gp::launch_scatter_int(m, idx_d, st_c, status, s) ||
            (prec == GP_MIXED && gp::launch_scatter(m, idx_d, cond_c, cond_all, s)) ||
            gp::launch_fill_int(st_c, m, prec, s) || gp::launch_scatter_int(m, idx_d, st_c, pu, s))
            return done(fail(ctx, GP_ECUDA, "GP_AUTO: scatter launch failed"));
        if (prec == GP_FP64) break;
        // statuses of the subset are in `status` now; the estimates in cond_c
        std::vector<int> sst(m);
        std::vector<double> sc(m);
        if (cudaMemcpyAsync(sc.data(), cond_c, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, s) ||
            cudaMemcpyAsync(hst.data(), status, (size_t)T * sizeof(int), cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s))
            return done(fail(ctx, GP_ECUDA, "GP_AUTO: reading the estimates failed"));
        std::vector<int> next;
        for (int i = 0; i < m; ++i)
            if (needs_more(hst[idx[i]], sc[i], ctx->opt.slices)) next.push_back(idx[i]);
        idx.swap(next);
    }
    return done(GP_OK);
}

// Workspace per candidate of gp_nll_grad_batch: the factor, L^-1, R^-1,
// [a | w], its record, tile partial sums, and mu / sigma2 / log|R| (which
// the caller does not ask for).
struct GradSizes {
    size_t a, z, st, part, sc, per;
};

GradSizes grad_sizes(int n, int d) {
    const int nt = gp::num_tiles(n);
    GradSizes g;
    g.a = align256(gp::packed_elems(n) * sizeof(double));
    g.z = align256((size_t)2 * nt * GP_NB * sizeof(double));
    g.st = align256(sizeof(gp::InstState));
    g.part = align256((size_t)gp::packed_tiles(nt) * d * sizeof(double));
    g.sc = align256(3 * sizeof(double));
    g.per = 3 * g.a + g.z + g.st + g.part + g.sc;
    return g;
}

// One allocation per model: the factor, [a | w], x, theta, the scalars, the
// status and the instance record.
struct ModelSizes {
    size_t L, Z, x, th, sc, stat, st, total;
};

ModelSizes model_sizes(int n, int d) {
    const int nt = gp::num_tiles(n);
    ModelSizes m;
    m.L = align256(gp::packed_elems(n) * sizeof(double));
    m.Z = align256((size_t)2 * nt * GP_NB * sizeof(double));
    m.x = align256((size_t)n * d * sizeof(double));
    m.th = align256((size_t)d * sizeof(double));
    m.sc = align256(8 * sizeof(double));
    m.stat = align256(sizeof(int));
    m.st = align256(sizeof(gp::InstState));
    m.total = m.L + m.Z + m.x + m.th + m.sc + m.stat + m.st;
    return m;
}

// Test points one gp_predict call takes: the launch arithmetic (point
// indices, CTA counts rounded up) stays in int with room to spare.
constexpr int kMaxPredictPoints = 1 << 30;

// Launch shape and workspace of gp_predict: test points per CTA, CTAs in
// all, CTAs per launch (at most four waves, fewer when their scratch would
// not fit `avail`), and the scratch those CTAs take when variances are asked
// for (else a token 256 bytes).
struct PredictShape {
    int ppc, blocks, chunk;
    size_t per_cta, bytes;
};

PredictShape predict_shape(int nt, int N, int sms, size_t avail, bool variances) {
    PredictShape s;
    s.ppc = gp::predict_points_per_cta(N, sms);
    s.per_cta = gp::predict_work_per_cta(nt, s.ppc);
    s.blocks = (N + s.ppc - 1) / s.ppc;
    s.chunk = s.blocks < 4 * sms ? s.blocks : 4 * sms;
    while (s.chunk > 1 && s.per_cta * s.chunk > avail) s.chunk /= 2;
    s.bytes = variances ? s.per_cta * s.chunk : 256;
    return s;
}

// Workspace of gp_predict on the tensor-core path (predict_tc): with
// variances the slice tables of the model, then an error flag, the r
// values (with variances) and partial means of a chunk of 128-point
// blocks, and per CTA of the tensor-core pass the slices of V and of C_J.
// A chunk is one wave of that pass (one block per SM; four waves' partial
// means without variances), fewer blocks when the budget is short.  With
// variances and more than one chunk, the blocks past the last whole chunk
// (the remainder, rem < chunk) get their own r values and CTA slices: their
// pass runs on the context's second stream while the main stream forms the
// r values of the whole chunks, one chunk ahead of its passes in a second
// slot, so that the remainder's partial wave is not a round of its own.
struct VarPlan {
    int blocks, chunk, grid, rem, slots;
    size_t tables, per_block, per_cta, bytes;
};

VarPlan var_plan(int nt, int N, int sms, size_t avail, bool variances) {
    VarPlan v;
    v.blocks = (N + GP_NB - 1) / GP_NB;
    v.tables = variances ? align256(gp::var_table_bytes(nt)) : 0;
    v.per_block = (variances ? gp::var_rx_bytes(nt) : 0) + gp::var_mp_bytes(nt);
    v.per_cta = variances ? gp::var_cta_bytes(nt) : 0;
    auto shape = [&](int c, int& rem, int& slots) {
        rem = (variances && v.blocks > c) ? v.blocks % c : 0;
        slots = (rem > 0 && (v.blocks - rem) / c >= 2) ? 2 : 1;
    };
    auto total = [&](int c) {
        int rem, slots;
        shape(c, rem, slots);
        return v.tables + 256 + gp::var_rhs_tab_bytes() + (size_t)slots * c * v.per_block + (size_t)(c < sms ? c : sms) * v.per_cta +
               (size_t)rem * (v.per_block + v.per_cta);
    };
    const int cap = variances ? sms : 4 * sms;
    v.chunk = v.blocks < cap ? v.blocks : cap;
    while (v.chunk > 1 && total(v.chunk) > avail) v.chunk -= (v.chunk / 4 > 1 ? v.chunk / 4 : 1);
    v.grid = v.chunk < sms ? v.chunk : sms;
    shape(v.chunk, v.rem, v.slots);
    v.bytes = total(v.chunk);
    return v;
}

// A model's device memory (one allocation, ModelSizes), counted against the
// context's budget next to its workspace.
int model_alloc(gp_ctx* ctx, int n, int d, double p, double delta, int prec, gp_model** out) {
    *out = nullptr;
    const ModelSizes ms = model_sizes(n, d);
    if (ms.total + ctx->models_bytes + ctx->ws_bytes > ctx->budget)
        return fail(ctx, GP_ENOMEM, "model of %zu bytes exceeds the HBM budget", ms.total);
    gp_model* m = new gp_model();
    m->ctx = ctx; m->n = n; m->d = d; m->nt = gp::num_tiles(n); m->p = p; m->delta = delta; m->prec = prec;
    m->corr = ctx->opt.correlation;
    if (cudaMallocAsync(&m->mem, ms.total, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return fail(ctx, GP_ENOMEM, "allocation of %zu bytes for the model failed", ms.total);
    }
    m->bytes = ms.total;
    char* c = (char*)m->mem;
    m->L = (double*)c; c += ms.L;
    m->Z = (double*)c; c += ms.Z;
    m->x = (double*)c; c += ms.x;
    m->theta = (double*)c; c += ms.th;
    m->scalars = (double*)c; c += ms.sc;
    m->status = (int*)c; c += ms.stat;
    m->st = (gp::InstState*)c;
    ctx->models_bytes += ms.total;
    *out = m;
    return GP_OK;
}

// Release a model that was never handed out (a failed fit).
int model_discard(gp_ctx* ctx, gp_model* m, int code) {
    cudaFreeAsync(m->mem, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    ctx->models_bytes -= m->bytes;
    delete m;
    return code;
}

// The kriging kernel reads the factor, [a | w] and x as double-float pairs:
// convert what is still in double, copy x and theta in, read the status and
// the scalars back, and hand the model out (GP_OK or GP_EDEGENERATE).
int model_finish(gp_ctx* ctx, gp_model* m, const double* x, const double* theta, bool df_factor,
                 gp_model** out) {
    const size_t npad = (size_t)m->nt * GP_NB;
    if (cudaMemcpyAsync(m->x, x, (size_t)m->n * m->d * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream) ||
        cudaMemcpyAsync(m->theta, theta, (size_t)m->d * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream) ||
        (!df_factor && gp::launch_to_df_inplace(m->L, gp::packed_elems(m->n), ctx->stream)) ||
        (!df_factor && gp::launch_to_df_inplace(m->Z, 2 * npad, ctx->stream)) ||
        gp::launch_to_df_inplace(m->x, (size_t)m->n * m->d, ctx->stream))
        return model_discard(ctx, m, fail(ctx, GP_ECUDA, "model conversion failed"));
    int hstatus = 0;
    cudaError_t e = cudaMemcpyAsync(&hstatus, m->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->host_scalars, m->scalars, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return model_discard(ctx, m, fail(ctx, GP_ECUDA, "fit: %s", cudaGetErrorString(e)));
    if (hstatus != GP_OK && hstatus != GP_EDEGENERATE)
        return model_discard(ctx, m, fail(ctx, hstatus, "fit failed with status %d", hstatus));
    ctx->models.push_back(m);
    *out = m;
    return hstatus;
}

// Model of candidate t (0-based inside the last chunk) of an FP64 batch: its
// factor and [a | b] copied out of the workspace, then w = L^-T (b - mu a)
// as gp_fit forms it.
int model_from_fp64(gp_ctx* ctx, gp_model* m, const LastChunk& lc, int t, const double* nll, const double* mu, const double* sigma2, const double* logdet,
                    const int* status) {
    const size_t npad = (size_t)m->nt * GP_NB;
    cudaStream_t s = ctx->stream;
    if (cudaMemcpyAsync(m->L, lc.A + (size_t)t * lc.a_stride, gp::packed_elems(m->n) * sizeof(double),
                        cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(m->Z, lc.Z + (size_t)t * lc.z_stride, 2 * npad * sizeof(double), cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(m->st, lc.st + t, sizeof(gp::InstState), cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(m->scalars + 0, nll, sizeof(double), cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(m->scalars + 1, mu, sizeof(double), cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync(m->scalars + 2, sigma2, sizeof(double), cudaMemcpyDeviceToDevice, s) ||
        (logdet && cudaMemcpyAsync(m->scalars + 3, logdet, sizeof(double), cudaMemcpyDeviceToDevice, s)) ||
        cudaMemcpyAsync(m->status, status, sizeof(int), cudaMemcpyDeviceToDevice, s))
        return fail(ctx, GP_ECUDA, "copy of the factor into the model failed");
    gp::Batch b{};
    b.n = m->n; b.nt = m->nt; b.count = 1; b.st = m->st; b.A = m->L; b.inst_stride = gp::packed_elems(m->n);
    PhaseScope ps(ctx, GP_PHASE_SOLVE, 1 + gp::solve_f64_launches(b.nt, true));
    if (gp::launch_fit_finish(b, m->Z, 2 * npad, m->scalars, s) ||
        gp::launch_backward_solve(b, m->Z, 2 * npad, 1, s))
        return fail(ctx, GP_ECUDA, "solve launch failed");
    return GP_OK;
}

// The one-candidate view of candidate t of a split batch.
gp::MixedBatch mixed_view(const gp::MixedBatch& mb, int t) {
    gp::MixedBatch v = mb;
    v.count = 1;
    v.A += (size_t)t * mb.inst_stride;
    v.Rc += (size_t)t * mb.inst_stride;
    v.PS += (size_t)t * mb.ps_stride;
    v.PE += (size_t)t * mb.pe_stride;
    v.WS += (size_t)t * mb.ws_stride;
    v.WE += (size_t)t * mb.we_stride;
    v.PF += (size_t)t * mb.pf_stride;
    v.FE += (size_t)t * mb.fe_stride;
    v.WT += (size_t)t * mb.wt_stride;
    v.WR += (size_t)t * mb.wt_stride;
    v.Z += (size_t)t * mb.z_stride;
    v.RP += (size_t)t * mb.rp_stride;
    v.SC += (size_t)t * mb.sc_stride;
    v.st += t;
    return v;
}

// Model of candidate t of a split batch: its double-float factor as it is,
// the last refinement correction applied (x += L^-T z, as a further step
// would), then [a | w] with w = x_y - mu x_1 (k_split_model).
int model_from_split(gp_ctx* ctx, gp_model* m, const LastChunk& lc, int t, const double* nll,
                     const int* status) {
    const gp::MixedBatch v = mixed_view(lc.mb, t);
    cudaStream_t s = ctx->stream;
    if (cudaMemcpyAsync(m->L, v.A, gp::packed_elems(m->n) * sizeof(float2), cudaMemcpyDeviceToDevice, s) ||
        cudaMemsetAsync(reinterpret_cast<char*>(v.st) + offsetof(gp::InstState, refine_done), 0, sizeof(int), s))
        return fail(ctx, GP_ECUDA, "copy of the factor into the model failed");
    const int sp = gp::subst_launches(v.nt);
    PhaseScope ps(ctx, GP_PHASE_SOLVE, (ctx->opt.refine_iters > 0 ? sp : 0) + 1);
    if ((ctx->opt.refine_iters > 0 && gp::launch_df_backward(v, 2, 0, s)) ||
        gp::launch_split_model(v, reinterpret_cast<float2*>(m->Z), m->scalars, nll, status, m->status, s))
        return fail(ctx, GP_ECUDA, "model launch failed");
    return GP_OK;
}

}  // namespace

namespace gp {

// Accessors for the entry points defined in other translation units.
int ctx_fail(gp_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

int ctx_device(const gp_ctx* ctx) { return ctx->device; }

int ctx_check_common(gp_ctx* ctx, int n, int d, double p, double delta) {
    return check_common(ctx, n, d, p, delta);
}

int ctx_correlation(const gp_ctx* ctx) { return ctx->opt.correlation; }

cudaStream_t ctx_stream(const gp_ctx* ctx) { return ctx->stream; }

}  // namespace gp

namespace {

// gp_predict on the tensor-core path: the tables of the model (with
// variances), then per chunk of point blocks r and the partial means, yhat,
// and the tensor-core pass for s2 (k_var_tc.cu).
int predict_tensor(gp_ctx* ctx, const gp_model* m, int N, const double* xstar, double* yhat, double* s2) {
    const bool var = s2 != nullptr;
    const int nt = m->nt, npad = nt * GP_NB;
    const size_t avail = ctx->budget > ctx->models_bytes ? ctx->budget - ctx->models_bytes : 0;
    const VarPlan v = var_plan(nt, N, ctx->sms, avail, var);
    if (var && v.bytes > ctx->ws_bytes && v.bytes + ctx->models_bytes > ctx->budget)
        return fail(ctx, GP_ENOMEM,
                    "the tensor-core variance needs %zu bytes of workspace (the factor's slices and one "
                    "128-point block), beyond the HBM budget (%zu, %zu held by models): set predict_tc = 0",
                    v.bytes, ctx->budget, ctx->models_bytes);
    int rc = ensure_ws(ctx, v.bytes);
    if (rc) return rc;
    if (v.rem > 0 && (rc = ensure_aux(ctx))) return rc;
    // the workspace, in the order var_plan counts it
    char* c = static_cast<char*>(ctx->ws);
    gp::VarCall call{};
    if (var) call.t = gp::var_tables_at(c, nt);
    c += v.tables;
    call.err = reinterpret_cast<int*>(c);
    c += 256;
    call.rtab = reinterpret_cast<float2*>(c);
    c += gp::var_rhs_tab_bytes();
    const size_t rx = var ? gp::var_rx_bytes(nt) : 0, mp = gp::var_mp_bytes(nt);
    const size_t vs = var ? gp::var_vs_bytes(nt) : 0, cs = var ? gp::var_cta_bytes(nt) - gp::var_vs_bytes(nt) : 0;
    float2* RX[2];
    float2* MP[2];
    for (int q = 0; q < v.slots; ++q, c += (size_t)v.chunk * rx) RX[q] = reinterpret_cast<float2*>(c);
    for (int q = 0; q < v.slots; ++q, c += (size_t)v.chunk * mp) MP[q] = reinterpret_cast<float2*>(c);
    if (v.slots == 1) {
        RX[1] = RX[0];
        MP[1] = MP[0];
    }
    __nv_bfloat16* VS = reinterpret_cast<__nv_bfloat16*>(c);
    c += (size_t)v.grid * vs;
    __nv_bfloat16* CS = reinterpret_cast<__nv_bfloat16*>(c);
    c += (size_t)v.grid * cs;
    float2* RXr = reinterpret_cast<float2*>(c);
    c += (size_t)v.rem * rx;
    float2* MPr = reinterpret_cast<float2*>(c);
    c += (size_t)v.rem * mp;
    __nv_bfloat16* VSr = reinterpret_cast<__nv_bfloat16*>(c);
    c += (size_t)v.rem * vs;
    __nv_bfloat16* CSr = reinterpret_cast<__nv_bfloat16*>(c);
    call.n = m->n; call.d = m->d; call.nt = nt; call.N = N; call.corr = m->corr;
    call.p = m->p;
    call.c0 = ctx->opt.nugget_in_var ? 1.0 + m->delta : 1.0;
    // |v_i|^2 <= v'v <= 1 + delta: the V slices' exponent E with
    // sqrt(1 + delta) < 2^E
    int ev = 0;
    std::frexp(std::sqrt(1.0 + m->delta) * (1.0 + 0x1p-20), &ev);
    call.ev = ev;
    call.inject_timeout = (ctx->opt.inject_timeout & 2) != 0;
    const float2* Zdf = reinterpret_cast<const float2*>(m->Z);
    call.x = reinterpret_cast<const float2*>(m->x);
    call.theta = m->theta; call.w = Zdf + npad; call.a = Zdf; call.sc = m->scalars;
    call.xs = xstar; call.yhat = yhat; call.s2 = s2;
    PhaseScope ps(ctx, GP_PHASE_PREDICT, 0);
    int k = 0;
    {
        const cudaError_t e = gp::launch_var_rhs_tables(call, ctx->stream, &k);
        ps.kernels += k;
        GP_CUDA(ctx, e);
    }
    auto points = [&](int b0, int nb, float2* rxp, float2* mpp) -> int {
        const cudaError_t e = gp::launch_var_points(call, b0 * GP_NB, nb, var ? rxp : nullptr, mpp, ctx->stream, &k);
        ps.kernels += k;
        GP_CUDA(ctx, e);
        return GP_OK;
    };
    auto pass = [&](int b0, int nb, const float2* rxp, __nv_bfloat16* vsp, __nv_bfloat16* csp, int grid,
                    cudaStream_t st) -> int {
        const cudaError_t e = gp::launch_var_pass(call, b0 * GP_NB, nb, rxp, vsp, csp, grid, st, &k);
        ps.kernels += k;
        if (e == cudaErrorNotSupported)
            return fail(ctx, GP_ENOTSUP, "the tensor-core variance kernel was built with too few registers "
                                         "for its register split: set predict_tc = 0");
        GP_CUDA(ctx, e);
        return GP_OK;
    };
    if (!var) {
        for (int b0 = 0; b0 < v.blocks; b0 += v.chunk)
            if ((rc = points(b0, v.blocks - b0 < v.chunk ? v.blocks - b0 : v.chunk, nullptr, MP[0]))) return rc;
        return GP_OK;
    }
    {
        const cudaError_t e = gp::launch_var_tables(reinterpret_cast<const float2*>(m->L), nt, call.t, ctx->stream, &k);
        ps.kernels += k;
        GP_CUDA(ctx, e);
    }
    const int full = v.blocks - v.rem;             // whole chunks
    const int chunks = (full + v.chunk - 1) / v.chunk;
    if (v.rem > 0) {
        // the remainder's r, then its pass on the second stream
        if ((rc = points(full, v.rem, RXr, MPr))) return rc;
        GP_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
        GP_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
        if ((rc = pass(full, v.rem, RXr, VSr, CSr, v.rem, ctx->aux))) return rc;
        GP_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->aux));
    }
    // whole chunks: with two slots the r of chunk q + 1 is formed before the
    // pass of chunk q (in-order on the main stream, so a slot is rewritten
    // only after the pass that read it)
    for (int q = 0; q < chunks; ++q) {
        const int b0 = q * v.chunk, nb = full - b0 < v.chunk ? full - b0 : v.chunk;
        if (v.slots == 1 || q == 0)
            if ((rc = points(b0, nb, RX[q & 1], MP[q & 1]))) return rc;
        if (v.slots == 2 && q + 1 < chunks) {
            const int b1 = b0 + v.chunk;
            if ((rc = points(b1, full - b1 < v.chunk ? full - b1 : v.chunk, RX[(q + 1) & 1], MP[(q + 1) & 1])))
                return rc;
        }
        if ((rc = pass(b0, nb, RX[q & 1], VS, CS, v.grid, ctx->stream))) return rc;
    }
    if (v.rem > 0) GP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    return GP_OK;
}

}  // namespace

extern "C" {

void gp_default_options(gp_options* opt) {
    if (!opt) return;
    opt->slices = 5;
    opt->panel_slices = GP_PANEL_SLICES;
    opt->refine_iters = 1;
    opt->nugget_in_var = 1;
    opt->max_batch = 0;
    opt->update_groups = 4;
    opt->inject_timeout = 0;
    opt->fuse_panels = 1;
    opt->auto_tol = 1e-6;
    opt->update_tile = 128;
    opt->assemble_cols = 16;
    opt->correlation = GP_CORR_POWEXP;
    opt->predict_tc = 1;
}

int gp_create(gp_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
    if (!out) return GP_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return GP_ECUDA;
    }
    if (device < 0 || device >= count) return GP_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GP_ECUDA;
    gp_ctx* ctx = new gp_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    gp_default_options(&ctx->opt);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete ctx;
        return GP_ECUDA;
    }
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (free_b / 4) * 3;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
        ctx->sms = sms;
    else
        cudaGetLastError();
    *out = ctx;
    return GP_OK;
}

void gp_destroy(gp_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    // models outlive their context safely: they are detached and freed on
    // their own later (synchronously)
    for (gp_model* m : ctx->models) m->ctx = nullptr;
    for (gp_plan* q : ctx->plans) q->ctx = nullptr;
    if (ctx->ws) cudaFreeAsync(ctx->ws, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    for (auto& o : ctx->ev_open) {
        cudaEventDestroy(o.second.first);
        cudaEventDestroy(o.second.second);
    }
    if (ctx->aux) {
        cudaStreamSynchronize(ctx->aux);
        cudaStreamDestroy(ctx->aux);
        cudaEventDestroy(ctx->ev_fork);
        cudaEventDestroy(ctx->ev_join);
    }
    if (ctx->la) {
        cudaStreamSynchronize(ctx->la);
        cudaStreamDestroy(ctx->la);
        cudaEventDestroy(ctx->ev_la0);
        cudaEventDestroy(ctx->ev_la1);
    }
    delete ctx;
}

const char* gp_last_error(const gp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int gp_set_stream(gp_ctx* ctx, void* stream) {
    if (!ctx) return GP_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return GP_OK;
}

int gp_set_options(gp_ctx* ctx, const gp_options* opt) {
    if (!ctx || !opt) return GP_EINVAL;
    if (opt->slices < 2 || opt->slices > 6)
        return fail(ctx, GP_EINVAL, "slices = %d outside [2, 6]", opt->slices);
    if (opt->panel_slices != GP_PANEL_SLICES)
        return fail(ctx, GP_EINVAL, "panel_slices is fixed at %d (GP_PANEL_SLICES, a compile-time constant)", GP_PANEL_SLICES);
    if (opt->refine_iters < 0 || opt->refine_iters > 10)
        return fail(ctx, GP_EINVAL, "refine_iters = %d outside [0, 10]", opt->refine_iters);
    if (opt->max_batch < 0) return fail(ctx, GP_EINVAL, "max_batch must be >= 0");
    if (opt->update_groups != 3 && opt->update_groups != 4 && opt->update_groups != 7)
        return fail(ctx, GP_EINVAL, "update_groups must be 3, 4 or 7");
    if (opt->fuse_panels && opt->update_groups != 4)
        return fail(ctx, GP_EINVAL, "fuse_panels needs update_groups = 4");
    if (!(opt->auto_tol > 0.0) || !std::isfinite(opt->auto_tol))
        return fail(ctx, GP_EINVAL, "auto_tol = %g must be positive and finite", opt->auto_tol);
    if (opt->update_tile != 128 && opt->update_tile != 64)
        return fail(ctx, GP_EINVAL, "update_tile must be 128 or 64");
    if (opt->update_tile == 64 && opt->update_groups != 4)
        return fail(ctx, GP_EINVAL, "update_tile = 64 needs update_groups = 4");
    if (opt->assemble_cols != 16 && opt->assemble_cols != 32)
        return fail(ctx, GP_EINVAL, "assemble_cols must be 16 or 32");
    if (opt->correlation < GP_CORR_POWEXP || opt->correlation > GP_CORR_MATERN52)
        return fail(ctx, GP_EINVAL, "correlation = %d is not a gp_correlation", opt->correlation);
    if (opt->predict_tc != 0 && opt->predict_tc != 1) return fail(ctx, GP_EINVAL, "predict_tc must be 0 or 1");
    if (opt->inject_timeout < 0 || opt->inject_timeout > 3)
        return fail(ctx, GP_EINVAL, "inject_timeout = %d outside [0, 3]", opt->inject_timeout);
    ctx->opt = *opt;
    return GP_OK;
}

int gp_get_options(const gp_ctx* ctx, gp_options* opt) {
    if (!ctx || !opt) return GP_EINVAL;
    *opt = ctx->opt;
    return GP_OK;
}

size_t gp_workspace_bytes(const gp_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

int gp_set_timing(gp_ctx* ctx, int on) {
    if (!ctx) return GP_EINVAL;
    ctx->timing = (on != 0);
    return GP_OK;
}

int gp_phase_times(gp_ctx* ctx, double* ms, long long* launches, int nphases) {
    if (!ctx || nphases < 0) return GP_EINVAL;
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& o : ctx->ev_open) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, o.second.first, o.second.second) == cudaSuccess)
            ctx->phase_ms[o.first] += t;
        ctx->ev_pool.push_back(o.second.first);
        ctx->ev_pool.push_back(o.second.second);
    }
    ctx->ev_open.clear();
    for (int i = 0; i < nphases && i < GP_NUM_PHASES; ++i) {
        if (ms) ms[i] = ctx->phase_ms[i];
        if (launches) launches[i] = ctx->phase_launches[i];
    }
    for (int i = 0; i < GP_NUM_PHASES; ++i) {
        ctx->phase_ms[i] = 0.0;
        ctx->phase_launches[i] = 0;
    }
    return GP_OK;
}

long long gp_launch_count(const gp_ctx* ctx) { return ctx ? ctx->launches : -1; }

int gp_corr_assemble(gp_ctx* ctx, int n, int d, const double* x, const double* theta, double p,
                     double delta, double* R, int layout) {
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (!x || !theta || !R) return fail(ctx, GP_EINVAL, "null pointer argument");
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    if (layout == 0) {
        if (n > 65535) return fail(ctx, GP_EINVAL, "dense layout limited to n <= 65535");
        GP_CUDA(ctx, gp::launch_assemble_dense(n, d, x, theta, p, ctx->opt.correlation, delta, R, ctx->stream));
        return GP_OK;
    }
    if (layout != 1 && layout != 2) return fail(ctx, GP_EINVAL, "layout must be 0, 1 or 2");
    rc = ensure_ws(ctx, align256(sizeof(gp::InstState)));
    if (rc) return rc;
    gp::Batch b{};
    b.n = n; b.d = d; b.nt = gp::num_tiles(n); b.count = 1; b.corr = ctx->opt.correlation;
    b.p = p; b.delta = delta; b.x = x; b.y = nullptr; b.theta = theta;
    if (layout == 1) {
        b.A = R;
    } else {
        b.A = nullptr;
        b.Adf = reinterpret_cast<float2*>(R);
        b.Rdf = reinterpret_cast<float2*>(R);
    }
    b.inst_stride = gp::packed_elems(n);
    b.st = (gp::InstState*)ctx->ws;
    GP_CUDA(ctx, gp::launch_validate_theta(b, ctx->stream));
    GP_CUDA(ctx, gp::launch_assemble_tiles(b, ctx->stream));
    return GP_OK;
}

int gp_cholesky(gp_ctx* ctx, int n, int d, const double* x, const double* theta, double p, double delta,
                int prec, double* L, int* status_host) {
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (!x || !theta || !L || !status_host) return fail(ctx, GP_EINVAL, "null pointer argument");
    if (prec == GP_AUTO) prec = GP_MIXED;
    if (prec != GP_FP64 && prec != GP_MIXED && prec != GP_FP32)
        return fail(ctx, GP_EINVAL, "unknown precision %d", prec);
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int nt = gp::num_tiles(n);
    gp::InstState* st = nullptr;
    if (prec == GP_FP64) {
        rc = ensure_ws(ctx, align256(sizeof(gp::InstState)));
        if (rc) return rc;
        st = (gp::InstState*)ctx->ws;
        gp::Batch b{};
        b.n = n; b.d = d; b.nt = nt; b.count = 1; b.p = p; b.delta = delta; b.corr = ctx->opt.correlation;
        b.x = x; b.y = nullptr; b.theta = theta; b.A = L; b.inst_stride = gp::packed_elems(n); b.st = st;
        {
            PhaseScope ps(ctx, GP_PHASE_ASSEMBLE, 2);
            GP_CUDA(ctx, gp::launch_validate_theta(b, ctx->stream));
            GP_CUDA(ctx, gp::launch_assemble_tiles(b, ctx->stream));
        }
        rc = run_factor_f64(ctx, b);
        if (rc) return rc;
    } else {
        const int slices = prec == GP_FP32 ? 3 : ctx->opt.slices;
        const MixedSizes z = mixed_sizes(n, slices);
        rc = ensure_ws(ctx, z.per + kMixedTail);
        if (rc) return rc;
        gp::MixedBatch mb = mixed_layout(ctx, n, 1, nullptr, (char*)ctx->ws, z, 1, slices);
        rc = run_mixed_factor(ctx, mb, d, x, theta, p, delta);
        if (rc) return rc;
        GP_CUDA(ctx, gp::launch_df_to_double(mb.A, L, gp::packed_elems(n), ctx->stream));
        st = mb.st;
    }
    GP_CUDA(ctx, cudaMemcpyAsync(status_host, &st->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GP_OK;
}

int gp_nll_batch_ex(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                    const double* theta, double p, double delta, int prec, double* nll,
                    double* mu_hat, double* sigma2_hat, double* logdet, int* status, double* cond1,
                    int* prec_used) {
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (T < 1 || T > gp::kMaxCandidates) return fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", T);
    if (!x || !y || !theta || !nll || !mu_hat || !sigma2_hat || !status)
        return fail(ctx, GP_EINVAL, "null pointer argument");
    if (prec != GP_FP64 && prec != GP_MIXED && prec != GP_FP32 && prec != GP_AUTO)
        return fail(ctx, GP_EINVAL, "unknown precision %d", prec);
    if (prec == GP_FP64 && cond1)
        return fail(ctx, GP_ENOTSUP, "the condition estimate comes with the split-precision factor only");
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    if (prec == GP_AUTO)
        return auto_nll_batch(ctx, n, d, x, y, T, theta, p, delta, nll, mu_hat, sigma2_hat, logdet, status,
                              cond1, prec_used);
    if (prec == GP_FP64)
        rc = fp64_nll_batch(ctx, n, d, x, y, T, theta, p, delta, nll, mu_hat, sigma2_hat, logdet, status);
    else
        rc = mixed_nll_batch(ctx, n, d, x, y, T, theta, p, delta, nll, mu_hat, sigma2_hat, logdet, status,
                             prec == GP_FP32 ? 3 : ctx->opt.slices, cond1);
    if (rc == GP_OK && prec_used) GP_CUDA(ctx, gp::launch_fill_int(prec_used, T, prec, ctx->stream));
    return rc;
}

int gp_nll_grad_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                      const double* theta, double p, double delta, double* nll, double* grad, int* status) {
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (T < 1 || T > gp::kMaxCandidates) return fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", T);
    if (d > 16) return fail(ctx, GP_ENOTSUP, "the gradient is built for d <= 16 (d = %d)", d);
    if (!x || !y || !theta || !nll || !grad || !status) return fail(ctx, GP_EINVAL, "null pointer argument");
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    const int nt = gp::num_tiles(n);
    const GradSizes g = grad_sizes(n, d);
    const size_t a_bytes = g.a, z_bytes = g.z, st_bytes = g.st, part_bytes = g.part;
    Chunking ch;
    if (!chunk_batch(ctx->opt, ctx->budget, ctx->models_bytes, g.per, 0, T, &ch))
        return fail(ctx, GP_ENOMEM, "one instance (%zu bytes) exceeds the HBM budget", g.per);
    const int Tc = ch.Tc;
    rc = ensure_ws(ctx, ch.bytes);
    if (rc) return rc;
    char* c = (char*)ctx->ws;
    double* A = (double*)c; c += a_bytes * Tc;
    double* X = (double*)c; c += a_bytes * Tc;
    double* Ri = (double*)c; c += a_bytes * Tc;
    double* Z = (double*)c; c += z_bytes * Tc;
    gp::InstState* st = (gp::InstState*)c; c += st_bytes * Tc;
    double* partial = (double*)c; c += part_bytes * Tc;
    double* sc = (double*)c;
    for (int c0 = 0; c0 < T; c0 += Tc) {
        const int cnt = (T - c0 < Tc) ? (T - c0) : Tc;
        gp::Batch b{};
        b.n = n; b.d = d; b.nt = nt; b.count = cnt; b.corr = ctx->opt.correlation;
        b.p = p; b.delta = delta; b.x = x; b.y = y; b.theta = theta + (size_t)c0 * d;
        b.A = A; b.inst_stride = a_bytes / sizeof(double); b.st = st;
        {
            PhaseScope ps(ctx, GP_PHASE_ASSEMBLE, 2);
            GP_CUDA(ctx, gp::launch_validate_theta(b, ctx->stream));
            GP_CUDA(ctx, gp::launch_assemble_tiles(b, ctx->stream));
        }
        rc = run_factor_f64(ctx, b);
        if (rc) return rc;
        const size_t zs = z_bytes / sizeof(double);
        {
            PhaseScope ps(ctx, GP_PHASE_SOLVE, gp::solve_f64_launches(b.nt, false) + 1);
            GP_CUDA(ctx, gp::launch_forward_solve(b, Z, zs, ctx->stream));
            GP_CUDA(ctx, gp::launch_finalize(b, Z, zs, nll + c0, sc, sc + Tc, sc + 2 * Tc, status + c0,
                                             ctx->stream));
        }
        int kernels = 0;
        cudaError_t e = gp::launch_grad(b, Z, zs, X, Ri, partial, status + c0, grad + (size_t)c0 * d,
                                        ctx->stream, &kernels);
        ctx->launches += kernels;
        ctx->phase_launches[GP_PHASE_SOLVE] += kernels;
        if (e != cudaSuccess) return fail(ctx, GP_ECUDA, "gradient launch: %s", cudaGetErrorString(e));
    }
    return GP_OK;
}

int gp_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                 const double* theta, double p, double delta, int prec, double* nll,
                 double* mu_hat, double* sigma2_hat, double* logdet, int* status) {
    return gp_nll_batch_ex(ctx, n, d, x, y, T, theta, p, delta, prec, nll, mu_hat, sigma2_hat, logdet,
                           status, nullptr, nullptr);
}

int gp_autotune(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T, const double* theta,
                double p, double delta, int prec, int reps, gp_tune_trial* trials, int max_trials, int* ntrials) {
    if (ntrials) *ntrials = 0;
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (T < 1 || T > gp::kMaxCandidates) return fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", T);
    if (!x || !y || !theta) return fail(ctx, GP_EINVAL, "null pointer argument");
    if (prec != GP_MIXED && prec != GP_FP32)
        return fail(ctx, GP_ENOTSUP, "the autotuner chooses split-precision launch shapes only");
    if (reps < 1) reps = 1;
    if (reps > 20) reps = 20;
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t bT = align256((size_t)T * sizeof(double));
    void* dev = nullptr;
    if (cudaMallocAsync(&dev, 4 * bT + align256((size_t)T * sizeof(int)), ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GP_ENOMEM, "autotuner staging allocation failed");
    }
    char* c = (char*)dev;
    double* o_nll = (double*)c;
    double* o_mu = (double*)(c + bT);
    double* o_s2 = (double*)(c + 2 * bT);
    double* o_ld = (double*)(c + 3 * bT);
    int* o_st = (int*)(c + 4 * bT);
    cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
    const gp_options base = ctx->opt;
    gp_options best = base;
    double best_ms = INFINITY;
    int count = 0;
    for (int ut : {128, 64}) {
        for (int fuse : {1, 0}) {
            for (int ac : {16, 32}) {
                if (base.update_groups != 4 && (fuse || ut == 64)) continue;
                gp_options o = base;
                o.update_tile = ut;
                o.fuse_panels = fuse;
                o.assemble_cols = ac;
                ctx->opt = o;
                std::vector<float> ms;
                for (int r = 0; r <= reps && rc == GP_OK; ++r) {
                    cudaEventRecord(e0, ctx->stream);
                    rc = gp_nll_batch(ctx, n, d, x, y, T, theta, p, delta, prec, o_nll, o_mu, o_s2, o_ld, o_st);
                    cudaEventRecord(e1, ctx->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess && rc == GP_OK)
                        rc = fail(ctx, GP_ECUDA, "autotuner: timing failed");
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (r > 0) ms.push_back(t);   // the first call is the warm-up
                }
                if (rc) break;
                std::sort(ms.begin(), ms.end());
                const double med = ms[ms.size() / 2];
                if (trials && count < max_trials) trials[count] = gp_tune_trial{ut, fuse, ac, med};
                ++count;
                if (med < best_ms) {
                    best_ms = med;
                    best = o;
                }
            }
            if (rc) break;
        }
        if (rc) break;
    }
    ctx->ev_pool.push_back(e0);
    ctx->ev_pool.push_back(e1);
    ctx->opt = rc ? base : best;
    cudaFreeAsync(dev, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (ntrials) *ntrials = count;
    return rc;
}

int gp_plan_nll_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                      const double* theta, double p, double delta, int prec, double* nll,
                      double* mu_hat, double* sigma2_hat, double* logdet, int* status, double* cond1,
                      gp_plan** out) {
    if (!out) return fail(ctx, GP_EINVAL, "null plan pointer");
    *out = nullptr;
    if (!ctx) return GP_EINVAL;
    if (prec == GP_AUTO)
        return fail(ctx, GP_ENOTSUP, "GP_AUTO routes candidates on the host and cannot be recorded");
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    // the plan gets a workspace of its own: the context's arena is set aside
    // (still counted against the budget) while the call runs and is recorded
    void* saved_ws = ctx->ws;
    const size_t saved_bytes = ctx->ws_bytes;
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    ctx->models_bytes += saved_bytes;
    auto restore = [&]() {
        ctx->models_bytes -= saved_bytes;
        ctx->ws = saved_ws;
        ctx->ws_bytes = saved_bytes;
    };
    auto release_own = [&]() {
        if (ctx->ws) cudaFreeAsync(ctx->ws, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    };
    // eager run: outputs valid, workspace sized, kernel attributes set
    int rc = gp_nll_batch_ex(ctx, n, d, x, y, T, theta, p, delta, prec, nll, mu_hat, sigma2_hat, logdet,
                             status, cond1, nullptr);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (rc == GP_OK && e != cudaSuccess) rc = fail(ctx, GP_ECUDA, "plan: %s", cudaGetErrorString(e));
    if (rc) {
        release_own();
        restore();
        return rc;
    }
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        release_own();
        restore();
        return fail(ctx, GP_ECUDA, "plan: stream creation failed");
    }
    cudaStream_t saved_stream = ctx->stream;
    const bool saved_timing = ctx->timing;
    const long long l0 = ctx->launches;
    long long ph0[GP_NUM_PHASES];
    std::memcpy(ph0, ctx->phase_launches, sizeof ph0);
    ctx->stream = cs;
    ctx->timing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = gp_nll_batch_ex(ctx, n, d, x, y, T, theta, p, delta, prec, nll, mu_hat, sigma2_hat, logdet,
                             status, cond1, nullptr);
        e = cudaStreamEndCapture(cs, &graph);
    }
    const long long kernels = ctx->launches - l0;
    ctx->launches = l0;   // recorded, not run
    std::memcpy(ctx->phase_launches, ph0, sizeof ph0);
    ctx->stream = saved_stream;
    ctx->timing = saved_timing;
    cudaStreamDestroy(cs);
    cudaGraphExec_t exec = nullptr;
    if (rc == GP_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (rc || e != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        release_own();
        restore();
        return rc ? rc : fail(ctx, GP_ECUDA, "plan: recording failed: %s", cudaGetErrorString(e));
    }
    gp_plan* q = new gp_plan();
    q->ctx = ctx;
    q->graph = graph;
    q->exec = exec;
    q->ws = ctx->ws;
    q->ws_bytes = ctx->ws_bytes;
    q->kernels = kernels;
    restore();
    ctx->models_bytes += q->ws_bytes;
    ctx->plans.push_back(q);
    *out = q;
    return GP_OK;
}

int gp_plan_launch(gp_plan* q) {
    if (!q) return GP_EINVAL;
    if (!q->ctx) return GP_EINVAL;   // its context is gone
    gp_ctx* ctx = q->ctx;
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    GP_CUDA(ctx, cudaGraphLaunch(q->exec, ctx->stream));
    ctx->launches += q->kernels;
    return GP_OK;
}

long long gp_plan_kernels(const gp_plan* q) { return q ? q->kernels : -1; }

size_t gp_plan_bytes(const gp_plan* q) { return q ? q->ws_bytes : 0; }

void gp_plan_destroy(gp_plan* q) {
    if (!q) return;
    if (q->ctx) {
        gp_ctx* ctx = q->ctx;
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        ctx->models_bytes -= q->ws_bytes;
        auto& v = ctx->plans;
        for (size_t i = 0; i < v.size(); ++i)
            if (v[i] == q) {
                v[i] = v.back();
                v.pop_back();
                break;
            }
        cudaGraphExecDestroy(q->exec);
        cudaGraphDestroy(q->graph);
        cudaFreeAsync(q->ws, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    } else {
        cudaDeviceSynchronize();
        cudaGraphExecDestroy(q->exec);
        cudaGraphDestroy(q->graph);
        cudaFree(q->ws);
    }
    delete q;
}

int gp_nll_batch_host(gp_ctx* ctx, int n, int d, const double* x_host, const double* y_host, int T,
                      const double* theta_host, double p, double delta, int prec, double* nll_host,
                      double* mu_hat_host, double* sigma2_hat_host, double* logdet_host,
                      int* status_host) {
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (T < 1 || T > gp::kMaxCandidates) return fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", T);
    if (!x_host || !y_host || !theta_host || !nll_host || !mu_hat_host || !sigma2_hat_host ||
        !status_host)
        return fail(ctx, GP_EINVAL, "null pointer argument");
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t bx = (size_t)n * d * sizeof(double), by = (size_t)n * sizeof(double);
    const size_t bt = (size_t)T * d * sizeof(double), bo = (size_t)T * sizeof(double);
    const size_t total = align256(bx) + align256(by) + align256(bt) + 4 * align256(bo) +
                         align256((size_t)T * sizeof(int));
    // the staging area is its own allocation so the batch can use the workspace
    void* dev = nullptr;
    cudaError_t e = cudaMallocAsync(&dev, total, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GP_ENOMEM, "staging allocation of %zu bytes failed", total);
    }
    char* c = (char*)dev;
    double* dx = (double*)c; c += align256(bx);
    double* dy = (double*)c; c += align256(by);
    double* dth = (double*)c; c += align256(bt);
    double* dnll = (double*)c; c += align256(bo);
    double* dmu = (double*)c; c += align256(bo);
    double* ds2 = (double*)c; c += align256(bo);
    double* dld = (double*)c; c += align256(bo);
    int* dst = (int*)c;
    cudaMemcpyAsync(dx, x_host, bx, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dy, y_host, by, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dth, theta_host, bt, cudaMemcpyHostToDevice, ctx->stream);
    rc = gp_nll_batch(ctx, n, d, dx, dy, T, dth, p, delta, prec, dnll, dmu, ds2, dld, dst);
    if (rc == GP_OK) {
        cudaMemcpyAsync(nll_host, dnll, bo, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(mu_hat_host, dmu, bo, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(sigma2_hat_host, ds2, bo, cudaMemcpyDeviceToHost, ctx->stream);
        if (logdet_host) cudaMemcpyAsync(logdet_host, dld, bo, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(status_host, dst, (size_t)T * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    }
    cudaFreeAsync(dev, ctx->stream);
    e = cudaStreamSynchronize(ctx->stream);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(ctx, GP_ECUDA, "stream synchronise: %s", cudaGetErrorString(e));
    return GP_OK;
}

int gp_fit(gp_ctx* ctx, int n, int d, const double* x, const double* y, const double* theta,
           double p, double delta, int prec, gp_model** model) {
    if (!model) return fail(ctx, GP_EINVAL, "null model pointer");
    *model = nullptr;
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (!x || !y || !theta) return fail(ctx, GP_EINVAL, "null pointer argument");
    if (prec != GP_FP64 && prec != GP_MIXED && prec != GP_FP32 && prec != GP_AUTO)
        return fail(ctx, GP_EINVAL, "unknown precision %d", prec);
    if (prec == GP_AUTO) prec = GP_FP64;
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    gp_model* m = nullptr;
    rc = model_alloc(ctx, n, d, p, delta, prec, &m);
    if (rc) return rc;
    const int npad = m->nt * GP_NB;
    if (prec != GP_FP64) {
        // the split factorisation of this one candidate in the workspace (its
        // outputs straight into the model's scalars), then the model from it
        LastChunk lc;
        rc = mixed_nll_batch(ctx, n, d, x, y, 1, theta, p, delta, m->scalars + 0, m->scalars + 1,
                             m->scalars + 2, m->scalars + 3, m->status, prec == GP_FP32 ? 3 : ctx->opt.slices,
                             nullptr, &lc);
        if (rc == GP_OK) rc = model_from_split(ctx, m, lc, 0, m->scalars + 0, m->status);
        if (rc) return model_discard(ctx, m, rc);
        return model_finish(ctx, m, x, theta, true, model);
    }
    // double: assembled and factored in the model's own storage
    if (cudaMemcpyAsync(m->theta, theta, (size_t)d * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream))
        return model_discard(ctx, m, fail(ctx, GP_ECUDA, "copy of theta into the model failed"));
    gp::Batch b{};
    b.n = n; b.d = d; b.nt = m->nt; b.count = 1; b.p = p; b.delta = delta; b.corr = m->corr;
    b.x = x; b.y = y; b.theta = m->theta; b.A = m->L; b.inst_stride = gp::packed_elems(n);
    b.st = m->st;
    {
        PhaseScope ps(ctx, GP_PHASE_ASSEMBLE, 2);
        if (gp::launch_validate_theta(b, ctx->stream) || gp::launch_assemble_tiles(b, ctx->stream))
            return model_discard(ctx, m, fail(ctx, GP_ECUDA, "assembly launch failed"));
    }
    rc = run_factor_f64(ctx, b);
    if (rc) return model_discard(ctx, m, rc);
    {
        PhaseScope ps(ctx, GP_PHASE_SOLVE,
                      gp::solve_f64_launches(b.nt, false) + 2 + gp::solve_f64_launches(b.nt, true));
        if (gp::launch_forward_solve(b, m->Z, (size_t)2 * npad, ctx->stream) ||
            gp::launch_finalize(b, m->Z, (size_t)2 * npad, m->scalars + 0, m->scalars + 1, m->scalars + 2,
                                m->scalars + 3, m->status, ctx->stream) ||
            gp::launch_fit_finish(b, m->Z, (size_t)2 * npad, m->scalars, ctx->stream) ||
            gp::launch_backward_solve(b, m->Z, (size_t)2 * npad, 1, ctx->stream))
            return model_discard(ctx, m, fail(ctx, GP_ECUDA, "solve launch failed"));
    }
    return model_finish(ctx, m, x, theta, false, model);
}

int gp_fit_batch(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T, const double* theta,
                 double p, double delta, int prec, double* nll, double* mu_hat, double* sigma2_hat,
                 double* logdet, int* status, int* best_host, gp_model** model) {
    if (!model || !best_host) return fail(ctx, GP_EINVAL, "null model or best pointer");
    *model = nullptr;
    *best_host = -1;
    int rc = check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (T < 1 || T > gp::kMaxCandidates) return fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", T);
    if (!x || !y || !theta || !nll || !mu_hat || !sigma2_hat || !status)
        return fail(ctx, GP_EINVAL, "null pointer argument");
    if (prec != GP_FP64 && prec != GP_MIXED && prec != GP_FP32)
        return fail(ctx, prec == GP_AUTO ? GP_ENOTSUP : GP_EINVAL,
                    "gp_fit_batch takes GP_FP64, GP_MIXED or GP_FP32 (precision %d)", prec);
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    LastChunk lc;
    if (prec == GP_FP64)
        rc = fp64_nll_batch(ctx, n, d, x, y, T, theta, p, delta, nll, mu_hat, sigma2_hat, logdet, status, &lc);
    else
        rc = mixed_nll_batch(ctx, n, d, x, y, T, theta, p, delta, nll, mu_hat, sigma2_hat, logdet, status,
                             prec == GP_FP32 ? 3 : ctx->opt.slices, nullptr, &lc);
    if (rc) return rc;
    std::vector<double> hn(T);
    std::vector<int> hs(T);
    GP_CUDA(ctx, cudaMemcpyAsync(hn.data(), nll, (size_t)T * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(ctx, cudaMemcpyAsync(hs.data(), status, (size_t)T * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int best = -1;
    for (int t = 0; t < T; ++t)
        if (hs[t] == GP_OK && (best < 0 || hn[t] < hn[best])) best = t;
    if (best < 0) return fail(ctx, GP_ENOTPD, "no candidate gave a likelihood (status of the first: %d)", hs[0]);
    *best_host = best;
    const double* th = theta + (size_t)best * d;
    if (best < lc.c0 || best >= lc.c0 + lc.cnt)   // its factor was overwritten by a later chunk
        return gp_fit(ctx, n, d, x, y, th, p, delta, prec, model);
    gp_model* m = nullptr;
    rc = model_alloc(ctx, n, d, p, delta, prec, &m);
    if (rc) return rc;
    const int t = best - lc.c0;
    if (prec == GP_FP64)
        rc = model_from_fp64(ctx, m, lc, t, nll + best, mu_hat + best, sigma2_hat + best,
                             logdet ? logdet + best : nullptr, status + best);
    else
        rc = model_from_split(ctx, m, lc, t, nll + best, status + best);
    if (rc) return model_discard(ctx, m, rc);
    if (prec == GP_FP64 && !logdet) {
        // log|R| was not asked for: the instance record has it
        const char* rec = reinterpret_cast<const char*>(lc.st + t) + offsetof(gp::InstState, logdet);
        GP_CUDA(ctx, cudaMemcpyAsync(m->scalars + 3, rec, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return model_finish(ctx, m, x, th, prec != GP_FP64, model);
}

int gp_model_scalars(const gp_model* m, double* out) {
    if (!m || !out) return GP_EINVAL;
    for (int i = 0; i < 6; ++i) out[i] = m->host_scalars[i];
    return GP_OK;
}

int gp_predict(gp_ctx* ctx, const gp_model* m, int N, const double* xstar, double* yhat, double* s2) {
    if (!ctx || !m) return GP_EINVAL;
    if (N < 0 || N > kMaxPredictPoints)
        return fail(ctx, GP_EINVAL, "N = %d outside [0, 2^30] test points per call", N);
    if (N == 0) return GP_OK;
    if (!xstar || !yhat) return fail(ctx, GP_EINVAL, "null pointer argument");
    GP_CUDA(ctx, cudaSetDevice(ctx->device));
    if (ctx->opt.predict_tc) return predict_tensor(ctx, m, N, xstar, yhat, s2);
    const int npad = m->nt * GP_NB;
    const size_t avail = ctx->budget > ctx->models_bytes ? ctx->budget - ctx->models_bytes : 0;
    const PredictShape sh = predict_shape(m->nt, N, ctx->sms, avail, s2 != nullptr);
    const int ppc = sh.ppc, blocks_total = sh.blocks, chunk = sh.chunk;
    int rc = ensure_ws(ctx, sh.bytes);
    if (rc) return rc;
    const double c0 = ctx->opt.nugget_in_var ? 1.0 + m->delta : 1.0;
    const float2* Ldf = reinterpret_cast<const float2*>(m->L);
    const float2* Zdf = reinterpret_cast<const float2*>(m->Z);
    PhaseScope ps(ctx, GP_PHASE_PREDICT, (blocks_total + chunk - 1) / chunk);
    GP_CUDA(ctx, gp::launch_predict(m->n, m->d, m->nt, reinterpret_cast<const float2*>(m->x), m->theta, m->p, m->corr,
                                    c0, Ldf, Zdf + npad, Zdf, m->scalars, N, xstar, yhat, s2,
                                    (float2*)ctx->ws, chunk, ppc, ctx->stream));
    return GP_OK;
}

void gp_model_free(gp_model* m) {
    if (!m) return;
    if (m->ctx) {
        cudaSetDevice(m->ctx->device);
        m->ctx->models_bytes -= m->bytes;
        auto& v = m->ctx->models;
        for (size_t i = 0; i < v.size(); ++i)
            if (v[i] == m) {
                v[i] = v.back();
                v.pop_back();
                break;
            }
        cudaFreeAsync(m->mem, m->ctx->stream);
        cudaStreamSynchronize(m->ctx->stream);
    } else {
        cudaFree(m->mem);
    }
    delete m;
}

size_t gp_model_bytes(const gp_model* m) { return m ? m->bytes : 0; }

int gp_call_bytes(gp_ctx* ctx, int call, int n, int d, int count, int prec, size_t* bytes) {
    if (!bytes) return fail(ctx, GP_EINVAL, "null bytes pointer");
    *bytes = 0;
    gp_options opt;
    size_t budget = SIZE_MAX, held = 0, ws = 0;
    int sms = 152;
    if (ctx) {
        opt = ctx->opt;
        budget = ctx->budget;
        held = ctx->models_bytes;
        ws = ctx->ws_bytes;
        sms = ctx->sms;
    } else {
        gp_default_options(&opt);
    }
    if (n < 1 || n > (1 << 20)) return fail(ctx, GP_EINVAL, "n = %d out of range [1, 2^20]", n);
    if (d < 1 || d > GP_MAX_D) return fail(ctx, GP_EINVAL, "d = %d out of range [1, %d]", d, GP_MAX_D);
    const size_t avail = budget > held ? budget - held : 0;
    // a workspace larger than the arena must fit the budget next to the models
    auto grow = [&](size_t need) {
        if (need > ws && need > avail)
            return fail(ctx, GP_ENOMEM, "workspace of %zu bytes exceeds the HBM budget", need);
        *bytes = need;
        return (int)GP_OK;
    };
    auto batch = [&](size_t per, size_t extra, size_t* out) {
        Chunking ch;
        if (!chunk_batch(opt, budget, held, per, extra, count, &ch))
            return fail(ctx, GP_ENOMEM, "one instance (%zu bytes) exceeds the HBM budget", per);
        *out = ch.bytes;
        return (int)GP_OK;
    };
    switch (call) {
    case GP_CALL_NLL_BATCH: {
        if (count < 1 || count > gp::kMaxCandidates)
            return fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", count);
        if (prec < GP_FP64 || prec > GP_AUTO) return fail(ctx, GP_EINVAL, "unknown precision %d", prec);
        size_t b64 = 0, bsplit = 0, b32 = 0;
        int rc = GP_OK;
        if (prec == GP_FP64 || prec == GP_AUTO) rc = batch(per_instance_bytes_f64(n), 0, &b64);
        if (rc == GP_OK && (prec == GP_MIXED || prec == GP_AUTO))
            rc = batch(mixed_sizes(n, opt.slices).per, kMixedTail, &bsplit);
        if (rc == GP_OK && (prec == GP_FP32 || prec == GP_AUTO))
            rc = batch(mixed_sizes(n, 3).per, kMixedTail, &b32);
        if (rc) return rc;
        *bytes = std::max(b64, std::max(bsplit, b32)) + (prec == GP_AUTO ? auto_staging_bytes(count, d) : 0);
        return GP_OK;
    }
    case GP_CALL_NLL_GRAD: {
        if (count < 1 || count > gp::kMaxCandidates)
            return fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", count);
        if (d > 16) return fail(ctx, GP_ENOTSUP, "the gradient is built for d <= 16 (d = %d)", d);
        return batch(grad_sizes(n, d).per, 0, bytes);
    }
    case GP_CALL_FIT: {
        const size_t total = model_sizes(n, d).total;
        if (total + held + ws > budget) return fail(ctx, GP_ENOMEM, "model of %zu bytes exceeds the HBM budget", total);
        *bytes = total;
        return GP_OK;
    }
    case GP_CALL_PREDICT:
        if (count < 0 || count > kMaxPredictPoints)
            return fail(ctx, GP_EINVAL, "N = %d outside [0, 2^30] test points per call", count);
        if (count == 0) return GP_OK;
        if (opt.predict_tc) return grow(var_plan(gp::num_tiles(n), count, sms, avail, true).bytes);
        return grow(predict_shape(gp::num_tiles(n), count, sms, avail, true).bytes);
    default:
        return fail(ctx, GP_EINVAL, "unknown call %d", call);
    }
}

}  // extern "C"
