// gp_noalloc.cu -- gp_nll_batch_noalloc: the double-precision -2logL batch
// with its working memory in a fixed device array instead of memory the
// library allocates.
//
// Some callers cannot let a library call cudaMalloc: services that reserve
// their whole device-memory budget at start-up and forbid growth afterwards,
// hosts whose own allocator must account for every byte on the device, and
// latency-critical callers that cannot afford the device-wide synchronisation
// that cudaMalloc and cudaFree may cause.  For them this entry point keeps its
// scratch in the array below, which is reserved on every GPU that loads the
// library and stays reserved until the process exits.
#include <mutex>

#include "gp_internal.cuh"

namespace {

// The one scratch area shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once
// per device; host code cannot use the symbol itself as an address).
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int gp_nll_batch_noalloc(gp_ctx* ctx, int n, int d, const double* x, const double* y, int T,
                                    const double* theta, double p, double delta, double* nll,
                                    double* mu_hat, double* sigma2_hat, double* logdet, int* status) {
    const int rc = gp::ctx_check_common(ctx, n, d, p, delta);
    if (rc) return rc;
    if (T < 1 || T > gp::kMaxCandidates) return gp::ctx_fail(ctx, GP_EINVAL, "T = %d outside [1, 2^30]", T);
    if (!x || !y || !theta || !nll || !mu_hat || !sigma2_hat || !status)
        return gp::ctx_fail(ctx, GP_EINVAL, "null pointer argument");
    const int device = gp::ctx_device(ctx);
    if (device < 0 || device >= kMaxDevices) return gp::ctx_fail(ctx, GP_EINVAL, "device index out of range");
    const cudaStream_t stream = gp::ctx_stream(ctx);
    const int nt = gp::num_tiles(n);
    const size_t a_bytes = align256(gp::packed_elems(n) * sizeof(double));
    const size_t z_bytes = align256((size_t)2 * nt * GP_NB * sizeof(double));
    const size_t s_bytes = align256(sizeof(gp::InstState));
    const size_t per = a_bytes + z_bytes + s_bytes;
    if (per > GP_NOALLOC_SCRATCH_BYTES)
        return gp::ctx_fail(ctx, GP_ENOMEM,
                            "gp_nll_batch_noalloc: n = %d needs %zu bytes of scratch per candidate, more than "
                            "the fixed %zu-byte array (n <= %d fits)",
                            n, per, (size_t)GP_NOALLOC_SCRATCH_BYTES, GP_NOALLOC_MAX_N);
    cudaError_t e = cudaSetDevice(device);
    void* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(device, &scratch);
    if (e != cudaSuccess)
        return gp::ctx_fail(ctx, GP_ECUDA, "gp_nll_batch_noalloc: scratch set-up: %s", cudaGetErrorString(e));
    long long cap = (long long)(GP_NOALLOC_SCRATCH_BYTES / per);
    if (cap > 65535) cap = 65535;
    const int Tc = (int)(cap < T ? cap : T);
    char* base = (char*)scratch;
    double* A = (double*)base;
    double* Z = (double*)(base + a_bytes * Tc);
    gp::InstState* st = (gp::InstState*)(base + (a_bytes + z_bytes) * Tc);
    for (int c0 = 0; c0 < T; c0 += Tc) {
        const int cnt = (T - c0 < Tc) ? (T - c0) : Tc;
        gp::Batch b{};
        b.n = n; b.d = d; b.nt = nt; b.count = cnt; b.corr = gp::ctx_correlation(ctx);
        b.p = p; b.delta = delta; b.x = x; b.y = y; b.theta = theta + (size_t)c0 * d;
        b.A = A; b.inst_stride = a_bytes / sizeof(double); b.st = st;
        // every buffer the kernels read is written first: the theta check
        // resets each record, the assembly writes every tile (padding too)
        // and the forward solve writes Z, so nothing is cleared here
        e = gp::launch_validate_theta(b, stream);
        if (e == cudaSuccess) e = gp::launch_assemble_tiles(b, stream);
        for (int J = 0; J < nt && e == cudaSuccess; ++J) {
            e = gp::launch_potrf_f64(b, J, stream);
            if (e == cudaSuccess) e = gp::launch_trsm_f64(b, J, stream);
            if (e == cudaSuccess) e = gp::launch_update_f64(b, J, stream);
        }
        const size_t zs = z_bytes / sizeof(double);
        if (e == cudaSuccess) e = gp::launch_forward_solve(b, Z, zs, stream);
        if (e == cudaSuccess)
            e = gp::launch_finalize(b, Z, zs, nll + c0, mu_hat + c0, sigma2_hat + c0,
                                    logdet ? logdet + c0 : nullptr, status + c0, stream);
        if (e != cudaSuccess)
            return gp::ctx_fail(ctx, GP_ECUDA, "gp_nll_batch_noalloc: launch: %s", cudaGetErrorString(e));
    }
    return GP_OK;
}
