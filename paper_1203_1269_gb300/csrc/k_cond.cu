// k_cond.cu -- 1-norm condition estimate of R for every candidate of a
// split-precision batch, from the factor already in the workspace.
//
// cond_1(R) = ||R||_1 ||R^-1||_1.  ||R||_1 is the largest absolute row sum of
// the stored copy of R (R is symmetric, so row and column sums agree).
// ||R^-1||_1 is estimated by Hager's method (W. W. Hager, "Condition
// estimates", SIAM J. Sci. Stat. Comput. 5, 1984), the iteration that
// LAPACK's condition estimators refine: starting from v = 1/n,
//     y = R^-1 v,  est = ||y||_1,  z = R^-1 sign(y),  j = argmax_i |z_i|;
//     stop when ||z||_inf <= z'v or j repeats, otherwise v = e_j;
// at most five rounds.  Each R^-1 application is a forward and a backward
// substitution with the double-float factor (the solve kernels of the split
// path, working on Z columns 5 and 6), so the estimate is that of the
// computed factor: it tracks cond_1(R) while cond_1(R) 2^-40 << 1.
//
// All candidates step through the rounds together; a candidate that has
// stopped is skipped by the kernels (InstState::hager_done).  The first y is
// R^-1 1 / n, which the likelihood solves already produced (Z column 0).
#include "df.cuh"
#include "gp_internal.cuh"

namespace gp {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kStage = GP_NB + 1;   // staged tile row stride (double-float entries)

__device__ __forceinline__ float2* zc(const MixedBatch& b, int t, int k) {
    return b.Z + (size_t)t * b.z_stride + (size_t)k * b.nt * GP_NB;
}

// Fixed-order block sum of one double per thread.
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s += red[i];
    __syncthreads();
    return s;
}

// Block max of one double per thread.
__device__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s = fmax(s, red[i]);
    __syncthreads();
    return s;
}

// ||R||_1 of each instance from the stored copy Rc.  Every lower tile (I, J)
// is staged once as |R| (double-float) and gives the row sums of rows in block
// I and, off the diagonal, through R_JI = R_IJ^T, the row sums of rows in
// block J.  The sums accumulate in Z column 7 as double-float pairs, each
// entry always by the same thread.  Dynamic smem: the staged tile.
__global__ void __launch_bounds__(kThreads) k_norm1(MixedBatch b) {
    extern __shared__ dfl S[];              // S[c * kStage + r] = |R_IJ(r, c)|
    __shared__ dfl part[4][GP_NB];
    __shared__ double red[kWarps];
    const int t = blockIdx.x;
    if (b.st[t].status != GP_OK) return;
    const int nt = b.nt, n = b.n;
    float2* acc = zc(b, t, 7);
    const int x = threadIdx.x & 127, h = threadIdx.x >> 7;
    if (threadIdx.x < GP_NB)
        for (int I = 0; I < nt; ++I) acc[I * GP_NB + x] = make_float2(0.f, 0.f);
    for (int J = 0; J < nt; ++J) {
        for (int I = J; I < nt; ++I) {
            const float2* T = b.Rc + (size_t)t * b.inst_stride + (size_t)tile_index(I, J, nt) * GP_TILE_ELEMS;
            __syncthreads();
            for (int q = threadIdx.x; q < GP_TILE_ELEMS; q += kThreads) {
                const float2 v = __ldg(T + q);
                S[(q >> 7) * kStage + (q & 127)] = (v.x < 0.f) ? dfl{-v.x, -v.y} : dfl{v.x, v.y};
            }
            __syncthreads();
            // rows of block I: thread (r, h) sums columns 32h .. 32h + 31
            dfl s = {0.f, 0.f};
            for (int c = 32 * h; c < 32 * h + 32; ++c) s = df_add(s, S[c * kStage + x]);
            part[h][x] = s;
            __syncthreads();
            if (threadIdx.x < GP_NB) {
                float2* a = acc + I * GP_NB + x;
                const dfl sum = df_add(df_add(part[0][x], part[1][x]), df_add(part[2][x], part[3][x]));
                df_store(a, df_add(df_load(a), sum));
            }
            if (I == J) continue;
            __syncthreads();
            // rows of block J (columns of this tile): thread (c, h) sums rows 32h .. 32h + 31
            s = {0.f, 0.f};
            for (int r = 32 * h; r < 32 * h + 32; ++r) s = df_add(s, S[x * kStage + r]);
            part[h][x] = s;
            __syncthreads();
            if (threadIdx.x < GP_NB) {
                float2* a = acc + J * GP_NB + x;
                const dfl sum = df_add(df_add(part[0][x], part[1][x]), df_add(part[2][x], part[3][x]));
                df_store(a, df_add(df_load(a), sum));
            }
        }
    }
    __syncthreads();
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) m = fmax(m, df_to_double(df_load(acc + i)));
    m = block_max(m, red);
    if (threadIdx.x == 0) b.st[t].anorm = m;
}

// One step of the estimate for every instance still running.
//   phase 0: first round: y = R^-1 1 / n from column 0; est = ||y||_1;
//            column 5 <- sign(y), column 6 <- 0
//   phase 1: y = R^-1 e_j in column 5: est = ||y||_1; column 5 <- sign(y)
//   phase 2: z = R^-1 sign(y) in column 5: the stopping test; column 5 <- e_j
//            for the next round unless the instance stops
//   phase 3: cond[t] = ||R||_1 est (NaN for a candidate without a factor)
__global__ void __launch_bounds__(kThreads) k_hager(MixedBatch b, int phase, double* cond) {
    __shared__ double red[kWarps];
    __shared__ int redi[kWarps];
    const int t = blockIdx.x;
    InstState* st = b.st + t;
    if (st->status != GP_OK) {
        if (phase == 3 && threadIdx.x == 0) cond[t] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    if (phase == 3) {
        if (threadIdx.x == 0) cond[t] = st->anorm * st->est;
        return;
    }
    if (phase != 0 && st->hager_done) return;
    const int n = b.n, npad = b.nt * GP_NB;
    float2* c5 = zc(b, t, 5);
    if (phase <= 1) {
        const float2* src = (phase == 0) ? zc(b, t, 0) : c5;
        const double scale = (phase == 0) ? 1.0 / n : 1.0;
        double s = 0.0;
        for (int i = threadIdx.x; i < npad; i += kThreads) {
            if (i < n) {
                const double v = df_to_double(df_load(src + i)) * scale;
                s += fabs(v);
                c5[i] = make_float2(v >= 0.0 ? 1.f : -1.f, 0.f);
            } else {
                c5[i] = make_float2(0.f, 0.f);
            }
        }
        if (phase == 0)
            for (int i = threadIdx.x; i < npad; i += kThreads) zc(b, t, 6)[i] = make_float2(0.f, 0.f);
        s = block_sum(s, red);
        if (threadIdx.x == 0) {
            st->est = s;
            if (phase == 0) {
                st->hager_iter = 0;
                st->hager_jprev = -1;
                st->hager_done = 0;
                st->refine_done = 0;   // the estimate's solves run for every instance
            }
        }
        return;
    }
    // phase 2: z = R^-1 sign(y)
    double zmax = -1.0, ztv = 0.0;
    int jmax = 0x7fffffff;
    const int it = st->hager_iter, jprev = st->hager_jprev;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const double z = df_to_double(df_load(c5 + i));
        if (fabs(z) > zmax) {   // i increases: the first index of a tie is kept
            zmax = fabs(z);
            jmax = i;
        }
        if (it == 0) ztv += z;
    }
    // block arg-max, ties to the smaller index
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, zmax, o);
        const int oj = __shfl_down_sync(0xffffffffu, jmax, o);
        if (ov > zmax || (ov == zmax && oj < jmax)) {
            zmax = ov;
            jmax = oj;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[w] = zmax;
        redi[w] = jmax;
    }
    __syncthreads();
    zmax = red[0];
    jmax = redi[0];
    for (int i = 1; i < kWarps; ++i)
        if (red[i] > zmax || (red[i] == zmax && redi[i] < jmax)) {
            zmax = red[i];
            jmax = redi[i];
        }
    __syncthreads();
    if (it == 0) {
        ztv = block_sum(ztv, red) / n;                       // z'v with v = 1/n
    } else {
        ztv = df_to_double(df_load(c5 + jprev));             // z'v with v = e_jprev
    }
    const bool stop = (zmax <= ztv) || (jmax == jprev) || (it + 1 >= 5);
    __syncthreads();
    if (!stop)
        for (int i = threadIdx.x; i < npad; i += kThreads) c5[i] = make_float2(i == jmax ? 1.f : 0.f, 0.f);
    if (threadIdx.x == 0) {
        if (stop) {
            st->hager_done = 1;
        } else {
            st->hager_jprev = jmax;
            st->hager_iter = it + 1;
        }
    }
}

__global__ void k_fill_int(int* dst, int count, int value) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = value;
}

// dst[idx[i]] = src[i]: results of a re-evaluated subset back into place.
template <typename V>
__global__ void k_scatter(int m, const int* __restrict__ idx, const V* __restrict__ src, V* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dst[idx[i]] = src[i];
}

}  // namespace

cudaError_t launch_fill_int(int* dst, int count, int value, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_fill_int<<<(count + 255) / 256, 256, 0, s>>>(dst, count, value);
    return cudaGetLastError();
}

cudaError_t launch_scatter(int m, const int* idx, const double* src, double* dst, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_scatter<double><<<(m + 255) / 256, 256, 0, s>>>(m, idx, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_scatter_int(int m, const int* idx, const int* src, int* dst, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_scatter<int><<<(m + 255) / 256, 256, 0, s>>>(m, idx, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_norm1(const MixedBatch& b, cudaStream_t s) {
    const size_t smem = (size_t)GP_NB * kStage * sizeof(dfl);
    static std::atomic<size_t> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(k_norm1, smem, attr);
    if (e != cudaSuccess) return e;
    k_norm1<<<b.count, kThreads, smem, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_hager(const MixedBatch& b, int phase, double* cond, cudaStream_t s) {
    k_hager<<<b.count, kThreads, 0, s>>>(b, phase, cond);
    return cudaGetLastError();
}

}  // namespace gp
