// Learned variant dispatcher.
//
// Every variant (squaring on tensor cores or on packed rows, frontier
// expansion on tensor cores or on packed rows) returns the same bits; they
// differ only in speed, and which is fastest depends on the graph. A small
// MLP predicts each variant's log2 run time from 16 cheap graph features
// computed on the GPU; the dispatcher runs the argmin. The network
// (16 -> 64 -> 64 -> 4, ReLU, FP16 weights, FP32 accumulation) is trained on
// the GPU by the forward / backward / Adam kernels below, on timings the
// library itself measures. Without a trained network BMLP_AUTO falls back to
// squaring on the tensor cores.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include <cuda_fp16.h>

#include "internal.h"

namespace bmlp {
namespace {

constexpr int NF = BMLP_NFEAT;        // 16 features
constexpr int NH = 64;                // hidden width
constexpr int NV = BMLP_NVAR;         // 4 variants
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NV * NH;
constexpr int NP = OB3 + NV;          // 5,508 parameters
static_assert(NP == BMLP_MLP_PARAMS, "parameter count");

constexpr int NSAMPLE = 1024;         // rows sampled for in-degree, reciprocity, locality
constexpr int NPROBE = 64;            // probe sources for the two frontier steps
constexpr int NBRANCH = 64;           // frontier rows OR-ed per probe in step two

// accumulator slots (double) of the feature pass
enum {
    A_NNZ = 0, A_NNZ2, A_MAXOUT, A_ZOUT, A_WORDS, A_DIAG,            // all rows
    A_SEDGES, A_RECIP, A_LOCAL,                                      // sampled rows
    A_INSUM, A_INSUM2, A_INMAX, A_INZERO,                            // sampled in-degrees
    A_P1, A_P2, A_PDEAD,                                             // probes
    A_COUNT
};

__device__ __forceinline__ void atomic_max_d(double* a, double v) {
    unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
    unsigned long long old = *p;
    while (__longlong_as_double(static_cast<long long>(old)) < v) {
        const unsigned long long got = atomicCAS(p, old, static_cast<unsigned long long>(__double_as_longlong(v)));
        if (got == old) break;
        old = got;
    }
}

// Pass 1: warp per row. Out-degree moments, empty rows, nonzero words, self loops.
__global__ void feat_rows_kernel(const uint64_t* __restrict__ P, int64_t n, int64_t ldw, double* acc) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t wpr = (n + 63) / 64;
    double s1 = 0, s2 = 0, mx = 0, z = 0, words = 0, diag = 0;
    for (int64_t i = warp; i < n; i += nw) {
        long long c = 0, nzw = 0;
        for (int64_t w = lane; w < wpr; w += 32) {
            const uint64_t x = P[i * ldw + w];
            c += __popcll(x);
            nzw += x != 0;
        }
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
            nzw += __shfl_xor_sync(0xFFFFFFFFu, nzw, o);
        }
        if (lane == 0) {
            s1 += c;
            s2 += static_cast<double>(c) * c;
            mx = fmax(mx, static_cast<double>(c));
            z += c == 0;
            words += nzw;
            diag += (P[i * ldw + (i >> 6)] >> (i & 63)) & 1ull;
        }
    }
    if (lane == 0) {
        atomicAdd(&acc[A_NNZ], s1);
        atomicAdd(&acc[A_NNZ2], s2);
        atomic_max_d(&acc[A_MAXOUT], mx);
        atomicAdd(&acc[A_ZOUT], z);
        atomicAdd(&acc[A_WORDS], words);
        atomicAdd(&acc[A_DIAG], diag);
    }
}

// Pass 2: block per sampled row i: in-degree counts, reciprocity, locality;
// the first NPROBE sampled rows also run two frontier steps (probes).
__global__ void __launch_bounds__(256) feat_sample_kernel(const uint64_t* __restrict__ P, int64_t n, int64_t ldw,
                                                          int ns, int* __restrict__ indeg, double* acc) {
    __shared__ unsigned long long s_edges, s_recip, s_p2;
    __shared__ double s_local;
    __shared__ int64_t branch[NBRANCH];
    __shared__ int nbranch;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * n / ns;
    const int64_t wpr = (n + 63) / 64;
    if (threadIdx.x == 0) {
        s_edges = s_recip = s_p2 = 0;
        s_local = 0;
        nbranch = 0;
    }
    __syncthreads();
    unsigned long long e = 0, r = 0;
    double loc = 0;
    for (int64_t w = threadIdx.x; w < wpr; w += blockDim.x) {
        uint64_t x = P[i * ldw + w];
        while (x) {
            const int b = __ffsll(static_cast<long long>(x)) - 1;
            x &= x - 1;
            const int64_t j = w * 64 + b;
            atomicAdd(&indeg[j], 1);
            ++e;
            r += (P[j * ldw + (i >> 6)] >> (i & 63)) & 1ull;
            loc += fabs(static_cast<double>(j - i));
        }
    }
    atomicAdd(&s_edges, e);
    atomicAdd(&s_recip, r);
    atomicAdd(&s_local, loc);
    __syncthreads();
    if (blockIdx.x < NPROBE) {
        // branches: the NBRANCH lowest set columns of row i (block scan of word popcounts)
        __shared__ int scan[256];
        for (int64_t c0 = 0; c0 < wpr && nbranch < NBRANCH; c0 += blockDim.x) {
            const int64_t w = c0 + threadIdx.x;
            const uint64_t x = w < wpr ? P[i * ldw + w] : 0ull;
            scan[threadIdx.x] = __popcll(x);
            __syncthreads();
            for (int off = 1; off < static_cast<int>(blockDim.x); off <<= 1) {
                const int v = threadIdx.x >= static_cast<unsigned>(off) ? scan[threadIdx.x - off] : 0;
                __syncthreads();
                scan[threadIdx.x] += v;
                __syncthreads();
            }
            int rank = nbranch + scan[threadIdx.x] - __popcll(x);
            uint64_t y = x;
            while (y && rank < NBRANCH) {
                const int b = __ffsll(static_cast<long long>(y)) - 1;
                y &= y - 1;
                branch[rank++] = w * 64 + b;
            }
            __syncthreads();
            if (threadIdx.x == 0) nbranch += scan[blockDim.x - 1];
            __syncthreads();
        }
        const int nb = min(nbranch, NBRANCH);
        unsigned long long p2 = 0;
        for (int64_t w = threadIdx.x; w < wpr; w += blockDim.x) {
            uint64_t f = 0;
            for (int k = 0; k < nb; ++k) f |= P[branch[k] * ldw + w];
            p2 += __popcll(f);
        }
        atomicAdd(&s_p2, p2);
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&acc[A_P1], static_cast<double>(s_edges));
            atomicAdd(&acc[A_P2], static_cast<double>(s_p2));
            atomicAdd(&acc[A_PDEAD], s_p2 == 0 ? 1.0 : 0.0);
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd(&acc[A_SEDGES], static_cast<double>(s_edges));
        atomicAdd(&acc[A_RECIP], static_cast<double>(s_recip));
        atomicAdd(&acc[A_LOCAL], s_local);
    }
}

// Pass 3: moments of the sampled in-degree counts.
__global__ void feat_indeg_kernel(const int* __restrict__ indeg, int64_t n, double* acc) {
    double s1 = 0, s2 = 0, mx = 0, z = 0;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double c = indeg[j];
        s1 += c;
        s2 += c * c;
        mx = fmax(mx, c);
        z += c == 0;
    }
    atomicAdd(&acc[A_INSUM], s1);
    atomicAdd(&acc[A_INSUM2], s2);
    atomic_max_d(&acc[A_INMAX], mx);
    atomicAdd(&acc[A_INZERO], z);
}

// The 16 features from the accumulators (one thread).
__global__ void feat_final_kernel(const double* acc, int64_t n, int ns, float* f) {
    const double N = static_cast<double>(n), S = ns;
    const double nnz = acc[A_NNZ], mean = nnz / N;
    const double var = fmax(acc[A_NNZ2] / N - mean * mean, 0.0);
    const double scale = N / S;  // sampled in-degrees -> whole-graph estimate
    const double imean = acc[A_INSUM] / N * scale;
    const double ivar = fmax(acc[A_INSUM2] / N * scale * scale - imean * imean, 0.0);
    const double se = fmax(acc[A_SEDGES], 1.0);
    const double p1 = acc[A_P1] / fmin(S, static_cast<double>(NPROBE));
    const double p2 = acc[A_P2] / fmin(S, static_cast<double>(NPROBE));
    f[0] = static_cast<float>(log2(N));
    f[1] = static_cast<float>(log2(1.0 + nnz));
    f[2] = static_cast<float>(mean);
    f[3] = static_cast<float>(sqrt(var));
    f[4] = static_cast<float>(acc[A_MAXOUT] / N);
    f[5] = static_cast<float>(acc[A_ZOUT] / N);
    f[6] = static_cast<float>(sqrt(ivar));
    f[7] = static_cast<float>(acc[A_INMAX] * scale / N);
    f[8] = static_cast<float>(acc[A_INZERO] / N);
    f[9] = static_cast<float>(acc[A_DIAG] / N);
    f[10] = static_cast<float>(acc[A_RECIP] / se);
    f[11] = static_cast<float>(acc[A_WORDS] / (N * ceil(N / 64.0)));
    f[12] = static_cast<float>(acc[A_LOCAL] / se / N);
    f[13] = static_cast<float>(p2 / N);
    f[14] = static_cast<float>(log2((p2 + 1.0) / (p1 + 1.0)));
    f[15] = static_cast<float>(acc[A_PDEAD] / fmin(S, static_cast<double>(NPROBE)));
}

// ------------------------------------------------------------- the MLP --
struct MlpData {
    const float* X;          // m x 16 raw features
    const float* Y;          // m x 4 log2 run times (ms)
    const uint8_t* C;        // m x 4: 1 = censored (true time >= Y)
    int m;
};

// Forward of one sample with FP16 weights w (smem), FP32 accumulation.
// x is normalised in place. h1, h2, y are outputs.
__device__ __forceinline__ void mlp_fwd(const __half* w, const float* mu, const float* sig, float* x, float* h1,
                                        float* h2, float* y) {
#pragma unroll
    for (int k = 0; k < NF; ++k) x[k] = (x[k] - mu[k]) / sig[k];
    for (int j = 0; j < NH; ++j) {
        float a = __half2float(w[OB1 + j]);
#pragma unroll
        for (int k = 0; k < NF; ++k) a += __half2float(w[OW1 + j * NF + k]) * x[k];
        h1[j] = fmaxf(a, 0.f);
    }
    for (int j = 0; j < NH; ++j) {
        float a = __half2float(w[OB2 + j]);
        for (int k = 0; k < NH; ++k) a += __half2float(w[OW2 + j * NH + k]) * h1[k];
        h2[j] = fmaxf(a, 0.f);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        float a = __half2float(w[OB3 + v]);
        for (int k = 0; k < NH; ++k) a += __half2float(w[OW3 + v * NH + k]) * h2[k];
        y[v] = a;
    }
}

// Loss of one sample (mean over the 4 outputs) and dL/dy. A censored time
// only bounds the truth from below: predicting above it costs nothing.
__device__ __forceinline__ float mlp_loss(const float* y, const float* t, const uint8_t* c, float* dy, float scale) {
    float l = 0.f;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        float d = y[v] - t[v];
        if (c[v] && d > 0.f) d = 0.f;
        l += d * d;
        dy[v] = 2.f * d * scale;
    }
    return l;
}

// Accumulate this sample's gradient into g (shared memory, FP32 atomics).
__device__ __forceinline__ void mlp_bwd(const __half* w, const float* x, const float* h1, const float* h2,
                                        const float* dy, float* g) {
    float dh2[NH];
    for (int k = 0; k < NH; ++k) {
        float a = 0.f;
#pragma unroll
        for (int v = 0; v < NV; ++v) a += __half2float(w[OW3 + v * NH + k]) * dy[v];
        dh2[k] = h2[k] > 0.f ? a : 0.f;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        atomicAdd(&g[OB3 + v], dy[v]);
        for (int k = 0; k < NH; ++k) atomicAdd(&g[OW3 + v * NH + k], dy[v] * h2[k]);
    }
    float dh1[NH];
    for (int k = 0; k < NH; ++k) dh1[k] = 0.f;
    for (int j = 0; j < NH; ++j) {
        if (dh2[j] == 0.f) continue;
        atomicAdd(&g[OB2 + j], dh2[j]);
        for (int k = 0; k < NH; ++k) {
            atomicAdd(&g[OW2 + j * NH + k], dh2[j] * h1[k]);
            dh1[k] += __half2float(w[OW2 + j * NH + k]) * dh2[j];
        }
    }
    for (int j = 0; j < NH; ++j) {
        const float d = h1[j] > 0.f ? dh1[j] : 0.f;
        if (d == 0.f) continue;
        atomicAdd(&g[OB1 + j], d);
#pragma unroll
        for (int k = 0; k < NF; ++k) atomicAdd(&g[OW1 + j * NF + k], d * x[k]);
    }
}

constexpr int MLP_THREADS = 256;

// Loss and gradient over all m samples at the current FP16 weights (for
// gradient checks). One block; g and loss in global memory.
__global__ void __launch_bounds__(MLP_THREADS) mlp_grad_kernel(const __half* wg, const float* mu, const float* sig,
                                                               MlpData d, float* g_out, float* loss_out) {
    __shared__ __half w[NP];
    __shared__ float g[NP];
    __shared__ float lsum;
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        w[p] = wg[p];
        g[p] = 0.f;
    }
    if (threadIdx.x == 0) lsum = 0.f;
    __syncthreads();
    const float scale = 1.f / (static_cast<float>(d.m) * NV);
    float l = 0.f;
    for (int s = threadIdx.x; s < d.m; s += blockDim.x) {
        float x[NF], h1[NH], h2[NH], y[NV], dy[NV];
        for (int k = 0; k < NF; ++k) x[k] = d.X[s * NF + k];
        mlp_fwd(w, mu, sig, x, h1, h2, y);
        l += mlp_loss(y, d.Y + s * NV, d.C + s * NV, dy, scale);
        mlp_bwd(w, x, h1, h2, dy, g);
    }
    atomicAdd(&lsum, l * scale);
    __syncthreads();
    for (int p = threadIdx.x; p < NP; p += blockDim.x) g_out[p] = g[p];
    if (threadIdx.x == 0) *loss_out = lsum;
}

// Adam training: one block runs every epoch; mini-batches of `batch`
// samples in a per-epoch shuffled order (xorshift permutation by thread 0).
// Master weights in FP32 (global), the forward/backward use FP16 copies.
__global__ void __launch_bounds__(MLP_THREADS) mlp_train_kernel(float* master, float* mom1, float* mom2, __half* wg,
                                                                const float* mu, const float* sig, MlpData d,
                                                                int* perm, int epochs, int batch, float lr, float wd,
                                                                unsigned long long seed, float* loss_out) {
    __shared__ __half w[NP];
    __shared__ float g[NP];
    __shared__ float lsum;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int step = 0;
    float last = 0.f;
    for (int p = threadIdx.x; p < NP; p += blockDim.x) w[p] = __float2half(master[p]);
    __syncthreads();
    for (int ep = 0; ep < epochs; ++ep) {
        if (threadIdx.x == 0) {
            unsigned long long s = seed * 0x9E3779B97F4A7C15ull + static_cast<unsigned long long>(ep) + 1;
            for (int i = 0; i < d.m; ++i) perm[i] = i;
            for (int i = d.m - 1; i > 0; --i) {
                s ^= s << 13;
                s ^= s >> 7;
                s ^= s << 17;
                const int j = static_cast<int>(s % static_cast<unsigned long long>(i + 1));
                const int t = perm[i];
                perm[i] = perm[j];
                perm[j] = t;
            }
            lsum = 0.f;
        }
        __syncthreads();
        for (int b0 = 0; b0 < d.m; b0 += batch) {
            const int bsz = min(batch, d.m - b0);
            for (int p = threadIdx.x; p < NP; p += blockDim.x) g[p] = 0.f;
            __syncthreads();
            const float scale = 1.f / (static_cast<float>(bsz) * NV);
            float l = 0.f;
            for (int t = threadIdx.x; t < bsz; t += blockDim.x) {
                const int s = perm[b0 + t];
                float x[NF], h1[NH], h2[NH], y[NV], dy[NV];
                for (int k = 0; k < NF; ++k) x[k] = d.X[s * NF + k];
                mlp_fwd(w, mu, sig, x, h1, h2, y);
                l += mlp_loss(y, d.Y + s * NV, d.C + s * NV, dy, scale);
                mlp_bwd(w, x, h1, h2, dy, g);
            }
            atomicAdd(&lsum, l * scale * (static_cast<float>(bsz) / d.m));
            __syncthreads();
            ++step;
            const float c1 = 1.f - powf(b1, static_cast<float>(step));
            const float c2 = 1.f - powf(b2, static_cast<float>(step));
            for (int p = threadIdx.x; p < NP; p += blockDim.x) {
                const float gr = g[p] + wd * master[p];
                mom1[p] = b1 * mom1[p] + (1.f - b1) * gr;
                mom2[p] = b2 * mom2[p] + (1.f - b2) * gr * gr;
                master[p] -= lr * (mom1[p] / c1) / (sqrtf(mom2[p] / c2) + eps);
                w[p] = __float2half(master[p]);
            }
            __syncthreads();
        }
        last = lsum;
        __syncthreads();
    }
    for (int p = threadIdx.x; p < NP; p += blockDim.x) wg[p] = w[p];
    if (threadIdx.x == 0) *loss_out = last;
}

__global__ void __launch_bounds__(MLP_THREADS) mlp_predict_kernel(const __half* wg, const float* mu, const float* sig,
                                                                  const float* X, int m, float* Y, int* choice) {
    __shared__ __half w[NP];
    for (int p = threadIdx.x; p < NP; p += blockDim.x) w[p] = wg[p];
    __syncthreads();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x) {
        float x[NF], h1[NH], h2[NH], y[NV];
        for (int k = 0; k < NF; ++k) x[k] = X[s * NF + k];
        mlp_fwd(w, mu, sig, x, h1, h2, y);
        int best = 0;
        for (int v = 0; v < NV; ++v) {
            Y[s * NV + v] = y[v];
            if (y[v] < y[best]) best = v;
        }
        choice[s] = best;
    }
}

}  // namespace

// Dispatcher state owned by a context.
struct Dispatch {
    bool trained = false;
    float mu[NF], sig[NF];
    std::vector<float> master;        // FP32 weights (host mirror)
    float* d_master = nullptr;        // FP32 master, Adam moments
    float* d_m1 = nullptr;
    float* d_m2 = nullptr;
    __half* d_w = nullptr;            // FP16 weights used by the kernels
    float* d_norm = nullptr;          // mu | sig
    double* d_acc = nullptr;          // feature accumulators
    float* d_feat = nullptr;
    float* d_small = nullptr;         // loss, scratch
    int* d_indeg = nullptr;
    int64_t indeg_cap = 0;
    float* d_px = nullptr;            // prediction inputs / outputs / choices, grow-only (no allocation per call)
    float* d_py = nullptr;
    int* d_pc = nullptr;
    int64_t pred_cap = 0;
};

void dispatch_free(bmlp_ctx* ctx) {
    Dispatch* d = static_cast<Dispatch*>(ctx->dispatch);
    if (!d) return;
    cudaFree(d->d_master);
    cudaFree(d->d_m1);
    cudaFree(d->d_m2);
    cudaFree(d->d_w);
    cudaFree(d->d_norm);
    cudaFree(d->d_acc);
    cudaFree(d->d_feat);
    cudaFree(d->d_small);
    cudaFree(d->d_indeg);
    cudaFree(d->d_px);
    cudaFree(d->d_py);
    cudaFree(d->d_pc);
    delete d;
    ctx->dispatch = nullptr;
}

namespace {

#define DCK(call, what)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, what);   \
    } while (0)

bmlp_status dispatch_state(bmlp_ctx* ctx, Dispatch** out) {
    Dispatch* d = static_cast<Dispatch*>(ctx->dispatch);
    if (!d) {
        d = new Dispatch();
        ctx->dispatch = d;
        d->master.assign(NP, 0.f);
        for (int k = 0; k < NF; ++k) {
            d->mu[k] = 0.f;
            d->sig[k] = 1.f;
        }
        DCK(cudaMalloc(&d->d_master, NP * sizeof(float)), "cudaMalloc(dispatcher)");
        DCK(cudaMalloc(&d->d_m1, NP * sizeof(float)), "cudaMalloc(dispatcher)");
        DCK(cudaMalloc(&d->d_m2, NP * sizeof(float)), "cudaMalloc(dispatcher)");
        DCK(cudaMalloc(&d->d_w, NP * sizeof(__half)), "cudaMalloc(dispatcher)");
        DCK(cudaMalloc(&d->d_norm, 2 * NF * sizeof(float)), "cudaMalloc(dispatcher)");
        DCK(cudaMalloc(&d->d_acc, A_COUNT * sizeof(double)), "cudaMalloc(dispatcher)");
        DCK(cudaMalloc(&d->d_feat, NF * sizeof(float)), "cudaMalloc(dispatcher)");
        DCK(cudaMalloc(&d->d_small, 16 * sizeof(float)), "cudaMalloc(dispatcher)");
    }
    *out = d;
    return BMLP_OK;
}

bmlp_status upload_params(bmlp_ctx* ctx, Dispatch* d) {
    std::vector<__half> h(NP);
    for (int p = 0; p < NP; ++p) h[p] = __float2half(d->master[p]);
    float norm[2 * NF];
    for (int k = 0; k < NF; ++k) {
        norm[k] = d->mu[k];
        norm[NF + k] = d->sig[k];
    }
    DCK(cudaMemcpy(d->d_master, d->master.data(), NP * sizeof(float), cudaMemcpyHostToDevice), "upload weights");
    DCK(cudaMemcpy(d->d_w, h.data(), NP * sizeof(__half), cudaMemcpyHostToDevice), "upload weights");
    DCK(cudaMemcpy(d->d_norm, norm, sizeof(norm), cudaMemcpyHostToDevice), "upload normalisation");
    return BMLP_OK;
}

template <class T>
bmlp_status to_device(bmlp_ctx* ctx, const T* h, size_t count, T** out) {
    DCK(cudaMalloc(out, count * sizeof(T) + 16), "cudaMalloc(dispatcher data)");
    DCK(cudaMemcpy(*out, h, count * sizeof(T), cudaMemcpyHostToDevice), "copy dispatcher data");
    return BMLP_OK;
}

}  // namespace

// The feature kernels of a device matrix in packed rows (n x ldw words): the 16 features land in dst (default
// d->d_feat).
static bmlp_status launch_features(bmlp_ctx* ctx, Dispatch* d, const uint64_t* P, int64_t n, int64_t ldw, cudaStream_t s,
                                   float* dst = nullptr) {
    if (d->indeg_cap < n) {
        if (d->d_indeg) cudaFree(d->d_indeg);
        d->d_indeg = nullptr;
        d->indeg_cap = 0;
        DCK(cudaMalloc(&d->d_indeg, static_cast<size_t>(n) * sizeof(int)), "cudaMalloc(in-degree counts)");
        d->indeg_cap = n;
    }
    const int ns = static_cast<int>(n < NSAMPLE ? n : NSAMPLE);
    DCK(cudaMemsetAsync(d->d_acc, 0, A_COUNT * sizeof(double), s), "clear accumulators");
    DCK(cudaMemsetAsync(d->d_indeg, 0, static_cast<size_t>(n) * sizeof(int), s), "clear in-degrees");
    int64_t blocks = (n + 7) / 8;
    if (blocks > ctx->sm_count * 16) blocks = ctx->sm_count * 16;
    feat_rows_kernel<<<static_cast<int>(blocks < 1 ? 1 : blocks), 256, 0, s>>>(P, n, ldw, d->d_acc);
    feat_sample_kernel<<<ns, 256, 0, s>>>(P, n, ldw, ns, d->d_indeg, d->d_acc);
    int64_t b3 = (n + 255) / 256;
    if (b3 > ctx->sm_count * 8) b3 = ctx->sm_count * 8;
    feat_indeg_kernel<<<static_cast<int>(b3 < 1 ? 1 : b3), 256, 0, s>>>(d->d_indeg, n, d->d_acc);
    feat_final_kernel<<<1, 1, 0, s>>>(d->d_acc, n, ns, dst != nullptr ? dst : d->d_feat);
    DCK(cudaGetLastError(), "feature kernels");
    ctx->stats.launches += 4;
    return BMLP_OK;
}

static bmlp_status pred_buffers(bmlp_ctx* ctx, Dispatch* d, int64_t m) {
    if (d->pred_cap >= m) return BMLP_OK;
    cudaFree(d->d_px);
    cudaFree(d->d_py);
    cudaFree(d->d_pc);
    d->d_px = d->d_py = nullptr;
    d->d_pc = nullptr;
    d->pred_cap = 0;
    const int64_t cap = m < 256 ? 256 : m;
    DCK(cudaMalloc(&d->d_px, cap * NF * sizeof(float)), "cudaMalloc(predict)");
    DCK(cudaMalloc(&d->d_py, cap * NV * sizeof(float)), "cudaMalloc(predict)");
    DCK(cudaMalloc(&d->d_pc, cap * sizeof(int)), "cudaMalloc(predict)");
    d->pred_cap = cap;
    return BMLP_OK;
}

// Features of a device matrix already in packed rows (n x ldw words).
bmlp_status dispatch_features_packed(bmlp_ctx* ctx, const uint64_t* P, int64_t n, int64_t ldw, float* feat_host,
                                     cudaStream_t s) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    st = launch_features(ctx, d, P, n, ldw, s);
    if (st != BMLP_OK) return st;
    DCK(cudaMemcpyAsync(feat_host, d->d_feat, NF * sizeof(float), cudaMemcpyDeviceToHost, s), "read features");
    DCK(host_sync(ctx, s), "synchronise features");
    return BMLP_OK;
}

// Features and prediction on the device in one go (the features never visit the host): *choice receives the
// predicted fastest bmlp_variant; one host wait.
bmlp_status dispatch_choose_packed(bmlp_ctx* ctx, const uint64_t* P, int64_t n, int64_t ldw, int32_t* choice,
                                   cudaStream_t s) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    st = launch_features(ctx, d, P, n, ldw, s);
    if (st != BMLP_OK) return st;
    st = pred_buffers(ctx, d, 1);
    if (st != BMLP_OK) return st;
    mlp_predict_kernel<<<1, MLP_THREADS, 0, s>>>(d->d_w, d->d_norm, d->d_norm + NF, d->d_feat, 1, d->d_py, d->d_pc);
    DCK(cudaGetLastError(), "predict kernel");
    ctx->stats.launches++;
    int c = 0;
    DCK(cudaMemcpyAsync(&c, d->d_pc, sizeof(int), cudaMemcpyDeviceToHost, s), "read choice");
    DCK(host_sync(ctx, s), "synchronise choice");
    *choice = c + 1;  // bmlp_variant numbering
    return BMLP_OK;
}

// Features and predictions for m device matrices in packed rows (P[i]: n[i] x ldw[i] words) with one host wait:
// the features of matrix i land in row i of the prediction input, one predict launch covers all m rows, and the
// choices (bmlp_variant numbering) and, if feat_host is not null, the features (m x 16) are read back together.
bmlp_status dispatch_choose_many_packed(bmlp_ctx* ctx, const uint64_t* const* P, const int64_t* n, const int64_t* ldw,
                                        int64_t m, float* feat_host, int32_t* choice, cudaStream_t s) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    if (m <= 0) return BMLP_OK;
    st = pred_buffers(ctx, d, m);
    if (st != BMLP_OK) return st;
    for (int64_t i = 0; i < m; ++i) {
        st = launch_features(ctx, d, P[i], n[i], ldw[i], s, d->d_px + i * NF);
        if (st != BMLP_OK) return st;
    }
    const int blocks = static_cast<int>((m + MLP_THREADS - 1) / MLP_THREADS);
    mlp_predict_kernel<<<blocks, MLP_THREADS, 0, s>>>(d->d_w, d->d_norm, d->d_norm + NF, d->d_px, static_cast<int>(m),
                                                      d->d_py, d->d_pc);
    DCK(cudaGetLastError(), "predict kernel");
    ctx->stats.launches++;
    std::vector<int> c(m);
    DCK(cudaMemcpyAsync(c.data(), d->d_pc, m * sizeof(int), cudaMemcpyDeviceToHost, s), "read choices");
    if (feat_host)
        DCK(cudaMemcpyAsync(feat_host, d->d_px, m * NF * sizeof(float), cudaMemcpyDeviceToHost, s), "read features");
    DCK(host_sync(ctx, s), "synchronise choices");
    for (int64_t i = 0; i < m; ++i) choice[i] = c[i] + 1;
    return BMLP_OK;
}

bool dispatch_trained(const bmlp_ctx* ctx) {
    const Dispatch* d = static_cast<const Dispatch*>(ctx->dispatch);
    return d && d->trained;
}

// Predictions for m host feature rows; pred (m x 4) and choice (m) on host.
bmlp_status dispatch_predict(bmlp_ctx* ctx, const float* feats, int64_t m, float* pred, int32_t* choice,
                             cudaStream_t s) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    if (m <= 0) return BMLP_OK;
    st = pred_buffers(ctx, d, m);
    if (st != BMLP_OK) return st;
    float* dX = d->d_px;
    float* dY = d->d_py;
    int* dC = d->d_pc;
    DCK(cudaMemcpyAsync(dX, feats, m * NF * sizeof(float), cudaMemcpyHostToDevice, s), "copy features");
    const int blocks = static_cast<int>((m + MLP_THREADS - 1) / MLP_THREADS);
    mlp_predict_kernel<<<blocks, MLP_THREADS, 0, s>>>(d->d_w, d->d_norm, d->d_norm + NF, dX, static_cast<int>(m), dY, dC);
    DCK(cudaGetLastError(), "predict kernel");
    std::vector<int> c(m);
    std::vector<float> y(m * NV);
    DCK(cudaMemcpyAsync(y.data(), dY, m * NV * sizeof(float), cudaMemcpyDeviceToHost, s), "read predictions");
    DCK(cudaMemcpyAsync(c.data(), dC, m * sizeof(int), cudaMemcpyDeviceToHost, s), "read choices");
    DCK(host_sync(ctx, s), "synchronise predict");
    if (pred) memcpy(pred, y.data(), y.size() * sizeof(float));
    if (choice)
        for (int64_t i = 0; i < m; ++i) choice[i] = c[i] + 1;  // bmlp_variant numbering
    return BMLP_OK;
}

bmlp_status dispatch_set_params(bmlp_ctx* ctx, const float* params, const float* mu, const float* sig) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    if (params) memcpy(d->master.data(), params, NP * sizeof(float));
    for (int k = 0; k < NF; ++k) {
        if (mu) d->mu[k] = mu[k];
        if (sig) d->sig[k] = sig[k] > 0.f ? sig[k] : 1.f;
    }
    st = upload_params(ctx, d);
    if (st == BMLP_OK) d->trained = true;
    return st;
}

bmlp_status dispatch_get_params(bmlp_ctx* ctx, float* params, float* mu, float* sig) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    if (params) memcpy(params, d->master.data(), NP * sizeof(float));
    for (int k = 0; k < NF; ++k) {
        if (mu) mu[k] = d->mu[k];
        if (sig) sig[k] = d->sig[k];
    }
    return BMLP_OK;
}

bmlp_status dispatch_loss_grad(bmlp_ctx* ctx, const float* X, const float* Y, const uint8_t* C, int64_t m, float* loss,
                               float* grad) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    float *dX = nullptr, *dY = nullptr, *dG = nullptr;
    uint8_t* dC = nullptr;
    if ((st = to_device(ctx, X, m * NF, &dX)) != BMLP_OK) return st;
    if ((st = to_device(ctx, Y, m * NV, &dY)) != BMLP_OK) return st;
    if ((st = to_device(ctx, C, m * NV, &dC)) != BMLP_OK) return st;
    DCK(cudaMalloc(&dG, NP * sizeof(float)), "cudaMalloc(gradient)");
    MlpData md{dX, dY, dC, static_cast<int>(m)};
    mlp_grad_kernel<<<1, MLP_THREADS>>>(d->d_w, d->d_norm, d->d_norm + NF, md, dG, d->d_small);
    DCK(cudaGetLastError(), "gradient kernel");
    DCK(cudaMemcpy(grad, dG, NP * sizeof(float), cudaMemcpyDeviceToHost), "read gradient");
    DCK(cudaMemcpy(loss, d->d_small, sizeof(float), cudaMemcpyDeviceToHost), "read loss");
    cudaFree(dX);
    cudaFree(dY);
    cudaFree(dC);
    cudaFree(dG);
    return BMLP_OK;
}

bmlp_status dispatch_train(bmlp_ctx* ctx, const float* X, const float* Y, const uint8_t* C, int64_t m,
                           const bmlp_train_cfg* cfg, float* final_loss) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    // normalisation from the training features
    for (int k = 0; k < NF; ++k) {
        double s1 = 0, s2 = 0;
        for (int64_t i = 0; i < m; ++i) {
            s1 += X[i * NF + k];
            s2 += static_cast<double>(X[i * NF + k]) * X[i * NF + k];
        }
        const double mean = s1 / m, var = s2 / m - mean * mean;
        d->mu[k] = static_cast<float>(mean);
        d->sig[k] = static_cast<float>(var > 1e-12 ? sqrt(var) : 1.0);
    }
    // He-uniform initialisation from the seed
    std::mt19937_64 rng(cfg->seed);
    auto init = [&](int off, int fan_out, int fan_in) {
        const double lim = sqrt(6.0 / fan_in);
        std::uniform_real_distribution<double> u(-lim, lim);
        for (int i = 0; i < fan_out * fan_in; ++i) d->master[off + i] = static_cast<float>(u(rng));
    };
    std::fill(d->master.begin(), d->master.end(), 0.f);
    init(OW1, NH, NF);
    init(OW2, NH, NH);
    init(OW3, NV, NH);
    if ((st = upload_params(ctx, d)) != BMLP_OK) return st;
    DCK(cudaMemset(d->d_m1, 0, NP * sizeof(float)), "clear Adam state");
    DCK(cudaMemset(d->d_m2, 0, NP * sizeof(float)), "clear Adam state");
    float *dX = nullptr, *dY = nullptr;
    uint8_t* dC = nullptr;
    int* dP = nullptr;
    if ((st = to_device(ctx, X, m * NF, &dX)) != BMLP_OK) return st;
    if ((st = to_device(ctx, Y, m * NV, &dY)) != BMLP_OK) return st;
    if ((st = to_device(ctx, C, m * NV, &dC)) != BMLP_OK) return st;
    DCK(cudaMalloc(&dP, m * sizeof(int)), "cudaMalloc(permutation)");
    MlpData md{dX, dY, dC, static_cast<int>(m)};
    mlp_train_kernel<<<1, MLP_THREADS>>>(d->d_master, d->d_m1, d->d_m2, d->d_w, d->d_norm, d->d_norm + NF, md, dP,
                                         cfg->epochs, cfg->batch > 0 ? cfg->batch : 256, cfg->lr, cfg->weight_decay,
                                         cfg->seed, d->d_small);
    DCK(cudaGetLastError(), "train kernel");
    DCK(cudaDeviceSynchronize(), "train");
    DCK(cudaMemcpy(d->master.data(), d->d_master, NP * sizeof(float), cudaMemcpyDeviceToHost), "read weights");
    if (final_loss) DCK(cudaMemcpy(final_loss, d->d_small, sizeof(float), cudaMemcpyDeviceToHost), "read loss");
    cudaFree(dX);
    cudaFree(dY);
    cudaFree(dC);
    cudaFree(dP);
    d->trained = true;
    return BMLP_OK;
}

bmlp_status dispatch_save(bmlp_ctx* ctx, const char* path) {
    Dispatch* d = nullptr;
    bmlp_status st = dispatch_state(ctx, &d);
    if (st != BMLP_OK) return st;
    FILE* f = fopen(path, "wb");
    if (!f) return set_err(ctx, BMLP_ERR_INVALID_ARG, "cannot write %s", path);
    const char magic[8] = {'B', 'M', 'L', 'P', 'M', 'L', 'P', '1'};
    const int32_t dims[4] = {NF, NH, NV, NP};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(dims, sizeof(dims), 1, f) == 1 &&
              fwrite(d->mu, sizeof(d->mu), 1, f) == 1 && fwrite(d->sig, sizeof(d->sig), 1, f) == 1 &&
              fwrite(d->master.data(), sizeof(float), NP, f) == static_cast<size_t>(NP);
    fclose(f);
    return ok ? BMLP_OK : set_err(ctx, BMLP_ERR_INVALID_ARG, "short write to %s", path);
}

bmlp_status dispatch_load(bmlp_ctx* ctx, const char* path) {
    FILE* f = fopen(path, "rb");
    if (!f) return set_err(ctx, BMLP_ERR_INVALID_ARG, "cannot read %s", path);
    char magic[8];
    int32_t dims[4];
    float mu[NF], sig[NF];
    std::vector<float> p(NP);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "BMLPMLP1", 8) == 0 && fread(dims, sizeof(dims), 1, f) == 1 &&
              dims[0] == NF && dims[1] == NH && dims[2] == NV && dims[3] == NP && fread(mu, sizeof(mu), 1, f) == 1 &&
              fread(sig, sizeof(sig), 1, f) == 1 && fread(p.data(), sizeof(float), NP, f) == static_cast<size_t>(NP);
    fclose(f);
    if (!ok) return set_err(ctx, BMLP_ERR_INVALID_ARG, "%s is not a dispatcher model", path);
    return dispatch_set_params(ctx, p.data(), mu, sig);
}

}  // namespace bmlp
