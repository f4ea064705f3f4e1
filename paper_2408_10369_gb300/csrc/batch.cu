// Grouped batch runner: many independent linear recursive programs of uneven
// sizes (closures, paper Sec. 3.3 program P2, and two-relation compositions,
// Sec. 3.4 Thm. 1) evaluated together.
//
// Per iteration, ONE persistent tensor-core launch (tc_group_kernel) runs the
// squaring step R <- R + R R of every unconverged tensor-core problem over a
// device work list of (problem, tile) items, and one packed launch does the
// same for the problems the autotuner put on packed rows. A single-block
// planner then retires problems whose changed flag stayed 0 (or that reached
// their cap), flips the ping-pong parity of the others, rebuilds both work
// lists and sets the condition of the CUDA graph WHILE node that holds the
// iteration. Encoding, the iteration, the final products of compositions and
// decoding are one graph launch; the host reads back the per-problem
// iteration counts once at the end.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace bmlp {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int TILE = 64;

// ------------------------------------------------------------ encoding --
__device__ __forceinline__ uint32_t src_bits16(const void* in, int fmt, int64_t n, int64_t r, int64_t c0) {
    if (r >= n || c0 >= n) return 0;
    uint32_t m = 0;
    if (fmt == BMLP_FMT_U8) {
        const uint8_t* row = static_cast<const uint8_t*>(in) + r * n;
        for (int x = 0; x < 16; ++x)
            if (c0 + x < n && row[c0 + x] != 0) m |= 1u << x;
    } else {
        const uint64_t w = static_cast<const uint64_t*>(in)[r * ((n + 63) / 64) + (c0 >> 6)];
        m = static_cast<uint32_t>((w >> (c0 & 63)) & 0xFFFFu);
        const int64_t valid = n - c0;
        if (valid < 16) m &= (1u << valid) - 1u;
    }
    return m;
}

__device__ __forceinline__ uint4 expand16(uint32_t m) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t v = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x) v |= (((m >> (4 * q + x)) & 1u) ? static_cast<uint32_t>(BMLP_E4M3_ONE) : 0u) << (8 * x);
        w[q] = v;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// R and R^T (ld x ld E4M3 bytes, zero padding) of one caller matrix, tiles
// strided over the blocks of this problem.
__device__ void encode_e4m3(const void* in, int fmt, int64_t n, uint8_t* R, uint8_t* RT, int64_t ld,
                            uint16_t (*masks)[TILE / 16 + 1]) {
    const int tid = threadIdx.x;
    const int r = tid >> 2, cseg = (tid & 3) * 16;
    const int64_t tiles1 = ld / TILE;
    for (int64_t t = blockIdx.x; t < tiles1 * tiles1; t += gridDim.x) {
        const int64_t row0 = (t / tiles1) * TILE, col0 = (t % tiles1) * TILE;
        const uint32_t m = src_bits16(in, fmt, n, row0 + r, col0 + cseg);
        masks[r][tid & 3] = static_cast<uint16_t>(m);
        *reinterpret_cast<uint4*>(R + (row0 + r) * ld + col0 + cseg) = expand16(m);
        __syncthreads();
        uint32_t tb = 0;
#pragma unroll
        for (int x = 0; x < 16; ++x) tb |= ((masks[cseg + x][r >> 4] >> (r & 15)) & 1u) << x;
        *reinterpret_cast<uint4*>(RT + (col0 + r) * ld + row0 + cseg) = expand16(tb);
        __syncthreads();
    }
}

// blockIdx.y = problem. 256 threads.
__global__ void __launch_bounds__(256) batch_encode_kernel(const GroupProblem* probs) {
    __shared__ uint16_t masks[TILE][TILE / 16 + 1];
    const GroupProblem& g = probs[blockIdx.y];
    if (g.n == 0) return;
    if (g.engine == 0) {
        encode_e4m3(g.kind == 1 ? g.in2 : g.in1, g.fmt, g.n, g.M[0], g.T[0], g.ld, masks);
        if (g.kind == 1) encode_e4m3(g.in1, g.fmt, g.n, g.X, g.R1T, g.ld, masks);  // X is scratch here
    } else {
        const int64_t wpr = (g.n + 63) / 64;
        const int64_t total = g.n * g.ldw;
        for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
             t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
            const int64_t r = t / g.ldw, w = t % g.ldw;
            uint64_t bits = 0;
            if (w < wpr) {
                if (g.fmt == BMLP_FMT_U8) {
                    const uint8_t* row = static_cast<const uint8_t*>(g.in1) + r * g.n + w * 64;
                    const int64_t valid = g.n - w * 64 < 64 ? g.n - w * 64 : 64;
                    for (int k = 0; k < valid; ++k)
                        if (row[k]) bits |= 1ull << k;
                } else {
                    bits = static_cast<const uint64_t*>(g.in1)[r * wpr + w];
                    const int64_t valid = g.n - w * 64;
                    if (valid < 64) bits &= (1ull << valid) - 1ull;
                }
            }
            g.P[0][t] = bits;
        }
    }
}

// ------------------------------------------------------------- planner --
// mode 0: start of the loop (every problem active); mode 1: after a product
// (retire, flip parity, count); mode 2: final products of compositions.
__global__ void __launch_bounds__(1024) batch_plan_kernel(const GroupProblem* probs, const GroupState* st, int nprob,
                                                          int mode, cudaGraphConditionalHandle h, int set_cond) {
    __shared__ int part_tc[1024], part_pk[1024];
    const int t = threadIdx.x;
    const int per = (nprob + 1023) / 1024;
    const int a = t * per, b = min(a + per, nprob);
    int stc = 0, spk = 0;
    for (int p = a; p < b; ++p) {
        const GroupProblem& g = probs[p];
        if (mode == 0) {
            st->parity[p] = 0;
            st->iters[p] = 0;
            st->notconv[p] = 0;
            st->active[p] = g.n > 0 ? 1 : 0;
        } else if (mode == 1) {
            if (st->active[p]) {
                st->iters[p] += 1;
                st->parity[p] ^= 1;
                if (!st->changed[p]) {
                    st->active[p] = 0;
                } else if (st->iters[p] >= g.cap) {
                    st->active[p] = 0;
                    st->notconv[p] = 1;
                }
            }
        } else {
            st->active[p] = (g.kind == 1 && g.n > 0) ? 1 : 0;
        }
        st->changed[p] = 0;
        const int act = st->active[p];
        const int ctc = (act && (mode == 2 || g.engine == 0)) ? g.m_tiles * g.n_tiles : 0;
        const int cpk = (act && mode != 2 && g.engine == 1) ? static_cast<int>(g.n) : 0;
        st->tc_offs[p] = ctc;
        st->pk_offs[p] = cpk;
        stc += ctc;
        spk += cpk;
    }
    part_tc[t] = stc;
    part_pk[t] = spk;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int vt = t >= off ? part_tc[t - off] : 0;
        const int vp = t >= off ? part_pk[t - off] : 0;
        __syncthreads();
        part_tc[t] += vt;
        part_pk[t] += vp;
        __syncthreads();
    }
    int rt = t > 0 ? part_tc[t - 1] : 0, rp = t > 0 ? part_pk[t - 1] : 0;
    for (int p = a; p < b; ++p) {
        const int ct = st->tc_offs[p], cp = st->pk_offs[p];
        st->tc_offs[p] = rt;
        st->pk_offs[p] = rp;
        rt += ct;
        rp += cp;
    }
    if (t == 0) {
        const int tt = part_tc[1023], tp = part_pk[1023];
        st->tc_offs[nprob] = tt;
        st->pk_offs[nprob] = tp;
        *st->tc_total = tt;
        *st->pk_total = tp;
        if (set_cond) cudaGraphSetConditional(h, (tt + tp) > 0 ? 1u : 0u);
    }
}

// ------------------------------------------------ packed squaring step --
// One warp per active row of every packed-engine problem:
// C_i = R_i | OR_{k : R_ik = 1} R_k, chunks of 32 lanes x VEC x 2 words.
template <int VEC>
__global__ void __launch_bounds__(256) packed_group_kernel(const GroupProblem* probs, const GroupState* st, int nprob) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int total = *st->pk_total;
    const int* offs = st->pk_offs;
    constexpr int64_t chunk_words = 64 * VEC;
    for (int64_t item = warp_id; item < total; item += nwarps) {
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const GroupProblem& g = probs[lo];
        const int par = st->parity[lo];
        const int64_t i = item - offs[lo];
        const int64_t ldw = g.ldw;
        const uint64_t* src = g.P[par];
        uint64_t* dst = g.P[par ^ 1];
        const uint64_t* arow = src + i * ldw;
        uint32_t any = 0;
        for (int64_t c0 = 0; c0 < ldw; c0 += chunk_words) {
            uint4 acc[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int64_t w = c0 + 2 * (lane + 32 * v);
                acc[v] = (w < ldw) ? *reinterpret_cast<const uint4*>(arow + w) : make_uint4(0, 0, 0, 0);
            }
            for (int64_t wb = 0; wb < ldw; wb += 32) {
                const uint64_t aw = (wb + lane < ldw) ? arow[wb + lane] : 0ull;
                unsigned m = __ballot_sync(FULL, aw != 0ull);
                while (m) {
                    const int sl = __ffs(m) - 1;
                    m &= m - 1;
                    uint64_t bits = __shfl_sync(FULL, aw, sl);
                    const int64_t kbase = (wb + sl) * 64;
                    while (bits) {
                        const int b0 = __ffsll(static_cast<long long>(bits)) - 1;
                        bits &= bits - 1;
                        const uint64_t* r0 = src + (kbase + b0) * ldw + c0;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const int64_t w = 2 * (lane + 32 * v);
                            if (c0 + w < ldw) {
                                const uint4 x = *reinterpret_cast<const uint4*>(r0 + w);
                                acc[v].x |= x.x;
                                acc[v].y |= x.y;
                                acc[v].z |= x.z;
                                acc[v].w |= x.w;
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int64_t w = c0 + 2 * (lane + 32 * v);
                if (w < ldw) {
                    const uint4 o = *reinterpret_cast<const uint4*>(arow + w);
                    any |= (o.x ^ acc[v].x) | (o.y ^ acc[v].y) | (o.z ^ acc[v].z) | (o.w ^ acc[v].w);
                    *reinterpret_cast<uint4*>(dst + i * ldw + w) = acc[v];
                }
            }
        }
        if (__any_sync(FULL, any != 0) && lane == 0) atomicOr(&st->changed[lo], 1);
    }
}

// I + R2+ for the compositions (diagonal of the closure buffer).
__global__ void batch_compose_prep_kernel(const GroupProblem* probs, const GroupState* st) {
    const GroupProblem& g = probs[blockIdx.y];
    if (g.kind != 1 || g.n == 0) return;
    uint8_t* R = g.M[st->parity[blockIdx.y]];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < g.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        R[i * g.ld + i] = BMLP_E4M3_ONE;
}

// Results into the callers' output buffers.
__global__ void __launch_bounds__(256) batch_decode_kernel(const GroupProblem* probs, const GroupState* st) {
    const GroupProblem& g = probs[blockIdx.y];
    if (g.n == 0) return;
    const int64_t n = g.n, wpr = (n + 63) / 64;
    const int refl = (g.kind == 0) ? g.reflexive : 0;
    const int par = st->parity[blockIdx.y];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g.engine == 0) {
        const uint8_t* src = (g.kind == 1) ? g.X : g.M[par];
        if (g.fmt == BMLP_FMT_U8) {
            uint8_t* out = static_cast<uint8_t*>(g.out);
            for (int64_t t = t0; t < n * n; t += stride) {
                const int64_t i = t / n, j = t % n;
                out[t] = (src[i * g.ld + j] != 0 || (refl && i == j)) ? 1 : 0;
            }
        } else {
            uint64_t* out = static_cast<uint64_t*>(g.out);
            for (int64_t t = t0; t < n * wpr; t += stride) {
                const int64_t i = t / wpr, w = t % wpr;
                const uint8_t* row = src + i * g.ld + w * 64;
                uint64_t bits = 0;
                for (int k = 0; k < 64; ++k)
                    if (row[k]) bits |= 1ull << k;
                const int64_t valid = n - w * 64;
                if (valid < 64) bits &= (1ull << valid) - 1ull;
                if (refl && (i >> 6) == w) bits |= 1ull << (i & 63);
                out[t] = bits;
            }
        }
    } else {
        const uint64_t* P = g.P[par];
        if (g.fmt == BMLP_FMT_U8) {
            uint8_t* out = static_cast<uint8_t*>(g.out);
            for (int64_t t = t0; t < n * n; t += stride) {
                const int64_t i = t / n, j = t % n;
                out[t] = (((P[i * g.ldw + (j >> 6)] >> (j & 63)) & 1ull) || (refl && i == j)) ? 1 : 0;
            }
        } else {
            uint64_t* out = static_cast<uint64_t*>(g.out);
            for (int64_t t = t0; t < n * wpr; t += stride) {
                const int64_t i = t / wpr, w = t % wpr;
                uint64_t bits = P[i * g.ldw + w];
                if (refl && (i >> 6) == w) bits |= 1ull << (i & 63);
                out[t] = bits;
            }
        }
    }
}

// --------------------------------------------------------------- host --
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int bucket_of(int64_t n) {
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

int log2_ceil(int64_t n) {
    int k = 0;
    while ((int64_t(1) << k) < n) ++k;
    return k;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

uint64_t fnv(uint64_t h, const void* data, size_t len) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < len; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

// Cached, instantiated batch graph of a context.
struct BatchCache {
    uint64_t key = 0;
    int nprob = 0;
    std::vector<int> order;          // device slot -> caller index
    GroupProblem* d_probs = nullptr;
    GroupState* d_st = nullptr;
    int* d_ints = nullptr;           // parity | active | iters | changed | notconv | tc_offs | pk_offs | totals
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t ws_bytes = 0;
    std::vector<int> h_iters, h_notconv;
};

void batch_cache_free(bmlp_ctx* ctx) {
    BatchCache* c = static_cast<BatchCache*>(ctx->batch);
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->d_probs) cudaFree(c->d_probs);
    if (c->d_st) cudaFree(c->d_st);
    if (c->d_ints) cudaFree(c->d_ints);
    delete c;
    ctx->batch = nullptr;
}

namespace {

#define BCK(call, what)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, what);   \
    } while (0)

#define BST(call)                      \
    do {                               \
        bmlp_status s_ = (call);       \
        if (s_ != BMLP_OK) return s_;  \
    } while (0)

bmlp_status add_kernel(bmlp_ctx* ctx, cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps,
                       void* func, dim3 grid, dim3 block, size_t smem, void** args) {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = static_cast<unsigned>(smem);
    kp.kernelParams = args;
    kp.extra = nullptr;
    BCK(cudaGraphAddKernelNode(node, g, deps, ndeps, &kp), "cudaGraphAddKernelNode");
    return BMLP_OK;
}

int engine_for(bmlp_ctx* ctx, const bmlp_problem& p, int variant) {
    if (p.kind == BMLP_PROBLEM_COMPOSE) return 0;
    if (p.variant == BMLP_RMS_TC) return 0;
    if (p.variant == BMLP_RMS_PACKED) return 1;
    if (variant == BMLP_RMS_TC) return 0;
    if (variant == BMLP_RMS_PACKED) return 1;
    const int b = bucket_of(p.n);
    if (b < 32 && ctx->tune[b] >= 0) return ctx->tune[b];
    return 0;
}

bmlp_status build_batch(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, int variant, long long wait_cycles,
                        uint64_t key, BatchCache** out) {
    batch_cache_free(ctx);
    BatchCache* c = new BatchCache();
    ctx->batch = c;
    c->key = key;
    c->nprob = static_cast<int>(count);
    const int np = c->nprob;
    // order: most expensive first (the work lists are then longest-first)
    c->order.resize(np);
    for (int i = 0; i < np; ++i) c->order[i] = i;
    std::stable_sort(c->order.begin(), c->order.end(),
                     [&](int a, int b) { return probs[a].n > probs[b].n; });
    std::vector<GroupProblem> hp(np);
    std::vector<size_t> offsets(np);
    size_t total = 0;
    auto take = [&](size_t bytes) {
        size_t o = total;
        total += round_up(static_cast<int64_t>(bytes), 1024);
        return o;
    };
    std::vector<size_t> offM0(np), offM1(np), offT0(np), offT1(np), offX(np), offR1T(np), offP0(np), offP1(np);
    for (int s = 0; s < np; ++s) {
        const bmlp_problem& p = probs[c->order[s]];
        GroupProblem& g = hp[s];
        memset(&g, 0, sizeof(g));
        g.n = p.n;
        g.kind = p.kind;
        g.fmt = p.fmt;
        g.reflexive = p.reflexive;
        g.in1 = p.R1;
        g.in2 = p.R2;
        g.out = p.out;
        g.engine = engine_for(ctx, p, variant);
        g.cap = log2_ceil(p.n > 1 ? p.n : 2) + 2;
        if (p.n == 0) continue;
        if (g.engine == 0) {
            g.ld = round_up(p.n, TC_PAD);
            g.m_tiles = static_cast<int32_t>(g.ld / TC_BM);
            g.n_tiles = static_cast<int32_t>(g.ld / TC_BN);
            g.k_blocks = static_cast<int32_t>(g.ld / TC_BK);
            const size_t mat = static_cast<size_t>(g.ld * g.ld);
            offM0[s] = take(mat);
            offM1[s] = take(mat);
            offT0[s] = take(mat);
            offT1[s] = take(mat);
            if (p.kind == BMLP_PROBLEM_COMPOSE) {
                offX[s] = take(mat);
                offR1T[s] = take(mat);
            }
        } else {
            g.ldw = round_up((p.n + 63) / 64, 2);
            const size_t bytes = static_cast<size_t>(p.n * g.ldw * 8);
            offP0[s] = take(bytes);
            offP1[s] = take(bytes);
        }
    }
    void* base = nullptr;
    BST(ws_get(ctx, WS_BATCH, total, &base));
    c->ws_bytes = total;
    uint8_t* b8 = static_cast<uint8_t*>(base);
    for (int s = 0; s < np; ++s) {
        GroupProblem& g = hp[s];
        if (g.n == 0) continue;
        if (g.engine == 0) {
            g.M[0] = b8 + offM0[s];
            g.M[1] = b8 + offM1[s];
            g.T[0] = b8 + offT0[s];
            g.T[1] = b8 + offT1[s];
            for (int par = 0; par < 2; ++par) {
                BST(make_tmap(ctx, &g.mapA[par], g.M[par], g.ld, g.ld, g.ld, TC_BM));
                BST(make_tmap(ctx, &g.mapB[par], g.T[par], g.ld, g.ld, g.ld, TC_BN));
            }
            if (g.kind == 1) {
                g.X = b8 + offX[s];
                g.R1T = b8 + offR1T[s];
                BST(make_tmap(ctx, &g.mapBF, g.R1T, g.ld, g.ld, g.ld, TC_BN));
            }
        } else {
            g.P[0] = reinterpret_cast<uint64_t*>(b8 + offP0[s]);
            g.P[1] = reinterpret_cast<uint64_t*>(b8 + offP1[s]);
        }
    }
    // device copies
    BCK(cudaMalloc(&c->d_probs, sizeof(GroupProblem) * (np > 0 ? np : 1)), "cudaMalloc(batch problems)");
    BCK(cudaMemcpy(c->d_probs, hp.data(), sizeof(GroupProblem) * np, cudaMemcpyHostToDevice), "copy batch problems");
    const size_t nints = static_cast<size_t>(5 * np + 2 * (np + 1) + 2);
    BCK(cudaMalloc(&c->d_ints, sizeof(int) * nints), "cudaMalloc(batch state)");
    BCK(cudaMemset(c->d_ints, 0, sizeof(int) * nints), "clear batch state");
    GroupState hs;
    int* q = c->d_ints;
    hs.parity = q; q += np;
    hs.active = q; q += np;
    hs.iters = q; q += np;
    hs.changed = q; q += np;
    hs.notconv = q; q += np;
    hs.tc_offs = q; q += np + 1;
    hs.pk_offs = q; q += np + 1;
    hs.tc_total = q; q += 1;
    hs.pk_total = q; q += 1;
    BCK(cudaMalloc(&c->d_st, sizeof(GroupState)), "cudaMalloc(batch state)");
    BCK(cudaMemcpy(c->d_st, &hs, sizeof(GroupState), cudaMemcpyHostToDevice), "copy batch state");
    c->h_iters.assign(np, 0);
    c->h_notconv.assign(np, 0);

    // ---- graph
    BCK(prepare_tc_group(), "tensor-core group kernel attributes");
    BCK(cudaGraphCreate(&c->graph, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle h;
    BCK(cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault), "conditional handle");
    GroupProblem* dp = c->d_probs;
    GroupState* ds = c->d_st;
    int nprob = np;
    int* err = ctx->d_ctl + CTL_ERROR;
    long long wc = wait_cycles;
    int mode0 = 0, mode1 = 1, mode2 = 2, phase0 = 0, phase1 = 1, set0 = 0, set1 = 1;
    const int sms = ctx->sm_count;
    const unsigned gy = static_cast<unsigned>(np > 0 ? np : 1);
    cudaGraphNode_t n_enc, n_init, n_while, n_prep, n_plan2, n_final, n_dec;
    {
        void* a[] = {&dp};
        BST(add_kernel(ctx, c->graph, &n_enc, nullptr, 0, reinterpret_cast<void*>(&batch_encode_kernel),
                       dim3(64, gy), dim3(256), 0, a));
    }
    {
        void* a[] = {&dp, &ds, &nprob, &mode0, &h, &set0};
        BST(add_kernel(ctx, c->graph, &n_init, &n_enc, 1, reinterpret_cast<void*>(&batch_plan_kernel), dim3(1),
                       dim3(1024), 0, a));
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    BCK(cudaGraphAddNode(&n_while, c->graph, &n_init, nullptr, 1, &cp), "while node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    {
        // the two engines touch disjoint problems, so their launches may overlap
        cudaGraphNode_t n_eng[2], n_plan;
        void* a[] = {&dp, &ds, &nprob, &phase0, &err, &wc};
        BST(add_kernel(ctx, body, &n_eng[0], nullptr, 0, tc_group_kernel_ptr(), dim3(sms), dim3(TC_THREADS),
                       tc_smem_bytes(), a));
        void* b[] = {&dp, &ds, &nprob};
        BST(add_kernel(ctx, body, &n_eng[1], nullptr, 0, reinterpret_cast<void*>(&packed_group_kernel<4>),
                       dim3(sms * 8), dim3(256), 0, b));
        void* d[] = {&dp, &ds, &nprob, &mode1, &h, &set1};
        BST(add_kernel(ctx, body, &n_plan, n_eng, 2, reinterpret_cast<void*>(&batch_plan_kernel), dim3(1),
                       dim3(1024), 0, d));
    }
    {
        void* a[] = {&dp, &ds};
        BST(add_kernel(ctx, c->graph, &n_prep, &n_while, 1, reinterpret_cast<void*>(&batch_compose_prep_kernel),
                       dim3(8, gy), dim3(256), 0, a));
    }
    {
        void* a[] = {&dp, &ds, &nprob, &mode2, &h, &set0};
        BST(add_kernel(ctx, c->graph, &n_plan2, &n_prep, 1, reinterpret_cast<void*>(&batch_plan_kernel), dim3(1),
                       dim3(1024), 0, a));
    }
    {
        void* a[] = {&dp, &ds, &nprob, &phase1, &err, &wc};
        BST(add_kernel(ctx, c->graph, &n_final, &n_plan2, 1, tc_group_kernel_ptr(), dim3(sms), dim3(TC_THREADS),
                       tc_smem_bytes(), a));
    }
    {
        void* a[] = {&dp, &ds};
        BST(add_kernel(ctx, c->graph, &n_dec, &n_final, 1, reinterpret_cast<void*>(&batch_decode_kernel),
                       dim3(64, gy), dim3(256), 0, a));
    }
    BCK(cudaGraphInstantiate(&c->exec, c->graph, 0), "cudaGraphInstantiate");
    *out = c;
    return BMLP_OK;
}

uint64_t batch_key(const bmlp_problem* probs, int64_t count, int variant, const int* tune) {
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &count, sizeof(count));
    h = fnv(h, &variant, sizeof(variant));
    h = fnv(h, tune, sizeof(int) * 32);
    for (int64_t i = 0; i < count; ++i) h = fnv(h, &probs[i], sizeof(bmlp_problem));
    return h;
}

}  // namespace

bmlp_status batch_run_impl(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, int variant,
                           long long wait_cycles, int32_t* iters_out, cudaStream_t s) {
    for (int64_t i = 0; i < count; ++i) {
        const bmlp_problem& p = probs[i];
        if (p.kind != BMLP_PROBLEM_CLOSURE && p.kind != BMLP_PROBLEM_COMPOSE)
            return set_err(ctx, BMLP_ERR_INVALID_ARG, "problem %lld: bad kind %d", (long long)i, p.kind);
        if (p.fmt != BMLP_FMT_U8 && p.fmt != BMLP_FMT_PACKED64)
            return set_err(ctx, BMLP_ERR_INVALID_ARG, "problem %lld: bad format %d", (long long)i, p.fmt);
        if (p.n < 0 || p.n > (int64_t(1) << 17))
            return set_err(ctx, BMLP_ERR_INVALID_ARG, "problem %lld: n out of range", (long long)i);
        if (p.n == 0) continue;
        if (!p.R1 || !p.out || (p.kind == BMLP_PROBLEM_COMPOSE && !p.R2))
            return set_err(ctx, BMLP_ERR_INVALID_ARG, "problem %lld: null pointer", (long long)i);
        if (!on_device(p.R1) || !on_device(p.out) || (p.kind == BMLP_PROBLEM_COMPOSE && !on_device(p.R2)))
            return set_err(ctx, BMLP_ERR_INVALID_ARG, "problem %lld: matrices must be device memory", (long long)i);
    }
    if (count > (int64_t(1) << 20)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "more than 2^20 problems");
    const uint64_t key = batch_key(probs, count, variant, ctx->tune);
    BatchCache* c = static_cast<BatchCache*>(ctx->batch);
    if (c == nullptr || c->key != key) BST(build_batch(ctx, probs, count, variant, wait_cycles, key, &c));
    BCK(cudaMemsetAsync(ctx->d_ctl, 0, CTL_WORDS * sizeof(int), s), "reset flags");
    ctx->stats.n_pad = static_cast<int64_t>(c->ws_bytes);
    BCK(cudaGraphLaunch(c->exec, s), "cudaGraphLaunch");
    const int np = c->nprob;
    BCK(cudaMemcpyAsync(c->h_iters.data(), c->d_ints + 2 * np, sizeof(int) * np, cudaMemcpyDeviceToHost, s),
        "read iterations");
    BCK(cudaMemcpyAsync(c->h_notconv.data(), c->d_ints + 4 * np, sizeof(int) * np, cudaMemcpyDeviceToHost, s),
        "read convergence");
    BCK(cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, CTL_WORDS * sizeof(int), cudaMemcpyDeviceToHost, s), "read flags");
    BCK(cudaStreamSynchronize(s), "synchronise batch");
    if (ctx->h_ctl[CTL_ERROR] != 0)
        return set_err(ctx, BMLP_ERR_TIMEOUT, "in-kernel wait timed out (code 0x%x)", ctx->h_ctl[CTL_ERROR]);
    int maxit = 0, bad = 0;
    for (int sl = 0; sl < np; ++sl) {
        const int i = c->order[sl];
        if (iters_out) iters_out[i] = c->h_iters[sl];
        maxit = std::max(maxit, c->h_iters[sl]);
        bad |= c->h_notconv[sl];
    }
    ctx->stats.iterations = maxit;
    ctx->stats.launches += 4 + 3 * maxit;
    ctx->stats.product_launches += maxit + 1;
    if (bad) return set_err(ctx, BMLP_ERR_NOT_CONVERGED, "a problem did not converge within its cap");
    return BMLP_OK;
}

}  // namespace bmlp
