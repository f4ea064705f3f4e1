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
//
// Problems large enough to fill the GPU on their own (n >= solo_n) run in the
// same graph as device-driven single-problem pipelines, one after another:
// squarings on word-indexed bit rows while the next one costs less than a
// tensor-core product (the same cost model and the same switch as the
// single-problem path, decided by a one-thread kernel that sets the
// condition of a WHILE node), then squarings on packed E2M1 operands on the
// tensor cores in a second WHILE node, two products per iteration with a
// guard word so that the second is skipped once the first changed nothing,
// then the decode (closures) or I + R2+ and the final product with R1
// (compositions). No host round trip per squaring.
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
            // frontier-engine problems (engine 2) take no part in the squaring loop; their closure rows are
            // written into P[1] by the grouped frontier launch
            st->parity[p] = g.engine == 2 ? 1 : 0;
            st->iters[p] = 0;
            st->notconv[p] = 0;
            st->active[p] = (g.n > 0 && g.engine != 2) ? 1 : 0;
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

// ------------------------------------------- device-driven large problems --
// Control words of one large problem (ints; 64-bit words at SW_COST, SW_SMP and SW_TSTAT, 8-byte aligned).
enum SoloWord : int {
    SW_ITERS = 0,     // squarings issued so far
    SW_NOTDONE = 1,   // 1 while the closure is not finished on bit rows
    SW_NOTCONV = 2,   // stopped at the cap while still changing
    SW_CHANGED = 3,   // set by the squaring kernels
    SW_GC = 4,        // guard of the first tensor-core product of a loop iteration
    SW_G1 = 5,        // guard of the second
    SW_TCHANGED = 6,  // set by a restricted squaring that found new ones
    SW_RES = 7,       // 1: a restricted squaring left the closure in Q1 (else Q0 holds it)
    SW_COST = 8,      // word ORs of the next bit-row squaring: total, largest row (2 x u64)
    SW_THIN_GO = 12,  // the restricted squaring is cheaper than a product (set inside its statistics' IF)
    SW_STOP = 13,     // a restricted squaring ended the loop
    SW_SMP = 16,      // the row sample after a product (2 x u64, thin.cu)
    SW_TSTAT = 20,    // the restricted squaring's statistics (6 x u64, thin.cu)
    SW_WORDS = 32
};

// dst = src, 16 bytes per thread and step (sizes are multiples of 16 bytes).
__global__ void solo_copy_kernel(uint4* __restrict__ dst, const uint4* __restrict__ src, int64_t n16) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[i] = src[i];
}

__global__ void solo_init_kernel(int* w) {
    for (int i = 0; i < SW_WORDS; ++i) w[i] = 0;
    w[SW_NOTDONE] = 1;
}

// After the cost pass on the current bit rows: stop if the last squaring changed nothing (the closure is done),
// hand over to the tensor cores if the next squaring is predicted dearer than a tensor-core product or would use
// the last product the cap allows, else run it (same rule as the single-problem path).
__global__ void solo_rows_decide_kernel(int* w, int cap, int first, double step_s, double s_word, double s_row,
                                        double limit, cudaGraphConditionalHandle h) {
    unsigned long long* cost = reinterpret_cast<unsigned long long*>(w + SW_COST);
    if (!first) {
        w[SW_ITERS] += 1;
        if (!w[SW_CHANGED]) {
            w[SW_NOTDONE] = 0;
            cudaGraphSetConditional(h, 0u);
            return;
        }
    }
    const double t = step_s + fmax(static_cast<double>(cost[0]) * s_word, static_cast<double>(cost[1]) * s_row);
    if (w[SW_ITERS] + 1 >= cap || t > limit) {
        cudaGraphSetConditional(h, 0u);
        return;
    }
    w[SW_CHANGED] = 0;
    cost[0] = 0;
    cost[1] = 0;
    cudaGraphSetConditional(h, 1u);
}

__global__ void solo_mid_kernel(int* w, cudaGraphConditionalHandle h) {
    const int go = w[SW_NOTDONE];
    w[SW_GC] = go;
    w[SW_G1] = 0;
    w[SW_CHANGED] = 0;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// After tensor-core product `half` (0: Q0 -> Q1, 1: Q1 -> Q0) of a loop iteration. A product that changed nothing
// wrote R' = R, so both buffers hold the closure and either may be decoded.
__global__ void solo_tc_decide_kernel(int* w, int cap, int half, cudaGraphConditionalHandle h) {
    if (!w[half == 0 ? SW_GC : SW_G1]) return;  // that product was skipped
    w[SW_ITERS] += 1;
    bool go = w[SW_CHANGED] != 0;
    w[SW_CHANGED] = 0;
    if (go && w[SW_ITERS] >= cap) {
        w[SW_NOTCONV] = 1;
        go = false;
    }
    if (half == 0) {
        w[SW_G1] = go ? 1 : 0;
        if (!go) {
            w[SW_GC] = 0;
            cudaGraphSetConditional(h, 0u);
        }
    } else {
        w[SW_G1] = 0;
        if (!go) w[SW_GC] = 0;
        cudaGraphSetConditional(h, go ? 1u : 0u);
    }
}

// After tensor-core product `half` (its R in Q[half ^ 1]): whether the next squaring may run only on the rows and
// columns of R that still hold zeros. Only while the loop goes on (the next product's guard is set) and when the
// sampled rows that reach at least n / 2 constants agree in count within spread x n; the sample is cleared for the
// next product. The statistics' IF reads hT; the squaring's IF stays off until they say it is cheaper.
__global__ void solo_thin_gate_kernel(int* w, int half, int64_t n, double spread, cudaGraphConditionalHandle hT) {
    unsigned long long* sm = reinterpret_cast<unsigned long long*>(w + SW_SMP);
    const int next = half == 0 ? w[SW_G1] : w[SW_GC];
    const double sp = static_cast<double>(sm[0]) - (static_cast<double>(n) - static_cast<double>(sm[1]));
    const bool go = next != 0 && sm[0] > 0 && sp <= spread * static_cast<double>(n);
    sm[0] = 0;
    sm[1] = 0;
    w[SW_THIN_GO] = 0;
    cudaGraphSetConditional(hT, go ? 1u : 0u);
}

// Inside the statistics' IF: the restricted squaring's cost by the bit-row model (the word ORs over the GPU, or one
// warp's heaviest list entry) against a tensor-core product, as on the host loop.
__global__ void solo_thin_decide_kernel(int* w, int64_t ldw, double fixed_s, double s_word, double s_row, double limit) {
    const unsigned long long* st = reinterpret_cast<const unsigned long long*>(w + SW_TSTAT);
    const double words = static_cast<double>(st[2] + st[3]) * static_cast<double>(ldw);
    const double row_words = static_cast<double>(st[4] > st[5] ? st[4] : st[5]) * static_cast<double>(ldw);
    const double t = fixed_s + fmax(words * s_word, row_words * s_row);
    w[SW_THIN_GO] = t < limit ? 1 : 0;
    w[SW_TCHANGED] = 0;
}

__global__ void solo_thin_arm_kernel(const int* w, cudaGraphConditionalHandle hT2) {
    cudaGraphSetConditional(hT2, w[SW_THIN_GO] ? 1u : 0u);
}

// After a restricted squaring that followed product `half` (R in Q[half ^ 1], updated in place): one more squaring
// counted; if it changed nothing that buffer holds the closure, and at the cap while changing the loop stops
// unconverged; either way the guards go off and the loop-control kernel ends the loop.
__global__ void solo_thin_post_kernel(int* w, int half, int cap) {
    w[SW_ITERS] += 1;
    bool stop = false;
    if (!w[SW_TCHANGED]) {
        stop = true;
    } else if (w[SW_ITERS] >= cap) {
        w[SW_NOTCONV] = 1;
        stop = true;
    }
    if (stop) {
        w[SW_RES] = half ^ 1;
        w[SW_GC] = 0;
        w[SW_G1] = 0;
        w[SW_STOP] = 1;
    }
    w[SW_THIN_GO] = 0;
}

__global__ void solo_loop_ctl_kernel(const int* w, cudaGraphConditionalHandle hC) {
    if (w[SW_STOP]) cudaGraphSetConditional(hC, 0u);
}

// After the tensor-core loop: the closure into Q0 when a restricted squaring left it in Q1 (16 bytes per thread).
__global__ void solo_result_copy_kernel(const int* w, uint4* __restrict__ q0, const uint4* __restrict__ q1, int64_t n16) {
    if (w[SW_RES] != 1) return;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        q0[i] = q1[i];
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
    FrontierJob* d_jobs = nullptr;   // closures by frontier expansion (engine 2), then a 64-bit row counter
    std::vector<int> solo;           // caller indices of the device-driven large problems, in run order
    int* d_solo = nullptr;           // SW_WORDS control words per large problem
    std::vector<int> h_solo;
};

void batch_cache_free(bmlp_ctx* ctx) {
    BatchCache* c = static_cast<BatchCache*>(ctx->batch);
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->d_probs) cudaFree(c->d_probs);
    if (c->d_st) cudaFree(c->d_st);
    if (c->d_ints) cudaFree(c->d_ints);
    if (c->d_solo) cudaFree(c->d_solo);
    if (c->d_jobs) cudaFree(c->d_jobs);
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

// 0: tensor-core squarings; 1: squarings on packed rows; 2: frontier expansion of every row (closures only).
int engine_for(bmlp_ctx* ctx, const bmlp_problem& p, int variant) {
    if (p.kind == BMLP_PROBLEM_COMPOSE) return 0;
    const int v = p.variant ? p.variant : variant;
    if (v == BMLP_RMS_TC || v == BMLP_SMP_TC) return 0;
    if (v == BMLP_RMS_PACKED) return 1;
    if (v == BMLP_SMP_PACKED) return 2;
    const int b = bucket_of(p.n);
    if (b < 32 && ctx->tune[b] >= 0) return ctx->tune[b];
    return 0;
}

// Captures the grouped frontier launches into the batch graph after `after`; *tail receives the nodes the next
// node must depend on.
bmlp_status add_frontier_chain(bmlp_ctx* ctx, BatchCache* c, int njobs, int64_t max_n, int64_t max_ldw, int64_t total,
                               cudaGraphNode_t after, std::vector<cudaGraphNode_t>* tail) {
    cudaStream_t cs = nullptr;
    BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    struct Stream {
        cudaStream_t a;
        ~Stream() { cudaStreamDestroy(a); }
    } guard_stream{cs};
    BCK(cudaStreamBeginCaptureToGraph(cs, c->graph, &after, nullptr, 1, cudaStreamCaptureModeRelaxed),
        "begin capture of the frontier launches");
    auto* counter = reinterpret_cast<unsigned long long*>(c->d_jobs + njobs);
    cudaError_t e = launch_frontier_group(c->d_jobs, njobs, max_n, max_ldw, total, counter, ctx->sm_count, cs);
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &nd);
    if (e == cudaSuccess) tail->assign(deps, deps + nd);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) return cuda_err(ctx, e != cudaSuccess ? e : e2, "frontier launches");
    return BMLP_OK;
}

bool is_solo(const bmlp_problem& p, int variant, int64_t solo_n) {
    if (solo_n <= 0 || p.n < solo_n) return false;
    if (p.kind == BMLP_PROBLEM_COMPOSE) return true;
    const int v = p.variant ? p.variant : variant;
    return v == BMLP_AUTO || v == BMLP_RMS_TC;
}

bmlp_status build_solo(bmlp_ctx* ctx, BatchCache* c, const bmlp_problem* probs, long long wait_cycles,
                       const cudaGraphNode_t* after, size_t nafter);

bmlp_status build_batch(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, int variant, long long wait_cycles,
                        uint64_t key, int64_t solo_n, BatchCache** out) {
    batch_cache_free(ctx);
    BatchCache* c = new BatchCache();
    ctx->batch = c;
    c->key = key;
    // large problems first, as device-driven pipelines after the grouped part; the rest grouped, most expensive
    // first (the work lists are then longest-first)
    for (int64_t i = 0; i < count; ++i)
        if (is_solo(probs[i], variant, solo_n)) c->solo.push_back(static_cast<int>(i));
        else c->order.push_back(static_cast<int>(i));
    std::stable_sort(c->solo.begin(), c->solo.end(), [&](int a, int b) { return probs[a].n > probs[b].n; });
    c->nprob = static_cast<int>(c->order.size());
    const int np = c->nprob;
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
    std::vector<size_t> offPT(np), offPtr[2], offIdx[2], offVal[2];
    for (int m = 0; m < 2; ++m) {
        offPtr[m].resize(np);
        offIdx[m].resize(np);
        offVal[m].resize(np);
    }
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
            if (g.engine == 2) {  // R^T and the word indexes of R and R^T (entries sized for the dense worst case)
                offPT[s] = take(bytes);
                for (int m = 0; m < 2; ++m) {
                    offPtr[m][s] = take(static_cast<size_t>((p.n + 2) * 8));
                    offIdx[m][s] = take(static_cast<size_t>(p.n * g.ldw * 4));
                    offVal[m][s] = take(bytes);
                }
            }
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
    // frontier jobs (engine 2): every row of the closure as one query, all jobs in one launch
    std::vector<FrontierJob> jobs;
    int64_t fr_total = 0, fr_max_n = 0, fr_max_ldw = 0;
    for (int s = 0; s < np; ++s) {
        const GroupProblem& g = hp[s];
        if (g.n == 0 || g.engine != 2) continue;
        FrontierJob j{};
        j.P = g.P[0];
        j.PT = reinterpret_cast<uint64_t*>(b8 + offPT[s]);
        j.wptr = reinterpret_cast<int64_t*>(b8 + offPtr[0][s]);
        j.widx = reinterpret_cast<int32_t*>(b8 + offIdx[0][s]);
        j.wval = reinterpret_cast<uint64_t*>(b8 + offVal[0][s]);
        j.wptrT = reinterpret_cast<int64_t*>(b8 + offPtr[1][s]);
        j.widxT = reinterpret_cast<int32_t*>(b8 + offIdx[1][s]);
        j.wvalT = reinterpret_cast<uint64_t*>(b8 + offVal[1][s]);
        j.out = g.P[1];
        j.n = g.n;
        j.ldw = g.ldw;
        j.first = fr_total;
        j.levels = nullptr;  // set below, once the state array exists
        jobs.push_back(j);
        fr_total += g.n;
        fr_max_n = std::max(fr_max_n, g.n);
        fr_max_ldw = std::max(fr_max_ldw, g.ldw);
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
    if (!jobs.empty()) {
        size_t k = 0;
        for (int s = 0; s < np; ++s)
            if (hp[s].n > 0 && hp[s].engine == 2) jobs[k++].levels = hs.iters + s;
        BCK(cudaMalloc(&c->d_jobs, sizeof(FrontierJob) * jobs.size() + sizeof(unsigned long long)),
            "cudaMalloc(frontier jobs)");
        BCK(cudaMemcpy(c->d_jobs, jobs.data(), sizeof(FrontierJob) * jobs.size(), cudaMemcpyHostToDevice),
            "copy frontier jobs");
    }
    c->h_iters.assign(np, 0);
    c->h_notconv.assign(np, 0);

    // ---- graph
    BCK(prepare_tc_group(), "tensor-core group kernel attributes");
    BCK(cudaGraphCreate(&c->graph, 0), "cudaGraphCreate");
    if (np == 0) {
        BST(build_solo(ctx, c, probs, wait_cycles, nullptr, 0));
        BCK(cudaGraphInstantiate(&c->exec, c->graph, 0), "cudaGraphInstantiate");
        *out = c;
        return BMLP_OK;
    }
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
    // the closures by frontier expansion: one chain of grouped launches after the planner's start
    std::vector<cudaGraphNode_t> before_while{n_init};
    if (!jobs.empty()) BST(add_frontier_chain(ctx, c, static_cast<int>(jobs.size()), fr_max_n, fr_max_ldw, fr_total,
                                              n_init, &before_while));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    BCK(cudaGraphAddNode(&n_while, c->graph, before_while.data(), nullptr, before_while.size(), &cp), "while node");
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
    if (!c->solo.empty()) BST(build_solo(ctx, c, probs, wait_cycles, &n_dec, 1));
    BCK(cudaGraphInstantiate(&c->exec, c->graph, 0), "cudaGraphInstantiate");
    *out = c;
    return BMLP_OK;
}

// Adds a conditional WHILE node after the current capture dependencies of `cs` and returns its body graph; the
// capture of `cs` continues after the node.
bmlp_status add_conditional(bmlp_ctx* ctx, cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            cudaGraph_t* body) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    BCK(cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, nullptr, &nd), "capture info");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    BCK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp), "conditional node");
    BCK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
        "capture dependencies");
    *body = cp.conditional.phGraph_out[0];
    return BMLP_OK;
}

bmlp_status add_while(bmlp_ctx* ctx, cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    return add_conditional(ctx, cs, h, cudaGraphCondTypeWhile, body);
}

// The large problems as device-driven single-problem pipelines, one after another (they share one scratch sized
// for the largest), captured into the batch graph after `after`.
bmlp_status build_solo(bmlp_ctx* ctx, BatchCache* c, const bmlp_problem* probs, long long wait_cycles,
                       const cudaGraphNode_t* after, size_t nafter) {
    const int ns = static_cast<int>(c->solo.size());
    int64_t nmax = 0;
    bool any_compose = false;
    for (int i : c->solo) {
        nmax = std::max(nmax, probs[i].n);
        any_compose |= probs[i].kind == BMLP_PROBLEM_COMPOSE;
    }
    const int64_t ldw_max = round_up((nmax + 63) / 64, 2);
    const int64_t np_max = round_up(nmax, TC_PAD);
    const size_t pk = static_cast<size_t>(nmax * ldw_max * 8);
    const size_t q = static_cast<size_t>(np_max * np_max / 2);
    size_t total = 0;
    auto take = [&](size_t bytes) {
        size_t o = total;
        total += round_up(static_cast<int64_t>(bytes), 1024);
        return o;
    };
    const size_t oP0 = take(pk), oP1 = take(pk), oPtr = take(static_cast<size_t>((nmax + 2) * 8)),
                 oIdx = take(static_cast<size_t>(nmax * ldw_max * 4)), oVal = take(pk);
    size_t oQ[2], oQT[2];
    for (int k = 0; k < 2; ++k) {
        oQ[k] = take(q);
        oQT[k] = take(q);
    }
    size_t oM0 = 0;
    if (any_compose) oM0 = take(q);  // a composition's final product: scratch for the transposed output
    // the squaring restricted to the rows and columns holding zeros: bit rows of R and R^T (written by the 4-bit
    // squarings' epilogue), its computed rows, and its counts and lists
    const bool thin_any = thin_is_enabled();
    const int64_t ldwt_max = np_max / 64;
    size_t oTP = 0, oTPT = 0, oTT = 0, oTAux = 0;
    if (thin_any) {
        const size_t bits = static_cast<size_t>(np_max * ldwt_max * 8);
        oTP = take(bits);
        oTPT = take(bits);
        oTT = take(2 * bits);
        oTAux = take(static_cast<size_t>(2 * nmax * 8 + (ldwt_max + 1) * 8 + 2 * nmax * 4));
    }
    void* base = nullptr;
    BST(ws_get(ctx, WS_SOLO, total, &base));
    uint8_t* b8 = static_cast<uint8_t*>(base);
    uint64_t* P0 = reinterpret_cast<uint64_t*>(b8 + oP0);
    uint64_t* P1 = reinterpret_cast<uint64_t*>(b8 + oP1);
    int64_t* wptr = reinterpret_cast<int64_t*>(b8 + oPtr);
    int32_t* widx = reinterpret_cast<int32_t*>(b8 + oIdx);
    uint64_t* wval = reinterpret_cast<uint64_t*>(b8 + oVal);
    uint8_t* Q[2] = {b8 + oQ[0], b8 + oQ[1]};
    uint8_t* QT[2] = {b8 + oQT[0], b8 + oQT[1]};
    uint8_t* M0 = b8 + oM0;
    uint64_t* TP = reinterpret_cast<uint64_t*>(b8 + oTP);
    uint64_t* TPT = reinterpret_cast<uint64_t*>(b8 + oTPT);
    uint64_t* TT = reinterpret_cast<uint64_t*>(b8 + oTT);
    int64_t* t_rowcnt = reinterpret_cast<int64_t*>(b8 + oTAux);
    int64_t* t_colcnt = t_rowcnt + nmax;
    uint64_t* t_bmask = reinterpret_cast<uint64_t*>(t_colcnt + nmax);
    int32_t* t_blist = reinterpret_cast<int32_t*>(t_bmask + ldwt_max + 1);
    int32_t* t_rlist = t_blist + nmax;
    BCK(cudaMalloc(&c->d_solo, sizeof(int) * SW_WORDS * ns), "cudaMalloc(large-problem state)");
    BCK(cudaMemset(c->d_solo, 0, sizeof(int) * SW_WORDS * ns), "clear large-problem state");
    c->h_solo.assign(static_cast<size_t>(SW_WORDS * ns), 0);

    cudaStream_t cs = nullptr, cb = nullptr, cc = nullptr;
    BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    cudaError_t ce = cudaStreamCreateWithFlags(&cb, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&cc, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
        cudaStreamDestroy(cs);
        if (cb) cudaStreamDestroy(cb);
        return cuda_err(ctx, ce, "capture stream");
    }
    struct Streams {
        cudaStream_t a, b, c;
        ~Streams() {
            cudaStreamDestroy(a);
            cudaStreamDestroy(b);
            cudaStreamDestroy(c);
        }
    } guard_streams{cs, cb, cc};
    BCK(cudaStreamBeginCaptureToGraph(cs, c->graph, after, nullptr, nafter, cudaStreamCaptureModeRelaxed),
        "begin capture of the large problems");
    bmlp_status status = BMLP_OK;
    auto fail = [&](bmlp_status st) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cs, &g);
        cudaGetLastError();
        return st;
    };
#define SCK(call, what)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return fail(cuda_err(ctx, e_, what));      \
    } while (0)
#define SST(call)                                  \
    do {                                           \
        bmlp_status s_ = (call);                   \
        if (s_ != BMLP_OK) return fail(s_);        \
    } while (0)
    const int sms = ctx->sm_count;
    const double s_word = bitrow_s_per_word(), s_row = bitrow_row_s_per_word(), step_s = bitrow_step_s();
    for (int k = 0; k < ns; ++k) {
        const bmlp_problem& p = probs[c->solo[k]];
        int* w = c->d_solo + SW_WORDS * k;
        const int64_t n = p.n, ldw = round_up((n + 63) / 64, 2), n_pad = round_up(n, TC_PAD), ld4 = n_pad / 2;
        const int cap = log2_ceil(n > 1 ? n : 2) + 2;
        const void* src = p.kind == BMLP_PROBLEM_COMPOSE ? p.R2 : p.R1;
        const double limit = tc4_product_s(n_pad);
        // ---- squarings on word-indexed bit rows while they are cheaper than a tensor-core product
        solo_init_kernel<<<1, 1, 0, cs>>>(w);
        if (p.fmt == BMLP_FMT_U8)
            launch_u8_to_packed(static_cast<const uint8_t*>(src), n, P0, ldw, cs);
        else
            launch_packed_copy(static_cast<const uint64_t*>(src), (n + 63) / 64, n, n, P0, ldw, 0, cs);
        SCK(launch_wcsr_build(P0, n, ldw, wptr, widx, wval, cs), "word index build");
        auto* cost = reinterpret_cast<unsigned long long*>(w + SW_COST);
        SCK(launch_square_cost(wptr, widx, wval, n, cost, sms, cs), "squaring cost");
        cudaGraph_t g = nullptr;
        cudaStreamCaptureStatus cst;
        SCK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr), "capture info");
        cudaGraphConditionalHandle hA, hC;
        SCK(cudaGraphConditionalHandleCreate(&hA, g, 0, cudaGraphCondAssignDefault), "conditional handle");
        SCK(cudaGraphConditionalHandleCreate(&hC, g, 0, cudaGraphCondAssignDefault), "conditional handle");
        solo_rows_decide_kernel<<<1, 1, 0, cs>>>(w, cap, 1, step_s, s_word, s_row, limit, hA);
        cudaGraph_t body = nullptr;
        SST(add_while(ctx, cs, hA, &body));
        SCK(cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
            "begin capture of the bit-row loop");
        {
            cudaError_t e = launch_square_rows(wptr, widx, wval, P0, n, ldw, P1, sms, cb, w + SW_CHANGED);
            if (e == cudaSuccess) {  // the next step reads P0 (ldw is even: rows are whole 16-byte units)
                solo_copy_kernel<<<sms * 4, 256, 0, cb>>>(reinterpret_cast<uint4*>(P0),
                                                           reinterpret_cast<const uint4*>(P1), n * ldw / 2);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = launch_wcsr_build(P0, n, ldw, wptr, widx, wval, cb);
            if (e == cudaSuccess) e = launch_square_cost(wptr, widx, wval, n, cost, sms, cb);
            if (e == cudaSuccess) {
                solo_rows_decide_kernel<<<1, 1, 0, cb>>>(w, cap, 0, step_s, s_word, s_row, limit, hA);
                e = cudaGetLastError();
            }
            cudaGraph_t tmp = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cb, &tmp);
            if (e != cudaSuccess || e2 != cudaSuccess) return fail(cuda_err(ctx, e != cudaSuccess ? e : e2, "bit-row loop"));
        }
        // ---- squarings on packed E2M1 operands (R^T as the B operand), two per loop iteration
        launch_packed_to_e2m1(P0, ldw, n, Q[0], QT[0], n_pad, cs);
        solo_mid_kernel<<<1, 1, 0, cs>>>(w, hC);
        CUtensorMap mA[2], mB0[2], mB1[2];
        for (int b = 0; b < 2; ++b) {
            SST(make_tmap(ctx, &mA[b], Q[b], n_pad, ld4, ld4, TC_BM));
            SST(make_tmap(ctx, &mB0[b], QT[b], n_pad, ld4, ld4, TC_BN / 2));
            SST(make_tmap(ctx, &mB1[b], QT[b], n_pad, ld4, ld4, tc4_b1_rows()));
        }
        SST(add_while(ctx, cs, hC, &body));
        // after each product, when R is close to its closure, the next squaring may run only on the rows and columns
        // that still hold zeros: IF nodes inside the loop's body, one for its statistics and one for the squaring
        const int64_t ldw_t = n_pad / 64;
        const bool thin_p = thin_any && thin_fixed_seconds(n_pad) < limit;
        cudaGraphConditionalHandle hT[2], hT2[2];
        if (thin_p) {
            for (int h = 0; h < 2; ++h) {
                SCK(cudaGraphConditionalHandleCreate(&hT[h], body, 0, cudaGraphCondAssignDefault), "conditional handle");
                SCK(cudaGraphConditionalHandleCreate(&hT2[h], body, 0, cudaGraphCondAssignDefault), "conditional handle");
            }
        }
        auto* t_smp = reinterpret_cast<unsigned long long*>(w + SW_SMP);
        auto* t_stat = reinterpret_cast<unsigned long long*>(w + SW_TSTAT);
        // captures one IF body on stream cc: fn() issues its launches
        auto capture_if = [&](cudaGraphConditionalHandle hh, auto fn) -> cudaError_t {
            cudaGraph_t ifb = nullptr;
            if (add_conditional(ctx, cb, hh, cudaGraphCondTypeIf, &ifb) != BMLP_OK) return cudaErrorUnknown;
            cudaError_t e1 = cudaStreamBeginCaptureToGraph(cc, ifb, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
            if (e1 != cudaSuccess) return e1;
            e1 = fn();
            cudaGraph_t tmp = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cc, &tmp);
            return e1 != cudaSuccess ? e1 : e2;
        };
        SCK(cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
            "begin capture of the tensor-core loop");
        {
            cudaError_t e = cudaSuccess;
            for (int half = 0; half < 2 && e == cudaSuccess; ++half) {
                TcParams p4{};
                p4.m_tiles = static_cast<int32_t>(n_pad / TC_BM);
                p4.n_tiles = static_cast<int32_t>((n_pad + tc4_tile_n() - 1) / tc4_tile_n());
                p4.k_blocks = static_cast<int32_t>(n_pad / 256);
                p4.mode = TC_MODE_RMS;
                p4.ld = ld4;
                p4.old_r = Q[half];
                p4.out_r = Q[half ^ 1];
                p4.out_rt = QT[half ^ 1];
                p4.changed = w + SW_CHANGED;
                p4.error = ctx->d_ctl + CTL_ERROR;
                p4.wait_cycles = wait_cycles;
                p4.guard = w + (half == 0 ? SW_GC : SW_G1);
                if (thin_p) {  // the epilogue keeps R and R^T as bit rows for the restricted squaring
                    p4.out_bits = reinterpret_cast<uint32_t*>(TP);
                    p4.out_bits_t = reinterpret_cast<uint32_t*>(TPT);
                    p4.ldb = 2 * ldw_t;
                }
                e = launch_tc4_product_duo(mA[half], mB0[half], mB1[half], p4, sms, cb);
                if (e == cudaSuccess) {
                    solo_tc_decide_kernel<<<1, 1, 0, cb>>>(w, cap, half, hC);
                    e = cudaGetLastError();
                }
                if (thin_p && e == cudaSuccess) {
                    uint8_t* Qn = Q[half ^ 1];
                    uint8_t* QTn = QT[half ^ 1];
                    e = launch_thin_sample(Qn, ld4, n, thin_sample_rows(), t_smp, cb);
                    if (e == cudaSuccess) {
                        solo_thin_gate_kernel<<<1, 1, 0, cb>>>(w, half, n, thin_row_spread(), hT[half]);
                        e = cudaGetLastError();
                    }
                    if (e == cudaSuccess)
                        e = capture_if(hT[half], [&]() -> cudaError_t {
                            cudaError_t e3 = launch_thin_stats(Qn, QTn, ld4, n, TP, TPT, ldw_t, t_rowcnt, t_colcnt,
                                                               t_bmask, t_blist, t_rlist, t_stat, true, sms, cc);
                            if (e3 != cudaSuccess) return e3;
                            solo_thin_decide_kernel<<<1, 1, 0, cc>>>(w, ldw_t, thin_fixed_seconds(n_pad), s_word, s_row,
                                                                     limit);
                            return cudaGetLastError();
                        });
                    if (e == cudaSuccess) {
                        solo_thin_arm_kernel<<<1, 1, 0, cb>>>(w, hT2[half]);
                        e = cudaGetLastError();
                    }
                    if (e == cudaSuccess)
                        e = capture_if(hT2[half], [&]() -> cudaError_t {
                            cudaError_t e3 = launch_thin_squaring_dev(TP, TPT, ldw_t, n, t_blist, t_rlist, t_stat, TT,
                                                                      Qn, QTn, ld4, w + SW_TCHANGED, sms, cc);
                            if (e3 != cudaSuccess) return e3;
                            solo_thin_post_kernel<<<1, 1, 0, cc>>>(w, half, cap);
                            return cudaGetLastError();
                        });
                    if (e == cudaSuccess) {
                        solo_loop_ctl_kernel<<<1, 1, 0, cb>>>(w, hC);
                        e = cudaGetLastError();
                    }
                }
            }
            cudaGraph_t tmp = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cb, &tmp);
            if (e != cudaSuccess || e2 != cudaSuccess)
                return fail(cuda_err(ctx, e != cudaSuccess ? e : e2, "tensor-core loop"));
        }
        if (thin_p) {  // a restricted squaring that ended the loop after the first product left the closure in Q1
            solo_result_copy_kernel<<<sms * 4, 256, 0, cs>>>(w, reinterpret_cast<uint4*>(Q[0]),
                                                             reinterpret_cast<const uint4*>(Q[1]), n_pad * ld4 / 16);
            SCK(cudaGetLastError(), "result copy");
        }
        // ---- results: Q[0] holds the closure (a product that changed nothing left both buffers equal)
        if (p.kind == BMLP_PROBLEM_CLOSURE) {
            if (p.fmt == BMLP_FMT_U8)
                launch_e2m1_to_u8(Q[0], ld4, n, static_cast<uint8_t*>(p.out), p.reflexive, cs);
            else
                launch_e2m1_to_packed(Q[0], ld4, n, static_cast<uint64_t*>(p.out), (n + 63) / 64, p.reflexive, cs);
        } else {
            // out = (I + R2+) R1 on 4-bit operands, on the squaring kernel: A = I + R2+ (Q[0], diagonal set),
            // B^T = R1^T (encoded with R1 into the free pair Q[1], QT[1]), and a zero "old R" (QT[0]), so that the
            // kernel's R' is C > 0; R' goes to Q[1] (R1 is no longer needed), R'^T to the scratch
            launch_set_diag_e2m1(Q[0], ld4, n, cs);
            if (p.fmt == BMLP_FMT_U8)
                launch_u8_to_e2m1(static_cast<const uint8_t*>(p.R1), n, Q[1], QT[1], n_pad, cs);
            else
                launch_packed_to_e2m1(static_cast<const uint64_t*>(p.R1), (n + 63) / 64, n, Q[1], QT[1], n_pad, cs);
            SCK(cudaMemsetAsync(QT[0], 0, static_cast<size_t>(n_pad) * static_cast<size_t>(ld4), cs), "clear old R");
            CUtensorMap fa, fb0, fb1;
            SST(make_tmap(ctx, &fa, Q[0], n_pad, ld4, ld4, TC_BM));
            SST(make_tmap(ctx, &fb0, QT[1], n_pad, ld4, ld4, TC_BN / 2));
            SST(make_tmap(ctx, &fb1, QT[1], n_pad, ld4, ld4, tc4_b1_rows()));
            TcParams pp{};
            pp.m_tiles = static_cast<int32_t>(n_pad / TC_BM);
            pp.n_tiles = static_cast<int32_t>((n_pad + tc4_tile_n() - 1) / tc4_tile_n());
            pp.k_blocks = static_cast<int32_t>(n_pad / 256);
            pp.mode = TC_MODE_RMS;
            pp.ld = ld4;
            pp.old_r = QT[0];
            pp.out_r = Q[1];
            pp.out_rt = M0;
            pp.changed = w + SW_CHANGED;
            pp.error = ctx->d_ctl + CTL_ERROR;
            pp.wait_cycles = wait_cycles;
            SCK(launch_tc4_product_duo(fa, fb0, fb1, pp, sms, cs), "final product");
            if (p.fmt == BMLP_FMT_U8)
                launch_e2m1_to_u8(Q[1], ld4, n, static_cast<uint8_t*>(p.out), 0, cs);
            else
                launch_e2m1_to_packed(Q[1], ld4, n, static_cast<uint64_t*>(p.out), (n + 63) / 64, 0, cs);
        }
        SCK(cudaGetLastError(), "large-problem launches");
    }
#undef SCK
#undef SST
    cudaGraph_t g = nullptr;
    BCK(cudaStreamEndCapture(cs, &g), "end capture of the large problems");
    return status;
}

uint64_t batch_key(const bmlp_problem* probs, int64_t count, int variant, const int* tune, int64_t solo_n) {
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &count, sizeof(count));
    h = fnv(h, &variant, sizeof(variant));
    h = fnv(h, &solo_n, sizeof(solo_n));
    h = fnv(h, tune, sizeof(int) * 32);
    for (int64_t i = 0; i < count; ++i) h = fnv(h, &probs[i], sizeof(bmlp_problem));
    return h;
}

}  // namespace

bmlp_status batch_run_impl(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, int variant,
                           long long wait_cycles, int32_t* iters_out, cudaStream_t s, int64_t solo_n) {
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
    const uint64_t key = batch_key(probs, count, variant, ctx->tune, solo_n);
    BatchCache* c = static_cast<BatchCache*>(ctx->batch);
    if (c == nullptr || c->key != key) BST(build_batch(ctx, probs, count, variant, wait_cycles, key, solo_n, &c));
    BCK(cudaMemsetAsync(ctx->d_ctl, 0, CTL_WORDS * sizeof(int), s), "reset flags");
    ctx->stats.n_pad = static_cast<int64_t>(c->ws_bytes);
    BCK(cudaGraphLaunch(c->exec, s), "cudaGraphLaunch");
    const int np = c->nprob;
    BCK(cudaMemcpyAsync(c->h_iters.data(), c->d_ints + 2 * np, sizeof(int) * np, cudaMemcpyDeviceToHost, s),
        "read iterations");
    BCK(cudaMemcpyAsync(c->h_notconv.data(), c->d_ints + 4 * np, sizeof(int) * np, cudaMemcpyDeviceToHost, s),
        "read convergence");
    const int ns = static_cast<int>(c->solo.size());
    if (ns > 0)
        BCK(cudaMemcpyAsync(c->h_solo.data(), c->d_solo, sizeof(int) * SW_WORDS * ns, cudaMemcpyDeviceToHost, s),
            "read large-problem state");
    BCK(cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, CTL_WORDS * sizeof(int), cudaMemcpyDeviceToHost, s), "read flags");
    BCK(host_sync(ctx, s), "synchronise batch");
    if (ctx->h_ctl[CTL_ERROR] != 0)
        return set_err(ctx, BMLP_ERR_TIMEOUT, "in-kernel wait timed out (code 0x%x)", ctx->h_ctl[CTL_ERROR]);
    int maxit = 0, bad = 0;
    for (int sl = 0; sl < np; ++sl) {
        const int i = c->order[sl];
        if (iters_out) iters_out[i] = c->h_iters[sl];
        maxit = std::max(maxit, c->h_iters[sl]);
        bad |= c->h_notconv[sl];
    }
    for (int k = 0; k < ns; ++k) {
        const int* w = c->h_solo.data() + SW_WORDS * k;
        if (iters_out) iters_out[c->solo[k]] = w[SW_ITERS];
        maxit = std::max(maxit, w[SW_ITERS]);
        bad |= w[SW_NOTCONV];
        ctx->stats.launches += 6 + 6 * w[SW_ITERS];
        ctx->stats.product_launches += w[SW_ITERS];
    }
    ctx->stats.iterations = maxit;
    ctx->stats.launches += 4 + 3 * maxit;
    ctx->stats.product_launches += maxit + 1;
    if (bad) return set_err(ctx, BMLP_ERR_NOT_CONVERGED, "a problem did not converge within its cap");
    return BMLP_OK;
}

}  // namespace bmlp
