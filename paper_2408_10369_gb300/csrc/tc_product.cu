// Boolean matrix product on the 5th-generation tensor cores (tcgen05), with
// the fixpoint arithmetic of the paper fused into the epilogue.
//
// The Boolean product (A B)_ij = OR_k A_ik AND B_kj (Sec. 2) is computed as
// the integer count C_ij = sum_k A_ik B_kj on 0/1 E4M3 operands with FP32
// accumulation, then thresholded: (A B)_ij = [C_ij > 0]. Every count is an
// integer <= n < 2^24, so FP32 holds it exactly and the threshold is exact:
// no rounding can change a bit.
//
// Kernel structure (one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer: 128 x 128 A tile and 256 x 128 B^T tile per
//               stage, 4-stage smem ring, 128-byte swizzle;
//   warp 1      MMA issuer: 4 x tcgen05.mma (M=128, N=256, K=32) per stage
//               into one of two TMEM accumulators (2 x 256 FP32 columns);
//   warps 2..5  epilogue: tcgen05.ld of the accumulator, threshold, and the
//               mode-specific update (below), while the MMA warp already
//               fills the other accumulator.
// Epilogue modes:
//   RMS   (Algorithm 1 / Eq. 4, squaring form R <- R + R R):
//         R'_ij = R_ij | [C_ij > 0]; writes R' and R'^T (the next
//         iteration's A and B operands) and raises `changed` if R' != R.
//   SMP   (Algorithm 2 / Eq. 5, frontier form): N = [C > 0] & ~V; V |= N;
//         writes N as the next frontier, marks its nonzero 128 x 128 blocks
//         so that the next level skips all-zero K blocks of the frontier.
//   PLAIN out = [C > 0] (the final product of a composition).
// Tile sources: one problem (tc_product_kernel, tensor maps as kernel
// parameters) or a device work list over many problems (tc_group_kernel,
// tensor maps in global memory; used by the grouped batch runner).
// Every wait on an mbarrier is bounded; on expiry the CTA records an error
// code, stops issuing work, waits (bounded) for its own copies and MMAs in
// flight, frees its TMEM and exits.
#include <cstdio>
#include <cudaTypedefs.h>

#include "internal.h"
#include "ptx.cuh"

namespace bmlp {
namespace {

constexpr int A_BYTES = TC_BM * TC_BK;       // 16 KiB
constexpr int B_BYTES = TC_BN * TC_BK;       // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int UMMA_K = 32;                   // E4M3 elements (bytes) of K per MMA
constexpr int ACC_COLS = TC_BN;              // FP32 TMEM columns per accumulator
constexpr int TMEM_COLS = 2 * ACC_COLS;      // double-buffered accumulator
constexpr int GROUP_M = 8;                   // raster: 8 row blocks share B tiles in L2

constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + TC_STAGES * A_BYTES;
constexpr int OFF_BAR = OFF_B + TC_STAGES * B_BYTES;
constexpr int NUM_BARS = 2 * TC_STAGES + 5;  // full[], empty[], tfull[2], tempty[2], done
constexpr int OFF_MISC = OFF_BAR + NUM_BARS * 8;
constexpr int SMEM_END = OFF_MISC + 16;
constexpr int SMEM_BYTES = SMEM_END + 1024;  // + slack to align the base to 1024

constexpr int ERR_WAIT_PRODUCER = 0x101;
constexpr int ERR_WAIT_MMA = 0x102;
constexpr int ERR_WAIT_EPILOGUE = 0x103;

__device__ __forceinline__ void tile_coords(int t, int m_tiles, int n_tiles, int& mb, int& nb) {
    const int per_group = GROUP_M * n_tiles;
    const int g = t / per_group;
    const int first_m = g * GROUP_M;
    const int gsz = min(m_tiles - first_m, GROUP_M);
    const int r = t % per_group;
    mb = first_m + r % gsz;
    nb = r / gsz;
}

// 32 bytes -> 32-bit mask of nonzero bytes
__device__ __forceinline__ uint32_t nz_mask32(const uint4& a, const uint4& b) {
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int x = 0; x < 4; ++x) m |= (((w[k] >> (8 * x)) & 0xFFu) != 0 ? 1u : 0u) << (4 * k + x);
    }
    return m;
}

// 16-bit mask -> 16 bytes of {0, E4M3 one}
__device__ __forceinline__ uint4 mask_to_bytes16(uint32_t m) {
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

// Waits for this CTA's own copies / MMAs in flight before it frees its shared
// memory and TMEM get at least ~1 s (at 2 GHz) even when the caller chose a
// very short timeout: they finish in microseconds once issued.
__device__ __forceinline__ long long drain_cycles(long long limit) {
    return limit > 2000000000LL ? limit : 2000000000LL;
}

__device__ __forceinline__ bool wait_lane0(uint64_t* bar, uint32_t parity, volatile int* abort, long long limit,
                                           int lane) {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(bar, parity, abort, limit) ? 1 : 0;
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// Everything one output tile needs.
struct Tile {
    const CUtensorMap* mapA;
    const CUtensorMap* mapB;
    int mb, nb, k_blocks, mode;
    int64_t ld;
    const uint8_t* old_r;
    uint8_t* out_r;
    uint8_t* out_rt;
    uint8_t* visited;
    const uint8_t* kflags;
    uint8_t* kflags_next;
    int* changed;
    bool masked;             // RMS with block maps: kmask lists the K blocks to run
    uint64_t kmask[4];
    uint8_t* fmap_next;      // block maps of the new R (RMS) or null
    uint8_t* fmapT_next;
    int fm_ld;
};

// 16 map bytes -> 16-bit mask of nonzero bytes
__device__ __forceinline__ uint32_t nz16(const uint4& v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int b = 0; b < 4; ++b) m |= (((w[k] >> (8 * b)) & 0xFFu) != 0 ? 1u : 0u) << (4 * k + b);
    return m;
}

// K blocks kb that contribute to output tile (A row blocks a0, a1; 256 output
// columns = column blocks 2 nb, 2 nb + 1): the A block (a0 or a1, kb) and the
// B^T block, i.e. R block (kb, 2 nb or 2 nb + 1), are both nonzero. Built from
// four contiguous map rows with 16-byte loads; a CTA pair passes both of its
// row blocks, so both CTAs run the same K sequence.
__device__ __forceinline__ void build_kmask(const TcParams* p, int a0, int a1, int nb, uint64_t (&km)[4]) {
    const uint4* ra0 = reinterpret_cast<const uint4*>(p->fmap + static_cast<int64_t>(a0) * p->fm_ld);
    const uint4* ra1 = reinterpret_cast<const uint4*>(p->fmap + static_cast<int64_t>(a1) * p->fm_ld);
    const uint4* rb0 = reinterpret_cast<const uint4*>(p->fmapT + static_cast<int64_t>(2 * nb) * p->fm_ld);
    const uint4* rb1 = reinterpret_cast<const uint4*>(p->fmapT + static_cast<int64_t>(2 * nb + 1) * p->fm_ld);
#pragma unroll
    for (int w = 0; w < 4; ++w) km[w] = 0;
    const int chunks = p->fm_ld / 16;
#pragma unroll
    for (int c = 0; c < 16; ++c) {  // fully unrolled: km stays in registers
        if (c < chunks) {
            const uint32_t a = nz16(ra0[c]) | nz16(ra1[c]);
            const uint32_t b = nz16(rb0[c]) | nz16(rb1[c]);
            km[c >> 2] |= static_cast<uint64_t>(a & b) << (16 * (c & 3));
        }
    }
}

// Does K block kb contribute to this tile? SMP: the frontier block is nonzero;
// RMS with block maps: the tile's mask; otherwise every K block.
__device__ __forceinline__ bool kactive(const Tile& x, int kb) {
    if (x.kflags != nullptr) return x.kflags[x.mb * x.k_blocks + kb] != 0;
    if (x.masked) {
        const uint64_t w = kb < 64 ? x.kmask[0] : kb < 128 ? x.kmask[1] : kb < 192 ? x.kmask[2] : x.kmask[3];
        return (w >> (kb & 63)) & 1ull;
    }
    return true;
}

// One problem: the tensor maps are kernel parameters.
struct SingleSource {
    const CUtensorMap* a;
    const CUtensorMap* b;
    const TcParams* p;
    __device__ int count() const { return p->m_tiles * p->n_tiles; }
    __device__ void get(int t, Tile& x) const {
        tile_coords(t, p->m_tiles, p->n_tiles, x.mb, x.nb);
        x.mapA = a;
        x.mapB = b;
        x.k_blocks = p->k_blocks;
        x.mode = p->mode;
        x.ld = p->ld;
        x.old_r = p->old_r;
        x.out_r = p->out_r;
        x.out_rt = p->out_rt;
        x.visited = p->visited;
        x.kflags = p->kflags;
        x.kflags_next = p->kflags_next;
        x.changed = p->changed;
        x.masked = p->fmap != nullptr;
        if (x.masked) build_kmask(p, x.mb, x.mb, x.nb, x.kmask);
        x.fmap_next = p->fmap_next;
        x.fmapT_next = p->fmapT_next;
        x.fm_ld = p->fm_ld;
    }
};

// Many problems: items are numbered problem by problem; offs[p] is the first
// item of problem p (exclusive prefix of its active tile count).
struct GroupSource {
    const GroupProblem* probs;
    const GroupState* st;
    int nprob;
    int total;
    int phase;
    __device__ int count() const { return total; }
    __device__ void get(int t, Tile& x) const {
        const int* offs = st->tc_offs;
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {  // largest p with offs[p] <= t (that problem is nonempty)
            const int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const GroupProblem& g = probs[lo];
        const int par = st->parity[lo];
        tile_coords(t - offs[lo], g.m_tiles, g.n_tiles, x.mb, x.nb);
        x.k_blocks = g.k_blocks;
        x.ld = g.ld;
        x.mapA = &g.mapA[par];
        x.visited = nullptr;
        x.kflags = nullptr;
        x.kflags_next = nullptr;
        x.masked = false;
        x.fmap_next = nullptr;
        x.fmapT_next = nullptr;
        x.fm_ld = 0;
        if (phase == 0) {
            x.mode = TC_MODE_RMS;
            x.mapB = &g.mapB[par];
            x.old_r = g.M[par];
            x.out_r = g.M[par ^ 1];
            x.out_rt = g.T[par ^ 1];
            x.changed = &st->changed[lo];
        } else {
            x.mode = TC_MODE_PLAIN;
            x.mapB = &g.mapBF;
            x.old_r = nullptr;
            x.out_r = g.X;
            x.out_rt = nullptr;
            x.changed = &st->changed[lo];
        }
    }
};

template <class Src>
__device__ __forceinline__ void tc_body(const Src& src, int* error, long long limit,
                                        unsigned long long* issued = nullptr) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem + OFF_A;
    uint8_t* sB = smem + OFF_B;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
    uint64_t* full = bars;
    uint64_t* empty = bars + TC_STAGES;
    uint64_t* tfull = bars + 2 * TC_STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + OFF_MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_tiles = src.count();
    const int first = static_cast<int>(blockIdx.x);
    const int step = static_cast<int>(gridDim.x);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 128);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_par[TC_STAGES];
#pragma unroll
            for (int s = 0; s < TC_STAGES; ++s) last_par[s] = -1;
            bool ok = true;
            for (int t = first; t < num_tiles && ok; t += step) {
                Tile x;
                src.get(t, x);
                for (int kb = 0; kb < x.k_blocks; ++kb) {
                    if (!kactive(x, kb)) continue;
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, limit)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], STAGE_BYTES);
                    tma_load_2d(sA + stage * A_BYTES, x.mapA, kb * TC_BK, x.mb * TC_BM, &full[stage]);
                    tma_load_2d(sB + stage * B_BYTES, x.mapB, kb * TC_BK, x.nb * TC_BN, &full[stage]);
                    last_par[stage] = static_cast<int>(phase);
                    if (++stage == TC_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                atomicCAS(error, 0, ERR_WAIT_PRODUCER);
                // let every copy this CTA issued land before the CTA exits
                volatile int never = 0;
                for (int s = 0; s < TC_STAGES; ++s)
                    if (last_par[s] >= 0)
                        mbar_wait_bounded(&full[s], static_cast<uint32_t>(last_par[s]), &never, drain_cycles(limit));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        const uint32_t idesc = idesc_e4m3_f32(TC_BM, TC_BN);
        int stage = 0;
        uint32_t phase = 0;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int t = first; t < num_tiles && ok; t += step) {
            Tile x;
            src.get(t, x);
            if (!wait_lane0(&tempty[acc], acc_phase ^ 1u, abort_flag, limit, lane)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * ACC_COLS);
            uint32_t accumulate = 0;
            unsigned long long nk = 0;
            for (int kb = 0; kb < x.k_blocks; ++kb) {
                if (!kactive(x, kb)) continue;
                ++nk;
                if (!wait_lane0(&full[stage], phase, abort_flag, limit, lane)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t a0 = smem_u32(sA + stage * A_BYTES);
                    const uint32_t b0 = smem_u32(sB + stage * B_BYTES);
#pragma unroll
                    for (int k = 0; k < TC_BK / UMMA_K; ++k) {
                        tc_mma_f8(d_tmem, smem_desc_kmajor_sw128(a0 + k * UMMA_K),
                                  smem_desc_kmajor_sw128(b0 + k * UMMA_K), idesc, accumulate);
                        accumulate = 1;
                    }
                    tc_commit(&empty[stage]);
                }
                __syncwarp();
                accumulate = 1;
                if (++stage == TC_STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
            // 128 x 256 x 128 multiply-adds per K block run = 8 units of 128 x 32 x 128
            if (lane == 0 && issued != nullptr) atomicAdd(issued, 8ull * nk);
            if (lane == 0) tc_commit(&tfull[acc]);
            __syncwarp();
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
        if (!ok && lane == 0) atomicCAS(error, 0, ERR_WAIT_MMA);
        // every MMA this thread issued must finish before TMEM is freed
        if (lane == 0) {
            tc_commit(done);
            volatile int never = 0;
            mbar_wait_bounded(done, 0, &never, drain_cycles(limit));
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue
        const int quarter = warp & 3;             // TMEM lanes this warp may access
        const int row_in_tile = quarter * 32 + lane;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = first; t < num_tiles; t += step) {
            Tile x;
            src.get(t, x);
            if (!wait_lane0(&tfull[acc], acc_phase, abort_flag, limit, lane)) {
                if (lane == 0) atomicCAS(error, 0, ERR_WAIT_EPILOGUE);
                break;
            }
            tc_fence_after();
            // no MMA ran for a tile whose K blocks were all skipped: its product is zero
            bool active = true;
            if (x.masked) {
                active = (x.kmask[0] | x.kmask[1] | x.kmask[2] | x.kmask[3]) != 0ull;
            } else if (x.kflags != nullptr) {
                active = false;
                for (int kb = 0; kb < x.k_blocks && !active; ++kb) active = kactive(x, kb);
            }
            const int64_t row = static_cast<int64_t>(x.mb) * TC_BM + row_in_tile;
            uint32_t any = 0;
#pragma unroll 1
            for (int c0 = 0; c0 < TC_BN; c0 += 32) {
                uint32_t v[32];
                if (active) {
                    tmem_ld_32x32b_x32(tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                           static_cast<uint32_t>(acc * ACC_COLS + c0), v);
                    tmem_ld_wait();
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0;
                }
                uint32_t cbits = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) cbits |= (v[j] != 0u ? 1u : 0u) << j;
                const int64_t col0 = static_cast<int64_t>(x.nb) * TC_BN + c0;
                const int64_t off = row * x.ld + col0;
                if (x.mode == TC_MODE_RMS) {
                    const uint4* o = reinterpret_cast<const uint4*>(x.old_r + off);
                    const uint32_t obits = nz_mask32(o[0], o[1]);
                    const uint32_t nbits = obits | cbits;
                    any |= nbits ^ obits;
                    uint4* w = reinterpret_cast<uint4*>(x.out_r + off);
                    w[0] = mask_to_bytes16(nbits & 0xFFFFu);
                    w[1] = mask_to_bytes16(nbits >> 16);
                    uint8_t* tcol = x.out_rt + col0 * x.ld + row;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        tcol[j * x.ld] = ((nbits >> j) & 1u) ? static_cast<uint8_t>(BMLP_E4M3_ONE) : 0;
                    if (x.fmap_next != nullptr && nbits != 0u) {
                        const int64_t cb = col0 / TC_BK;
                        x.fmap_next[static_cast<int64_t>(x.mb) * x.fm_ld + cb] = 1;
                        x.fmapT_next[cb * x.fm_ld + x.mb] = 1;
                    }
                } else if (x.mode == TC_MODE_SMP) {
                    uint4* vp = reinterpret_cast<uint4*>(x.visited + off);
                    const uint32_t vbits = nz_mask32(vp[0], vp[1]);
                    const uint32_t nbits = cbits & ~vbits;
                    any |= nbits;
                    if (nbits) {
                        const uint32_t nv = vbits | nbits;
                        vp[0] = mask_to_bytes16(nv & 0xFFFFu);
                        vp[1] = mask_to_bytes16(nv >> 16);
                        x.kflags_next[x.mb * x.k_blocks + static_cast<int>(col0 / TC_BK)] = 1;
                    }
                    uint4* w = reinterpret_cast<uint4*>(x.out_r + off);
                    w[0] = mask_to_bytes16(nbits & 0xFFFFu);
                    w[1] = mask_to_bytes16(nbits >> 16);
                } else {
                    uint4* w = reinterpret_cast<uint4*>(x.out_r + off);
                    w[0] = mask_to_bytes16(cbits & 0xFFFFu);
                    w[1] = mask_to_bytes16(cbits >> 16);
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty[acc]);
            if (__any_sync(0xFFFFFFFFu, any != 0) && lane == 0) atomicOr(x.changed, 1);
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_product_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcParams p) {
    if (threadIdx.x == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    SingleSource src{&tmA, &tmB, &p};
    tc_body(src, p.error, p.wait_cycles, p.issued);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_group_kernel(const GroupProblem* probs, const GroupState* st, int nprob, int phase, int* error,
                long long wait_cycles) {
    GroupSource src{probs, st, nprob, *st->tc_total, phase};
    tc_body(src, error, wait_cycles);
}

}  // namespace

int tc_smem_bytes() { return SMEM_BYTES; }

bmlp_status make_tmap(bmlp_ctx* ctx, CUtensorMap* map, const void* base, int64_t rows, int64_t cols_bytes, int64_t ld,
                      int box_rows) {
    if (ctx->encode_fn == nullptr) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr)
            return set_err(ctx, BMLP_ERR_CUDA, "cuTensorMapEncodeTiled not available from the driver");
        ctx->encode_fn = fn;
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ctx->encode_fn);
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols_bytes), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(TC_BK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, BMLP_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return BMLP_OK;
}

cudaError_t launch_tc_product(const CUtensorMap& a, const CUtensorMap& b, const TcParams& p, int grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(tc_product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_product_kernel<<<grid, TC_THREADS, SMEM_BYTES, s>>>(a, b, p);
    return cudaGetLastError();
}

void* tc_group_kernel_ptr() { return reinterpret_cast<void*>(&tc_group_kernel); }

cudaError_t prepare_tc_group() {
    return cudaFuncSetAttribute(tc_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

}  // namespace bmlp
