// Squaring step of BMLP-RMS (Algorithm 1 / Eq. 4, form R <- R + R R) on
// 4-bit tensor-core operands.
//
// The Boolean product is the integer count C_ij = sum_k R_ik R_kj
// thresholded at zero (Sec. 2). Here the 0/1 operands are E2M1 values
// (0 = 0b0000, 1.0 = 0b0010) packed two per byte, element k of a row in byte
// k / 2 (low nibble for even k), and the MMA is tcgen05 kind::mxf4 with every
// UE8M0 block scale equal to 2^0, so each product term is exactly 1.0 x 1.0
// and the FP32 accumulator holds the exact count (<= n < 2^24). Compared with
// the E4M3 kernel, a 128-byte K block carries 256 elements instead of 128:
// half the operand bytes per Boolean operation.
//
// Structure (2-CTA clusters, one CTA per SM, persistent over pair tiles of
// 256 rows x 480 columns):
//   warp 0      TMA producer (both CTAs): the CTA's own 128 rows of A and its
//               240 of the tile's 480 B^T rows (128 of the first 256, 112 of
//               the last 224), 128 bytes of K per stage, 4 stages of 46 KB,
//               128-byte swizzle; both CTAs' copies complete on the even
//               CTA's barrier (no multicast loads);
//   warp 1      MMA issuer (even CTA): per 64-deep K step one
//               tcgen05.mma.cta_group::2 kind::mxf4 of M=256, N=256 into TMEM
//               columns 0..255 and one of M=256, N=224 into columns 256..479
//               (in each CTA); the unit scale factors fill columns 480..511;
//   warps 2..5  epilogue (both CTAs): drains the accumulator into registers as
//               bits and frees it at once, then computes R' = R | [C > 0],
//               writes R' and R'^T (transposed through warp ballots) and
//               raises `changed` if R' != R.
// Every mbarrier wait is bounded; on expiry the CTA records an error code,
// waits (bounded) for its own copies and MMAs in flight, frees TMEM and exits.
#include <cudaTypedefs.h>

#include "internal.h"
#include "ptx.cuh"

namespace bmlp {
namespace {

constexpr int F4_BK = 128;                     // bytes of K per stage (256 elements)
constexpr int F4_UMMA_K_BYTES = 32;            // 64 E2M1 elements per MMA
constexpr int F4_TMEM_COLS = 512;
constexpr uint32_t F4_UE8M0_ONE4 = 0x7F7F7F7Fu;  // four UE8M0 scales of 2^0

constexpr int F4_GROUP_M = 8;  // raster: 8 row-block pairs share B tiles in L2

__device__ __forceinline__ long long f4_drain_cycles(long long limit) {
    return limit > 2000000000LL ? limit : 2000000000LL;
}

__device__ __forceinline__ bool f4_wait_lane0(uint64_t* bar, uint32_t parity, volatile int* abort, long long limit,
                                              int lane) {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(bar, parity, abort, limit) ? 1 : 0;
    return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// Pair t -> (row-block pair mp, column block nb), grouped so that F4_GROUP_M
// pairs in a row share each B tile while it is in L2.
__device__ __forceinline__ void f4_pair_coords(int t, int m_pairs, int n_tiles, int& mp, int& nb) {
    const int per_group = F4_GROUP_M * n_tiles;
    const int g = t / per_group;
    const int first = g * F4_GROUP_M;
    const int gsz = min(m_pairs - first, F4_GROUP_M);
    const int r = t % per_group;
    mp = first + r % gsz;
    nb = r / gsz;
}

// 8 bits -> 8 nibbles of {0, E2M1 one}: bit k becomes nibble k.
__device__ __forceinline__ uint32_t f4_spread8(uint32_t b) {
    uint32_t t = b & 0xFFu;
    t = (t | (t << 12)) & 0x000F000Fu;
    t = (t | (t << 6)) & 0x03030303u;
    t = (t | (t << 3)) & 0x11111111u;
    return t << 1;
}

// 8 nibbles -> 8 bits: bit k = (nibble k != 0).
__device__ __forceinline__ uint32_t f4_gather8(uint32_t w) {
    uint32_t x = w | (w >> 1);
    x |= x >> 2;
    x &= 0x11111111u;
    x = (x | (x >> 3)) & 0x03030303u;
    x = (x | (x >> 6)) & 0x000F000Fu;
    x = (x | (x >> 12)) & 0xFFu;
    return x;
}

__device__ __forceinline__ uint4 f4_nibbles32(uint32_t bits) {
    return make_uint4(f4_spread8(bits), f4_spread8(bits >> 8), f4_spread8(bits >> 16), f4_spread8(bits >> 24));
}

__device__ __forceinline__ uint32_t f4_bits32(const uint4& v) {
    return f4_gather8(v.x) | (f4_gather8(v.y) << 8) | (f4_gather8(v.z) << 16) | (f4_gather8(v.w) << 24);
}

// ---- The squaring kernel: one M = 256 MMA per CTA pair (tcgen05
// .cta_group::2) per 64-deep K step, on a pair tile of 256 rows x BN columns.
// Each CTA keeps only its own 128 rows of A and its half of the B rows the
// pair needs, and the even CTA issues every MMA; the accumulator rows land in
// each CTA's own TMEM (CTA r holds output rows 128 r .. 128 r + 127 of the
// pair's tile). A wider tile reads fewer operand bytes per Boolean operation
// from L2: per 256-deep K block a CTA stages 16 KB of A and 128 (N1 = 0) or
// 240 (N1 = 224) rows of B for 256 x BN x 256 multiply-adds.
//
// N1 = 0:   BN = 256, one N = 256 MMA per K step, 6 stages of 32 KB.
// N1 = 224: BN = 480, an N = 256 MMA into TMEM columns 0..255 and an N = 224
//           MMA into columns 256..479 per K step (the scale factors take
//           columns 480..511), 4 stages of 46 KB; a tile whose columns from
//           256 on all lie beyond n_pad issues only the first MMA.
// KIND 1: packed E2M1 operands, kind::mxf4 with unit scale factors (256 elements per 128-byte K block);
// KIND 0: E4M3 operands, kind::f8f6f4 (128 elements per 128-byte K block, no scale factors, so the second MMA can
// be N = 256 and all 512 TMEM columns hold accumulators).
template <int KIND, int N1>
struct Duo {
    static constexpr int BN = TC_BN + N1;               // output columns of a pair tile
    static constexpr int B0_ROWS = TC_BN / 2;           // this CTA's rows of the N = 256 part
    static constexpr int B1_ROWS = N1 / 2;              // and of the N1 part
    static constexpr int A_BYTES = TC_BM * F4_BK;       // 16 KiB
    static constexpr int B0_BYTES = B0_ROWS * F4_BK;    // 16 KiB
    static constexpr int B1_BYTES = B1_ROWS * F4_BK;
    static constexpr int B_BYTES = B0_BYTES + B1_BYTES;
    static constexpr int STAGES = N1 ? 4 : 6;
    static constexpr int CHUNKS = BN / 32;              // 32-column chunks of the epilogue
    static constexpr int SFA_COL = N1 ? 480 : 256;      // E2M1 scale factors (all 2^0; with N1 both operands
    static constexpr int SFB_COL = N1 ? 480 : 384;      // read the same filled columns)
    static constexpr int SF_FILL = N1 ? 32 : 0;         // N1: columns 480..511 hold 2^0 scales
    static constexpr int OFF_A = 0;
    static constexpr int OFF_B = OFF_A + STAGES * A_BYTES;
    static constexpr int OFF_BAR = OFF_B + STAGES * B_BYTES;
    static constexpr int NUM_BARS = 2 * STAGES + 3;     // full[], empty[], tfull, tempty, done
    static constexpr int OFF_MISC = OFF_BAR + NUM_BARS * 8;
    static constexpr int SMEM_BYTES = OFF_MISC + 16 + 1024;
    static_assert(N1 == 0 || (N1 % 32 == 0 && N1 <= (KIND ? 224 : 256)), "second MMA width");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
    static_assert(B_BYTES % 1024 == 0 && A_BYTES % 1024 == 0, "swizzle atoms stay 1024-byte aligned");
};

// Second MMA width of the squaring kernel's pair tile (BN = 480). Measured on GB300 at n = 32,768: 8.88 PFLOP/s
// against 7.33 for the 256-column tile (N1 = 0), which reads a third more operand bytes per Boolean operation.
constexpr int TC4_N1 = 224;
// The E4M3 form has no scale factors in TMEM, so its pair tile is 256 x 512 (two N = 256 MMAs per K step).
constexpr int TC8_N1 = 256;

constexpr int ERR_D_PRODUCER = 0x211;
constexpr int ERR_D_MMA = 0x212;
constexpr int ERR_D_EPILOGUE = 0x213;

// 32 accumulator counts (FP32, exact integers 0 .. 2^24) -> bit j = (count j > 0).
// The top byte of a count is 0 for 0 and 0x3F .. 0x4B for 1 .. 2^24, so adding
// 0x41 sets its bit 7 exactly for the nonzero counts, without a carry into the
// next byte. Word k gathers the top bytes of columns k, 8 + k, 16 + k and
// 24 + k with byte permutes, so that its flags (bits 7, 15, 23, 31) shifted
// right by 7 - k land on bits k, 8 + k, 16 + k, 24 + k: six integer operations
// per four counts instead of a compare and a select for each.
__device__ __forceinline__ uint32_t f4_threshold32(const uint32_t (&v)[32]) {
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t lo = __byte_perm(v[k], v[8 + k], 0x0073);        // top bytes in bytes 0, 1
        const uint32_t hi = __byte_perm(v[16 + k], v[24 + k], 0x7300);  // and in bytes 2, 3
        const uint32_t w = __byte_perm(lo, hi, 0x7610) + 0x41414141u;
        bits |= (w >> (7 - k)) & (0x80808080u >> (7 - k));
    }
    return bits;
}

// Epilogue, part 1: C > 0 for the accumulator columns of this thread's TMEM
// lane, as CHUNKS x 32 bits. The load of chunk c + 1 is in flight while chunk
// c is thresholded.
template <int CHUNKS>
__device__ __forceinline__ void f4_drain(uint32_t taddr, uint32_t (&cb)[CHUNKS]) {
    uint32_t va[32], vb[32];
    tmem_ld_32x32b_x32(taddr, va);
#pragma unroll
    for (int c = 0; c < CHUNKS; ++c) {
        uint32_t(&cur)[32] = (c & 1) ? vb : va;
        tmem_ld_wait_regs(cur);
        if (c + 1 < CHUNKS) tmem_ld_32x32b_x32(taddr + static_cast<uint32_t>((c + 1) * 32), (c & 1) ? va : vb);
        cb[c] = f4_threshold32(cur);
    }
}

// cb[c] for a run-time c through selects, so that cb stays in registers.
template <int CHUNKS>
__device__ __forceinline__ uint32_t f4_pick(const uint32_t (&cb)[CHUNKS], int c) {
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < CHUNKS; ++j) v = (j == c) ? cb[j] : v;
    return v;
}

// Epilogue, part 2: R' = R | C for row (mb, quarter, lane) of the pair tile
// whose first column is col_base: writes R' and, through warp ballots, R'^T
// for every 32-column chunk below n_pad; returns the bits that changed
// (nonzero in some lane iff R' != R in this warp's rows).
// E4M3 bytes: 4 bytes -> 4 bits (bit k = byte k nonzero), and back (0 / one).
__device__ __forceinline__ uint32_t e4_bits4(uint32_t w) {
    const uint32_t x = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
    return ((x >> 7) & 1u) | ((x >> 14) & 2u) | ((x >> 21) & 4u) | ((x >> 28) & 8u);
}
__device__ __forceinline__ uint32_t e4_bits16(const uint4& v) {
    return e4_bits4(v.x) | (e4_bits4(v.y) << 4) | (e4_bits4(v.z) << 8) | (e4_bits4(v.w) << 12);
}
__device__ __forceinline__ uint32_t e4_bytes4(uint32_t b) {
    const uint32_t t = b & 0xFu;
    return ((t | (t << 7) | (t << 14) | (t << 21)) & 0x01010101u) * static_cast<uint32_t>(BMLP_E4M3_ONE);
}
__device__ __forceinline__ uint4 e4_bytes16(uint32_t m) {
    return make_uint4(e4_bytes4(m), e4_bytes4(m >> 4), e4_bytes4(m >> 8), e4_bytes4(m >> 12));
}

// 32 columns of a row as bits, and back, in the operand form of KIND.
template <int KIND>
__device__ __forceinline__ uint32_t load_bits32(const uint8_t* p) {
    if (KIND) return f4_bits32(*reinterpret_cast<const uint4*>(p));
    return e4_bits16(reinterpret_cast<const uint4*>(p)[0]) | (e4_bits16(reinterpret_cast<const uint4*>(p)[1]) << 16);
}
template <int KIND>
__device__ __forceinline__ void store_bits32(uint8_t* p, uint32_t bits) {
    if (KIND) {
        *reinterpret_cast<uint4*>(p) = f4_nibbles32(bits);
    } else {
        reinterpret_cast<uint4*>(p)[0] = e4_bytes16(bits & 0xFFFFu);
        reinterpret_cast<uint4*>(p)[1] = e4_bytes16(bits >> 16);
    }
}

template <int KIND, int CHUNKS>
__device__ __forceinline__ uint32_t f4_update(const TcParams& p, int mb, int64_t col_base, int64_t n_pad, int quarter,
                                              int lane, const uint32_t (&cb)[CHUNKS]) {
    constexpr int CB = KIND ? 16 : 32;  // bytes of 32 columns
    const int64_t row = static_cast<int64_t>(mb) * TC_BM + quarter * 32 + lane;
    // byte of this warp's 32 rows inside a row of R'^T
    const int64_t rt_col = (static_cast<int64_t>(mb) * TC_BM + quarter * 32) / 32 * CB;
    uint32_t any = 0;
#pragma unroll 1
    for (int c = 0; c < CHUNKS; ++c) {
        const int64_t col0 = col_base + c * 32;
        if (col0 >= n_pad) break;
        const int64_t off = row * p.ld + col0 / 32 * CB;
        const uint32_t obits = load_bits32<KIND>(p.old_r + off);
        const uint32_t nbits = obits | f4_pick(cb, c);
        any |= nbits ^ obits;
        store_bits32<KIND>(p.out_r + off, nbits);
        if (p.out_bits != nullptr) p.out_bits[row * p.ldb + col0 / 32] = nbits;
        // column col0 + j of these 32 rows is row col0 + j of R'^T: lane j gathers it
        uint32_t mine = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, (nbits >> j) & 1u);
            mine = (lane == j) ? b : mine;
        }
        store_bits32<KIND>(p.out_rt + (col0 + lane) * p.ld + rt_col, mine);
        if (p.out_bits_t != nullptr) p.out_bits_t[(col0 + lane) * p.ldb + rt_col / CB] = mine;
    }
    return any;
}

// tmA: A = R (box 128 rows x 128 bytes); tmB0 / tmB1: B^T = R^T (boxes of
// B0_ROWS / B1_ROWS rows x 128 bytes; tmB1 unused when N1 = 0).
template <int KIND, int N1>
__global__ void __launch_bounds__(TC_THREADS, 1) __cluster_dims__(2, 1, 1)
tc_duo_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
               const __grid_constant__ CUtensorMap tmB1, const TcParams p) {
    using C = Duo<KIND, N1>;
    // a step of a device-side loop that was switched off: every CTA of every pair leaves before it allocates TMEM or
    // touches a barrier (they all read the same word, written by an earlier kernel in stream order)
    if (p.guard != nullptr && *reinterpret_cast<const volatile int*>(p.guard) == 0) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem + C::OFF_A;
    uint8_t* sB = smem + C::OFF_B;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    uint64_t* full = bars;                  // even CTA: both CTAs' copies of a stage complete here
    uint64_t* empty = bars + C::STAGES;     // each CTA: the even CTA's MMAs released the stage
    uint64_t* tfull = bars + 2 * C::STAGES; // each CTA: the accumulator holds a finished tile
    uint64_t* tempty = tfull + 1;           // even CTA: both CTAs' epilogues drained the accumulator
    uint64_t* done = tempty + 1;            // even CTA: every MMA it issued has completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::OFF_MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    const int m_pairs = p.m_tiles / 2;
    const int num_pairs = m_pairs * p.n_tiles;
    const int first = static_cast<int>(blockIdx.x >> 1);
    const int step = static_cast<int>(gridDim.x >> 1);
    const long long limit = p.wait_cycles;
    const int64_t n_pad = static_cast<int64_t>(p.m_tiles) * TC_BM;

    if (threadIdx.x == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB0);
        if (N1) tma_prefetch_desc(&tmB1);
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, 256);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc_2sm(tmem_slot, F4_TMEM_COLS);
        tmem_relinquish_2sm();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (KIND == 1 && warp >= 2) {
        // every scale factor of A and B is 2^0, in all 128 lanes of this CTA
        const uint32_t lanes = static_cast<uint32_t>((warp & 3) * 32) << 16;
        const uint32_t ones[8] = {F4_UE8M0_ONE4, F4_UE8M0_ONE4, F4_UE8M0_ONE4, F4_UE8M0_ONE4,
                                  F4_UE8M0_ONE4, F4_UE8M0_ONE4, F4_UE8M0_ONE4, F4_UE8M0_ONE4};
        if (C::SF_FILL) {
#pragma unroll
            for (int c = 0; c < C::SF_FILL; c += 8)
                tmem_st_32x32b_x8(tmem_base + lanes + static_cast<uint32_t>(C::SFA_COL + c), ones);
        } else {
            tmem_st_32x32b_x8(tmem_base + lanes + C::SFA_COL, ones);
            tmem_st_32x32b_x8(tmem_base + lanes + C::SFB_COL, ones);
        }
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // barriers and scale factors of both CTAs are in place
    tc_fence_after();

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            bool issued = false;
            for (int t = first; t < num_pairs && ok; t += step) {
                int mp, nb;
                f4_pair_coords(t, m_pairs, p.n_tiles, mp, nb);
                const int mb = 2 * mp + static_cast<int>(rank);
                const int64_t col_base = static_cast<int64_t>(nb) * C::BN;
                const bool has1 = N1 != 0 && col_base + TC_BN < n_pad;
                const uint32_t tx = 2u * static_cast<uint32_t>(C::A_BYTES + C::B0_BYTES + (has1 ? C::B1_BYTES : 0));
                for (int kb = 0; kb < p.k_blocks; ++kb) {
                    if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, limit)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bar = mapa_shared(smem_u32(&full[stage]), 0);
                    if (leader) mbar_arrive_expect_tx(&full[stage], tx);
                    uint8_t* sb = sB + stage * C::B_BYTES;
                    tma_load_2d_2sm(sA + stage * C::A_BYTES, &tmA, kb * F4_BK, mb * TC_BM, bar);
                    tma_load_2d_2sm(sb, &tmB0, kb * F4_BK,
                                    static_cast<int>(col_base) + static_cast<int>(rank) * C::B0_ROWS, bar);
                    if (has1)
                        tma_load_2d_2sm(sb + C::B0_BYTES, &tmB1, kb * F4_BK,
                                        static_cast<int>(col_base) + TC_BN + static_cast<int>(rank) * C::B1_ROWS,
                                        bar);
                    issued = true;
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                atomicCAS(p.error, 0, ERR_D_PRODUCER);
                // copies complete on the even CTA's barriers: give the last ones time to land
                if (issued) {
                    const long long t0 = clock64();
                    while (clock64() - t0 < 2000000) __nanosleep(1000);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (even CTA)
        if (leader) {
            const uint32_t idesc0 = KIND ? idesc_mxf4_ue8m0(2 * TC_BM, TC_BN) : idesc_e4m3_f32(2 * TC_BM, TC_BN);
            const uint32_t idesc1 = KIND ? idesc_mxf4_ue8m0(2 * TC_BM, N1 ? N1 : TC_BN)
                                         : idesc_e4m3_f32(2 * TC_BM, N1 ? N1 : TC_BN);
            const uint32_t sfa = tmem_base + C::SFA_COL, sfb = tmem_base + C::SFB_COL;
            int stage = 0;
            uint32_t phase = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (int t = first; t < num_pairs && ok; t += step) {
                int mp, nb;
                f4_pair_coords(t, m_pairs, p.n_tiles, mp, nb);
                const bool has1 = N1 != 0 && static_cast<int64_t>(nb) * C::BN + TC_BN < n_pad;
                if (!f4_wait_lane0(tempty, acc_phase ^ 1u, abort_flag, limit, lane)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint32_t accumulate = 0;
                for (int kb = 0; kb < p.k_blocks; ++kb) {
                    if (!f4_wait_lane0(&full[stage], phase, abort_flag, limit, lane)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (lane == 0) {
                        const uint32_t a0 = smem_u32(sA + stage * C::A_BYTES);
                        const uint32_t b0 = smem_u32(sB + stage * C::B_BYTES);
#pragma unroll
                        for (int k = 0; k < F4_BK / F4_UMMA_K_BYTES; ++k) {
                            const uint64_t ad = smem_desc_kmajor_sw128(a0 + k * F4_UMMA_K_BYTES);
                            const uint64_t bd0 = smem_desc_kmajor_sw128(b0 + k * F4_UMMA_K_BYTES);
                            const uint64_t bd1 = smem_desc_kmajor_sw128(b0 + C::B0_BYTES + k * F4_UMMA_K_BYTES);
                            if (KIND) {
                                tc_mma_mxf4_2sm(tmem_base, ad, bd0, idesc0, sfa, sfb, accumulate);
                                if (has1) tc_mma_mxf4_2sm(tmem_base + TC_BN, ad, bd1, idesc1, sfa, sfb, accumulate);
                            } else {
                                tc_mma_f8_2sm(tmem_base, ad, bd0, idesc0, accumulate);
                                if (has1) tc_mma_f8_2sm(tmem_base + TC_BN, ad, bd1, idesc1, accumulate);
                            }
                            accumulate = 1;
                        }
                        tc_commit_2sm_mcast(&empty[stage], 0x3);  // the stage is free in both CTAs
                    }
                    __syncwarp();
                    accumulate = 1;
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                // multiply-adds issued, in units of 128 x 32 x 128: per K block two 128-row halves, one (E4M3) or
                // two (E2M1) 128-deep parts and 8 (+ N1 / 32) column chunks
                if (lane == 0 && p.issued != nullptr)
                    atomicAdd(p.issued, (KIND ? 4ull : 2ull) *
                                            static_cast<unsigned long long>(TC_BN / 32 + (has1 ? N1 / 32 : 0)) *
                                            static_cast<unsigned long long>(p.k_blocks));
                if (lane == 0) tc_commit_2sm_mcast(tfull, 0x3);
                __syncwarp();
                acc_phase ^= 1u;
            }
            if (!ok && lane == 0) atomicCAS(p.error, 0, ERR_D_MMA);
            if (lane == 0) {
                tc_commit_2sm_mcast(done, 0x1);
                volatile int never = 0;
                mbar_wait_bounded(done, 0, &never, f4_drain_cycles(limit));
            }
            __syncwarp();
        }
    } else {
        // ------------------------------------------------ epilogue (both CTAs)
        const int quarter = warp & 3;
        const uint32_t lanes = static_cast<uint32_t>(quarter * 32) << 16;
        const uint32_t tempty_even = mapa_shared(smem_u32(tempty), 0);
        uint32_t acc_phase = 0;
        for (int t = first; t < num_pairs; t += step) {
            int mp, nb;
            f4_pair_coords(t, m_pairs, p.n_tiles, mp, nb);
            const int mb = 2 * mp + static_cast<int>(rank);
            if (!f4_wait_lane0(tfull, acc_phase, abort_flag, limit, lane)) {
                if (lane == 0) atomicCAS(p.error, 0, ERR_D_EPILOGUE);
                break;
            }
            tc_fence_after();
            // drain C > 0 into registers, then free the accumulator for the next tile's MMAs (columns of a
            // tile that got no second MMA hold stale counts; f4_update stops before them)
            uint32_t cb[C::CHUNKS];
            f4_drain<C::CHUNKS>(tmem_base + lanes, cb);
            tc_fence_before();
            mbar_arrive_cluster(tempty_even);
            acc_phase ^= 1u;
            const uint32_t any =
                f4_update<KIND, C::CHUNKS>(p, mb, static_cast<int64_t>(nb) * C::BN, n_pad, quarter, lane, cb);
            if (__any_sync(0xFFFFFFFFu, any != 0) && lane == 0) atomicOr(p.changed, 1);
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();  // the even CTA's MMAs into this CTA's TMEM have completed
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_2sm(tmem_base, F4_TMEM_COLS);
    }
}

// E4M3 bytes (0 / nonzero) -> packed E2M1 nibbles, 16 bytes -> 8 bytes per thread.
__global__ void e4m3_to_e2m1_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int64_t bytes_in) {
    const int64_t chunks = bytes_in / 16;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < chunks;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4*>(in)[i];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint32_t bits = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int b = 0; b < 4; ++b) bits |= (((w[q] >> (8 * b)) & 0xFFu) != 0 ? 1u : 0u) << (4 * q + b);
        reinterpret_cast<uint2*>(out)[i] = make_uint2(f4_spread8(bits), f4_spread8(bits >> 8));
    }
}

// Packed E2M1 nibbles -> E4M3 bytes (0 / one), 8 bytes -> 16 bytes per thread.
__global__ void e2m1_to_e4m3_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int64_t bytes_out) {
    const int64_t chunks = bytes_out / 16;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < chunks;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint2 v = reinterpret_cast<const uint2*>(in)[i];
        const uint32_t bits = f4_gather8(v.x) | (f4_gather8(v.y) << 8);
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t x = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                x |= (((bits >> (4 * q + b)) & 1u) ? static_cast<uint32_t>(BMLP_E4M3_ONE) : 0u) << (8 * b);
            w[q] = x;
        }
        reinterpret_cast<uint4*>(out)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

int f4_grid(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

}  // namespace

template <int KIND, int N1>
cudaError_t launch_duo(const CUtensorMap& a, const CUtensorMap& b0, const CUtensorMap& b1, const TcParams& p, int sms,
                       cudaStream_t s) {
    // set on every launch: the attribute belongs to the current device, and a call costs well under a microsecond
    cudaError_t e = cudaFuncSetAttribute(tc_duo_kernel<KIND, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Duo<KIND, N1>::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int pairs = (p.m_tiles / 2) * p.n_tiles;
    int clusters = sms / 2;
    if (clusters > pairs) clusters = pairs;
    if (clusters < 1) clusters = 1;
    tc_duo_kernel<KIND, N1><<<2 * clusters, TC_THREADS, Duo<KIND, N1>::SMEM_BYTES, s>>>(a, b0, b1, p);
    return cudaGetLastError();
}

int tc4_tile_n() { return Duo<1, TC4_N1>::BN; }
int tc4_b1_rows() { return Duo<1, TC4_N1>::B1_ROWS; }
int tc8_tile_n() { return Duo<0, TC8_N1>::BN; }

cudaError_t launch_tc4_product_duo(const CUtensorMap& a, const CUtensorMap& b0, const CUtensorMap& b1,
                                   const TcParams& p, int sms, cudaStream_t s) {
    return launch_duo<1, TC4_N1>(a, b0, b1, p, sms, s);
}

cudaError_t launch_tc8_product_duo(const CUtensorMap& a, const CUtensorMap& b_half, const TcParams& p, int sms,
                                   cudaStream_t s) {
    return launch_duo<0, TC8_N1>(a, b_half, b_half, p, sms, s);
}

void launch_e4m3_to_e2m1(const uint8_t* in, uint8_t* out, int64_t bytes_in, cudaStream_t s) {
    e4m3_to_e2m1_kernel<<<f4_grid(bytes_in / 16, 256), 256, 0, s>>>(in, out, bytes_in);
}

void launch_e2m1_to_e4m3(const uint8_t* in, uint8_t* out, int64_t bytes_out, cudaStream_t s) {
    e2m1_to_e4m3_kernel<<<f4_grid(bytes_out / 16, 256), 256, 0, s>>>(in, out, bytes_out);
}

}  // namespace bmlp
