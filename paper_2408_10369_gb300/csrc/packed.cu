// Bit-packed kernels: rows of R are uint64 bit codes (paper Sec. 3.2, bit j
// of row i = R_ij, least significant bit first).
//
//  * product_m4rm / product_gather  one Boolean product on bitsets,
//                 C_i = OR_{k : A_ik = 1} B_k, optionally OR-ed with A_i; with
//                 A = B = R that is one squaring step of Eq. 4:
//                 C_i = R_i | OR_{k : R_ik = 1} R_k. Dense words: tiles of 256
//                 rows x 1,024 columns, per word of A 16 shared-memory tables
//                 of the ORs of 4 rows of B (Four Russians), one lookup per
//                 nibble; few bits per word: one warp per row gathers the
//                 named rows of B.
//  * wcsr_build   the nonzero words of every row (word index + value), so
//                 that frontier expansion touches only words that hold bits.
//  * smp_packed   the selective product of Eq. 5 / Algorithm 2 per query row:
//                 D = v; V = 0; repeat N = (OR_{k in D} R_k) & ~V; V |= N;
//                 D = N until D is empty; out = V = v R+.
//                 One warp per query row, frontier and next bitsets in shared
//                 memory, the visited set in the query's output row, all
//                 frontier levels of a query in one launch
//                 (queries are independent, so no grid-wide step is needed;
//                 a warp takes the next query from a global counter when its
//                 query has converged).
//  * square_rows  R + R R through the word index, before the frontier closure
//                 of a path-like relation (same closure, fewer levels).
//  * smp_cluster  Algorithm 2 for 64 sources or 64 query rows at once,
//                 bit-sliced, with the frontier spread over the shared
//                 memory of a thread-block cluster (read through DSMEM).
//  * insert_fact  one new fact into a transitive closure (rank-1 update).
#include "internal.h"
#include "ptx.cuh"

namespace bmlp {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// 64 x 64 bit transpose across a warp: lane l holds rows l (a0) and l + 32 (a1) and receives columns l (c0) and
// l + 32 (c1), where bit r of column c is bit c of row r.
__device__ __forceinline__ void warp_transpose64(uint64_t a0, uint64_t a1, int lane, uint64_t& c0, uint64_t& c1) {
    c0 = 0ull;
    c1 = 0ull;
#pragma unroll 8
    for (int j = 0; j < 64; ++j) {
        const unsigned lo = __ballot_sync(FULL, ((a0 >> j) & 1ull) != 0ull);
        const unsigned hi = __ballot_sync(FULL, ((a1 >> j) & 1ull) != 0ull);
        const uint64_t col = static_cast<uint64_t>(lo) | (static_cast<uint64_t>(hi) << 32);
        if (j == lane) c0 = col;
        if (j == lane + 32) c1 = col;
    }
}

__device__ __forceinline__ void or4(uint4& a, const uint4& b) {
    a.x |= b.x;
    a.y |= b.y;
    a.z |= b.z;
    a.w |= b.w;
}

// Ones and nonzero words of two output words (a uint4), and a block's totals added into pstat[0] / pstat[1]
// (called by every thread of the block: one pair of atomics per block, since all blocks add to the same two words).
__device__ __forceinline__ void count_words(const uint4& v, unsigned long long& ones, unsigned long long& words) {
    ones += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
    words += ((v.x | v.y) != 0u ? 1u : 0u) + ((v.z | v.w) != 0u ? 1u : 0u);
}
__device__ __forceinline__ void block_add_counts(unsigned long long* pstat, unsigned long long ones,
                                                 unsigned long long words) {
    __shared__ unsigned long long part[2][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ones += __shfl_xor_sync(FULL, ones, off);
        words += __shfl_xor_sync(FULL, words, off);
    }
    if (lane == 0) {
        part[0][warp] = ones;
        part[1][warp] = words;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = static_cast<int>(blockDim.x >> 5);
        ones = lane < nw ? part[0][lane] : 0ull;
        words = lane < nw ? part[1][lane] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ones += __shfl_xor_sync(FULL, ones, off);
            words += __shfl_xor_sync(FULL, words, off);
        }
        if (lane == 0 && (ones | words) != 0ull) {
            atomicAdd(pstat, ones);
            atomicAdd(pstat + 1, words);
        }
    }
}

// ---- one Boolean product on bit rows by gathering the named rows
// C_i = (A_i if or_a) OR (OR over the set bits k of A_i of B_k): one warp per row i; the set bits of A_i are found
// with warp ballots and find-first-set, and row k is ORed in with coalesced 128-bit loads (two rows in flight).
// Its work is nnz(A_i) rows of B per row: the form for rows with few bits per nonzero word.
template <int VEC>
__global__ void __launch_bounds__(256) product_gather_kernel(const uint64_t* __restrict__ A, const uint64_t* __restrict__ B,
                                                             uint64_t* __restrict__ dst, int64_t n, int64_t ldw, int or_a,
                                                             int* changed, Deadline dl,
                                                             unsigned long long* __restrict__ pstat) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t chunk_words = 64 * VEC;  // 32 lanes x VEC x 2 words
    uint32_t any = 0;
    unsigned long long ones = 0, words = 0;  // of the rows written
    for (int64_t i = warp_id; i < n; i += nwarps) {
        if (dl.budget_ns && __shfl_sync(FULL, lane == 0 ? static_cast<int>(dl.past()) : 0, 0)) break;
        const uint64_t* arow = A + i * ldw;
        for (int64_t c0 = 0; c0 < ldw; c0 += chunk_words) {
            uint4 acc[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int64_t w = c0 + 2 * (lane + 32 * v);
                acc[v] = (or_a && w < ldw) ? *reinterpret_cast<const uint4*>(arow + w) : make_uint4(0, 0, 0, 0);
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
                        int b1 = -1;
                        if (bits) {
                            b1 = __ffsll(static_cast<long long>(bits)) - 1;
                            bits &= bits - 1;
                        }
                        const uint64_t* r0 = B + (kbase + b0) * ldw + c0;
                        const uint64_t* r1 = B + (kbase + (b1 < 0 ? b0 : b1)) * ldw + c0;
                        uint4 x0[VEC], x1[VEC];
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const int64_t w = 2 * (lane + 32 * v);
                            if (c0 + w < ldw) {
                                x0[v] = __ldg(reinterpret_cast<const uint4*>(r0 + w));
                                x1[v] = __ldg(reinterpret_cast<const uint4*>(r1 + w));
                            } else {
                                x0[v] = make_uint4(0, 0, 0, 0);
                                x1[v] = x0[v];
                            }
                        }
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            or4(acc[v], x0[v]);
                            or4(acc[v], x1[v]);
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const int64_t w = c0 + 2 * (lane + 32 * v);
                if (w < ldw) {
                    const uint4 o = *reinterpret_cast<const uint4*>(arow + w);  // A_i: the squaring's old row
                    any |= (o.x ^ acc[v].x) | (o.y ^ acc[v].y) | (o.z ^ acc[v].z) | (o.w ^ acc[v].w);
                    *reinterpret_cast<uint4*>(dst + i * ldw + w) = acc[v];
                    if (pstat != nullptr) count_words(acc[v], ones, words);
                }
            }
        }
    }
    if (__any_sync(FULL, any != 0) && lane == 0) atomicOr(changed, 1);
    if (pstat != nullptr) block_add_counts(pstat, ones, words);
}

// ---- one Boolean product on bit rows by the method of Four Russians (Arlazarov, Dinic, Kronrod, Faradzev 1970)
// C_i = (A_i if or_a) OR (OR over the set bits k of A_i of B_k). A CTA owns a tile of kM4Rows rows and kM4Cols
// words (64 kM4Cols columns) of C and walks k one word of A (64 values of k) at a time. For each nibble h of that
// word it tabulates, in shared memory, the 16 ORs of the four B rows 64 kw + 4 h .. 64 kw + 4 h + 3 over the tile's
// columns; a row then ORs in one table entry per nibble of each nonzero word of A_i instead of one B row per set
// bit. So an output word costs at most n / 4 shared-memory reads however dense A is, where gathering the named
// rows costs nnz(A_i) reads of B through L2. Every nibble of a nonzero word is looked up, zero or not (measured
// faster than testing each: the loads issue back to back). The tables are double buffered (one barrier per word
// of A), and the B words of the next table are loaded while the current one is read.
// Thread layouts: a table is built by thread (h = tid / 16, column word c = tid % 16), entry x at T[h][x][c]; a
// lookup thread owns row slot r = tid / 8 (rows r, r + 32, ..., r + 224 of the tile) and the column words
// 2 (tid % 8), 2 (tid % 8) + 1, so each row slot reads one whole 128-byte entry per lookup (no bank conflicts).
constexpr int kM4Threads = 256;
constexpr int kM4Cols = 16;
constexpr int kM4Rows = 256;
constexpr int kM4RowsPerThread = kM4Rows / (kM4Threads / 8);
constexpr int kM4TableWords = 16 * 16 * kM4Cols;  // one buffer: 16 nibbles x 16 values x kM4Cols words (32 KiB)
constexpr size_t kM4Smem = 2 * kM4TableWords * sizeof(uint64_t);

__global__ void __launch_bounds__(kM4Threads, 2) product_m4rm_kernel(const uint64_t* __restrict__ A,
                                                                     const uint64_t* __restrict__ B,
                                                                     uint64_t* __restrict__ dst, int64_t n,
                                                                     int64_t ldw, int or_a, int* changed, Deadline dl,
                                                                     unsigned long long* __restrict__ pstat) {
    extern __shared__ __align__(16) uint64_t m4t[];
    const int tid = threadIdx.x;
    const int64_t nch = (ldw + kM4Cols - 1) / kM4Cols;
    const int64_t row0 = (static_cast<int64_t>(blockIdx.x) / nch) * kM4Rows;
    const int64_t c0 = (static_cast<int64_t>(blockIdx.x) % nch) * kM4Cols;
    const int64_t kwn = (n + 63) >> 6;  // words of A that hold columns < n
    // table building: B words of column c0 + bc for rows 64 kw + 4 bh + q
    const int bh = tid >> 4, bc = tid & 15;
    const bool bcol = c0 + bc < ldw;
    auto load_b = [&](int64_t kw, uint64_t (&b)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t k = kw * 64 + bh * 4 + q;
            b[q] = (bcol && k < n) ? B[k * ldw + c0 + bc] : 0ull;
        }
    };
    auto build = [&](int buf, const uint64_t (&b)[4]) {
        uint64_t* t = m4t + buf * kM4TableWords + bh * 16 * kM4Cols + bc;
        const uint64_t e3 = b[0] | b[1], e5 = b[2] | b[0], e6 = b[2] | b[1], e7 = b[2] | e3;
        t[0 * kM4Cols] = 0ull;
        t[1 * kM4Cols] = b[0];
        t[2 * kM4Cols] = b[1];
        t[3 * kM4Cols] = e3;
        t[4 * kM4Cols] = b[2];
        t[5 * kM4Cols] = e5;
        t[6 * kM4Cols] = e6;
        t[7 * kM4Cols] = e7;
        t[8 * kM4Cols] = b[3];
        t[9 * kM4Cols] = b[3] | b[0];
        t[10 * kM4Cols] = b[3] | b[1];
        t[11 * kM4Cols] = b[3] | e3;
        t[12 * kM4Cols] = b[3] | b[2];
        t[13 * kM4Cols] = b[3] | e5;
        t[14 * kM4Cols] = b[3] | e6;
        t[15 * kM4Cols] = b[3] | e7;
    };
    // lookups: rows row0 + lr + 32 j, words c0 + 2 lc, c0 + 2 lc + 1
    const int lr = tid >> 3, lc = tid & 7;
    const int64_t wcol = c0 + 2 * lc;  // ldw is even, so wcol < ldw covers both words
    uint4 acc[kM4RowsPerThread];
#pragma unroll
    for (int j = 0; j < kM4RowsPerThread; ++j) {
        const int64_t i = row0 + lr + 32 * j;
        acc[j] = (or_a && i < n && wcol < ldw) ? *reinterpret_cast<const uint4*>(A + i * ldw + wcol)
                                               : make_uint4(0, 0, 0, 0);
    }
    uint64_t bq[4];
    if (kwn > 0) {
        load_b(0, bq);
        build(0, bq);
    }
    for (int64_t kw = 0; kw < kwn; ++kw) {
        int stop = 0;
        if (tid == 0 && dl.budget_ns && (kw & 63) == 0) stop = dl.past() ? 1 : 0;
        // table kw is complete, and every thread is done with table kw - 1, whose buffer the next build reuses
        if (__syncthreads_or(stop)) return;
        if (kw + 1 < kwn) load_b(kw + 1, bq);
        uint64_t aw[kM4RowsPerThread];
#pragma unroll
        for (int j = 0; j < kM4RowsPerThread; ++j) {
            const int64_t i = row0 + lr + 32 * j;
            aw[j] = i < n ? A[i * ldw + kw] : 0ull;
        }
        const char* tb = reinterpret_cast<const char*>(m4t + (kw & 1) * kM4TableWords) + lc * 16;
#pragma unroll
        for (int j = 0; j < kM4RowsPerThread; ++j) {
            if (aw[j] == 0ull) continue;
#pragma unroll
            for (int h = 0; h < 16; ++h) {
                const uint32_t half = h < 8 ? static_cast<uint32_t>(aw[j]) : static_cast<uint32_t>(aw[j] >> 32);
                const uint32_t x = (half >> (4 * (h & 7))) & 15u;  // entry 0 is zero: no test needed
                const uint4 v = *reinterpret_cast<const uint4*>(tb + (h * 16 + x) * (kM4Cols * 8));
                acc[j].x |= v.x;
                acc[j].y |= v.y;
                acc[j].z |= v.z;
                acc[j].w |= v.w;
            }
        }
        if (kw + 1 < kwn) build(static_cast<int>((kw + 1) & 1), bq);
    }
    uint32_t any = 0;
    unsigned long long ones = 0, words = 0;
#pragma unroll
    for (int j = 0; j < kM4RowsPerThread; ++j) {
        const int64_t i = row0 + lr + 32 * j;
        if (i < n && wcol < ldw) {
            const uint4 o = *reinterpret_cast<const uint4*>(A + i * ldw + wcol);  // A_i: the squaring's old row
            any |= (o.x ^ acc[j].x) | (o.y ^ acc[j].y) | (o.z ^ acc[j].z) | (o.w ^ acc[j].w);
            *reinterpret_cast<uint4*>(dst + i * ldw + wcol) = acc[j];
            if (pstat != nullptr) count_words(acc[j], ones, words);
        }
    }
    if (__any_sync(FULL, any != 0) && (tid & 31) == 0) atomicOr(changed, 1);
    if (pstat != nullptr) block_add_counts(pstat, ones, words);
}

// ---- word-CSR of packed rows
// Word x of a row of an n x n matrix with its bits at columns >= n cleared (a caller's padding bits are not
// columns; words past ceil(n / 64) are padding too).
__device__ __forceinline__ uint64_t wcsr_columns(uint64_t w, int64_t x, int64_t n) {
    const int64_t nw = (n + 63) >> 6;
    if (x < nw - 1) return w;
    if (x > nw - 1) return 0ull;
    return (n & 63) ? (w & ((1ull << (n & 63)) - 1ull)) : w;
}

// Rows warp_id, warp_id + nwarps, ... of P: their counts of nonzero words into wptr[i + 1].
__device__ __forceinline__ void wcsr_count_rows(const uint64_t* __restrict__ P, int64_t n, int64_t ldw,
                                                int64_t* __restrict__ wptr, int64_t warp_id, int64_t nwarps,
                                                int lane) {
    for (int64_t i = warp_id; i < n; i += nwarps) {
        const uint64_t* row = P + i * ldw;
        int64_t c = 0;
        int64_t wb = 0;
        for (; wb + 128 <= ldw; wb += 128) {  // four loads in flight per lane
            uint64_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = row[wb + 32 * k + lane];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                c += __popc(__ballot_sync(FULL, wcsr_columns(w[k], wb + 32 * k + lane, n) != 0ull));
        }
        for (; wb < ldw; wb += 32) {
            const uint64_t w = (wb + lane < ldw) ? wcsr_columns(row[wb + lane], wb + lane, n) : 0ull;
            c += __popc(__ballot_sync(FULL, w != 0ull));
        }
        if (lane == 0) wptr[i + 1] = c;
        if (i == 0 && lane == 0) wptr[0] = 0;
    }
}

__global__ void wcsr_count_kernel(const uint64_t* __restrict__ P, int64_t n, int64_t ldw, int64_t* __restrict__ wptr) {
    const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    wcsr_count_rows(P, n, ldw, wptr, warp_id, nwarps, threadIdx.x & 31);
}

// In-place inclusive scan of wptr[1..n] by one block of 1024 threads, in tiles of 4,096 counts (4 consecutive
// counts per thread, so a warp reads 1 KB contiguously); wptr[n + 1] = the largest count.
__device__ __forceinline__ void scan_block(int64_t* __restrict__ wptr, int64_t n) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    __shared__ unsigned long long top;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) {
        carry = 0;
        top = 0ull;
    }
    __syncthreads();
    int64_t mx = 0;
    for (int64_t base = 1; base <= n; base += 4096) {
        int64_t v[4];
        int64_t s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t x = base + 4 * t + k;
            const int64_t c = x <= n ? wptr[x] : 0;
            mx = c > mx ? c : mx;
            s += c;
            v[k] = s;  // inclusive within the thread
        }
        int64_t ws = s;  // inclusive over the warp's threads
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, ws, off);
            if (lane >= off) ws += y;
        }
        if (lane == 31) warp_tot[wid] = ws;
        __syncthreads();
        if (wid == 0) {
            int64_t x = warp_tot[lane];  // inclusive over the block's warps
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t y = __shfl_up_sync(FULL, x, off);
                if (lane >= off) x += y;
            }
            warp_tot[lane] = x;
        }
        __syncthreads();
        const int64_t before = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + (ws - s);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t x = base + 4 * t + k;
            if (x <= n) wptr[x] = before + v[k];
        }
        __syncthreads();  // every thread has read carry and warp_tot
        if (t == 0) carry += warp_tot[31];
        __syncthreads();
    }
    atomicMax(&top, static_cast<unsigned long long>(mx));
    __syncthreads();
    if (t == 0) wptr[n + 1] = static_cast<int64_t>(top);
}

__global__ void __launch_bounds__(1024) scan_kernel(int64_t* __restrict__ wptr, int64_t n) { scan_block(wptr, n); }

// The same prefix over many blocks. Pass 1: chunk b, the counts wptr[1 + 4096 b .. 4096 (b + 1)], is scanned in
// place (inclusive within the chunk); sums[b] = its total and sums[chunks + b] = its largest count.
constexpr int kScanChunk = 4096;
__global__ void __launch_bounds__(1024) scan_chunks_kernel(int64_t* __restrict__ wptr, int64_t n,
                                                           int64_t* __restrict__ sums, int chunks) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t warp_max[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t base = 1 + static_cast<int64_t>(blockIdx.x) * kScanChunk + 4 * t;
    int64_t v[4];
    int64_t s = 0, mx = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t c = base + k <= n ? wptr[base + k] : 0;
        mx = c > mx ? c : mx;
        s += c;
        v[k] = s;
    }
    int64_t ws = s;
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, ws, off);
        if (lane >= off) ws += y;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const int64_t y = __shfl_xor_sync(FULL, mx, off);
        mx = y > mx ? y : mx;
    }
    if (lane == 31) warp_tot[wid] = ws;
    if (lane == 0) warp_max[wid] = mx;
    __syncthreads();
    if (wid == 0) {
        int64_t x = warp_tot[lane], m = warp_max[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        for (int off = 16; off > 0; off >>= 1) {
            const int64_t y = __shfl_xor_sync(FULL, m, off);
            m = y > m ? y : m;
        }
        warp_tot[lane] = x;
        if (lane == 31) {
            sums[blockIdx.x] = x;
            sums[chunks + blockIdx.x] = m;
        }
    }
    __syncthreads();
    const int64_t before = (wid > 0 ? warp_tot[wid - 1] : 0) + (ws - s);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k <= n) wptr[base + k] = before + v[k];
}

// Pass 2: chunk b gains the totals of the chunks before it; block 0 writes wptr[0] = 0 and wptr[n + 1] = the
// largest count.
__global__ void __launch_bounds__(1024) scan_add_kernel(int64_t* __restrict__ wptr, int64_t n,
                                                        const int64_t* __restrict__ sums, int chunks) {
    __shared__ int64_t offset;
    const int t = threadIdx.x, lane = t & 31;
    if (t < 32) {
        int64_t o = 0, m = 0;
        for (int b = lane; b < chunks; b += 32) {
            if (b < static_cast<int>(blockIdx.x)) o += sums[b];
            m = sums[chunks + b] > m ? sums[chunks + b] : m;
        }
        for (int off = 16; off > 0; off >>= 1) {
            o += __shfl_xor_sync(FULL, o, off);
            const int64_t y = __shfl_xor_sync(FULL, m, off);
            m = y > m ? y : m;
        }
        if (t == 0) {
            offset = o;
            if (blockIdx.x == 0) {
                wptr[0] = 0;
                wptr[n + 1] = m;
            }
        }
    }
    __syncthreads();
    if (blockIdx.x == 0) return;  // the first chunk's prefix is already final
    const int64_t base = 1 + static_cast<int64_t>(blockIdx.x) * kScanChunk + 4 * t;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k <= n) wptr[base + k] += offset;
}

__device__ __forceinline__ void wcsr_fill_rows(const uint64_t* __restrict__ P, int64_t n, int64_t ldw,
                                               const int64_t* __restrict__ wptr, int32_t* __restrict__ widx,
                                               uint64_t* __restrict__ wval, int64_t warp_id, int64_t nwarps, int lane) {
    const unsigned below = (1u << lane) - 1u;
    for (int64_t i = warp_id; i < n; i += nwarps) {
        const uint64_t* row = P + i * ldw;
        int64_t o = wptr[i];
        int64_t wb = 0;
        for (; wb + 128 <= ldw; wb += 128) {  // four loads in flight per lane
            uint64_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = row[wb + 32 * k + lane];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = wcsr_columns(w[k], wb + 32 * k + lane, n);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned m = __ballot_sync(FULL, w[k] != 0ull);
                if (w[k]) {
                    const int64_t at = o + __popc(m & below);
                    widx[at] = static_cast<int32_t>(wb + 32 * k + lane);
                    wval[at] = w[k];
                }
                o += __popc(m);
            }
        }
        for (; wb < ldw; wb += 32) {
            const uint64_t w = (wb + lane < ldw) ? wcsr_columns(row[wb + lane], wb + lane, n) : 0ull;
            const unsigned m = __ballot_sync(FULL, w != 0ull);
            if (w) {
                const int64_t at = o + __popc(m & below);
                widx[at] = static_cast<int32_t>(wb + lane);
                wval[at] = w;
            }
            o += __popc(m);
        }
    }
}

__global__ void wcsr_fill_kernel(const uint64_t* __restrict__ P, int64_t n, int64_t ldw, const int64_t* __restrict__ wptr,
                                 int32_t* __restrict__ widx, uint64_t* __restrict__ wval) {
    const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    wcsr_fill_rows(P, n, ldw, wptr, widx, wval, warp_id, nwarps, threadIdx.x & 31);
}

// Bit-matrix transpose of n x n packed rows (ldw words each), one 64 x 64
// tile per 64-thread block: out row c, word bi = bit c of the tile's rows.
__device__ __forceinline__ void bit_transpose_tile(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                   int64_t n, int64_t ldw, int64_t bi, int64_t bj, uint64_t* t) {
    const int tid = threadIdx.x;
    const int64_t r = bi * 64 + tid;
    t[tid] = r < n ? in[r * ldw + bj] : 0ull;
    __syncthreads();
    uint64_t o = 0;
#pragma unroll 8
    for (int k = 0; k < 64; ++k) o |= ((t[k] >> tid) & 1ull) << k;
    const int64_t c = bj * 64 + tid;
    if (c < n) out[c * ldw + bi] = o;
    __syncthreads();  // t is reused by the block's next tile
}

// The whole-matrix transpose, a tile of 256 rows (4 groups of 64) x 8 words (512 columns) per block: the tile is
// read with sector-wide loads into shared memory, transposed 64 x 64 at a time by warp ballots (all-zero blocks
// skipped), and written as 512 output rows x 4 words (one 32-byte sector each). Every word of out, padding words
// included, is written.
constexpr int kTrRows = 256, kTrWords = 8;
__global__ void __launch_bounds__(256) bit_transpose_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                            int64_t n, int64_t ldw) {
    __shared__ uint64_t ti[kTrRows][kTrWords + 1];
    __shared__ uint64_t to[kTrWords * 64][5];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * kTrRows;   // first input row
    const int64_t w0 = static_cast<int64_t>(blockIdx.x) * kTrWords;  // first input word
    uint64_t v[kTrRows * kTrWords / 256];  // all of a thread's loads in flight at once
#pragma unroll
    for (int j = 0; j < kTrRows * kTrWords / 256; ++j) {
        const int k = tid + 256 * j, r = k >> 3, w = k & 7;
        const int64_t gr = r0 + r, gw = w0 + w;
        v[j] = (gr < n && gw < ldw) ? in[gr * ldw + gw] : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kTrRows * kTrWords / 256; ++j) {
        const int k = tid + 256 * j;
        ti[k >> 3][k & 7] = v[j];
    }
    __syncthreads();
    for (int b = warp; b < 4 * kTrWords; b += 8) {
        const int g = b / kTrWords, w = b % kTrWords;
        const uint64_t a0 = ti[64 * g + lane][w], a1 = ti[64 * g + lane + 32][w];
        uint64_t c0 = 0ull, c1 = 0ull;
        if (__any_sync(FULL, (a0 | a1) != 0ull)) warp_transpose64(a0, a1, lane, c0, c1);
        to[64 * w + lane][g] = c0;  // output row 64 (w0 + w) + lane, word 4 blockIdx.y + g
        to[64 * w + lane + 32][g] = c1;
    }
    __syncthreads();
    for (int k = tid; k < kTrWords * 64 * 4; k += 256) {
        const int orow = k >> 2, ow = k & 3;
        const int64_t gr = w0 * 64 + orow, gw = static_cast<int64_t>(blockIdx.y) * 4 + ow;
        if (gr < n && gw < ldw) out[gr * ldw + gw] = to[orow][ow];
    }
}

// Direction of a level, by the words each would touch: a push ORs the nonzero words of every frontier
// constant's row (w_out per constant on average); a pull scans an unvisited constant's column words (rows of
// R^T, w_in on average) until one meets the frontier, which on a frontier of nf constants spread over n takes
// about n / nf words, plus PULL_OVERHEAD words' worth of row-range loads per constant. A level pulls when
// nf w_out > nu (PULL_OVERHEAD + min(w_in, n / nf)).
constexpr float PULL_OVERHEAD = 1.0f;

// ---- selective product per query row
// Per warp in shared memory: D, N (ldw words each), FL, the list of the
// frontier's nonzero words (ldw 16-bit word indices), and GM, 64 bytes that
// map a rank to the index of a touched word group. The visited set V is the
// query's own output row in global memory (only its warp touches it). The
// stride is rounded up to 16 bytes so every warp's uint64 arrays stay aligned.
__host__ __device__ __forceinline__ int64_t smp_warp_bytes(int64_t ldw) {
    return (18 * ldw + 64 + 16 + 15) & ~int64_t(15);
}

// Rows of up to NQ frontier constants per lane (k < 0: none) ORed into N:
// their nonzero words, by shared-memory atomics without return value. The row
// ranges and the first four entries of every light row (<= 16 nonzero words)
// are loaded before the first atomic; heavy rows are walked by the whole warp.
// tm collects the word groups written (bit x >> gshift for word x).
template <int NQ>
__device__ __forceinline__ void push_rows(const int64_t (&k)[NQ], int lane, const int64_t* __restrict__ wptr,
                                          const int32_t* __restrict__ widx, const uint64_t* __restrict__ wval,
                                          uint64_t* N, int gshift, uint64_t& tm) {
    int64_t e0[NQ], e1[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int64_t kk = k[q] >= 0 ? k[q] : 0;  // an in-range index even where the value is dropped
        e0[q] = k[q] >= 0 ? wptr[kk] : 0;
        e1[q] = k[q] >= 0 ? wptr[kk + 1] : 0;
    }
    bool light[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) light[q] = k[q] >= 0 && (e1[q] - e0[q]) <= 16;
    int x[NQ][4];
    uint64_t val[NQ][4];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = light[q] && e0[q] + j < e1[q];
            const int64_t ee = in ? e0[q] + j : 0;
            x[q][j] = in ? widx[ee] : -1;
            val[q][j] = in ? wval[ee] : 0ull;
        }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x[q][j] >= 0) {
                atomicOr(reinterpret_cast<unsigned long long*>(&N[x[q][j]]), static_cast<unsigned long long>(val[q][j]));
                tm |= 1ull << (x[q][j] >> gshift);
            }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (light[q])
            for (int64_t e = e0[q] + 4; e < e1[q]; e += 4) {
                int y[4];
                uint64_t yv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t ee = e + j < e1[q] ? e + j : 0;
                    y[j] = e + j < e1[q] ? widx[ee] : -1;
                    yv[j] = e + j < e1[q] ? wval[ee] : 0ull;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (y[j] >= 0) {
                        atomicOr(reinterpret_cast<unsigned long long*>(&N[y[j]]), static_cast<unsigned long long>(yv[j]));
                        tm |= 1ull << (y[j] >> gshift);
                    }
            }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        unsigned hm = __ballot_sync(FULL, k[q] >= 0 && !light[q]);
        while (hm) {
            const int sl = __ffs(hm) - 1;
            hm &= hm - 1;
            const int64_t h0 = __shfl_sync(FULL, e0[q], sl), h1 = __shfl_sync(FULL, e1[q], sl);
            for (int64_t e = h0 + lane; e < h1; e += 32) {
                const int xx = widx[e];
                atomicOr(reinterpret_cast<unsigned long long*>(&N[xx]), static_cast<unsigned long long>(wval[e]));
                tm |= 1ull << (xx >> gshift);
            }
        }
    }
}

// One push step of a lane on its own frontier word d (the constants of word w): up to NQ of its set bits.
template <int NQ>
__device__ __forceinline__ void push_step(uint64_t& d, int64_t w, int lane, const int64_t* __restrict__ wptr,
                                          const int32_t* __restrict__ widx, const uint64_t* __restrict__ wval,
                                          uint64_t* N, int gshift, uint64_t& tm) {
    int64_t k[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        k[q] = -1;
        if (d) {
            const int b = __ffsll(static_cast<long long>(d)) - 1;
            d &= d - 1;
            k[q] = w * 64 + b;
        }
    }
    push_rows<NQ>(k, lane, wptr, widx, wval, N, gshift, tm);
}

// Position of the set bit of rank r (r < popcount) in x.
__device__ __forceinline__ int select_bit(uint64_t x, int r) {
    int pos = 0;
    int c = __popc(static_cast<unsigned>(x));
    if (r >= c) {
        r -= c;
        x >>= 32;
        pos = 32;
    }
    unsigned v = static_cast<unsigned>(x);
    c = __popc(v & 0xFFFFu);
    if (r >= c) { r -= c; v >>= 16; pos += 16; }
    c = __popc(v & 0xFFu);
    if (r >= c) { r -= c; v >>= 8; pos += 8; }
    c = __popc(v & 0xFu);
    if (r >= c) { r -= c; v >>= 4; pos += 4; }
    c = __popc(v & 0x3u);
    if (r >= c) { r -= c; v >>= 2; pos += 2; }
    if (r >= static_cast<int>(v & 1u)) pos += 1;
    return pos;
}

// Push of a chunk of frontier words (lane l holds word d of index w) with the set bits dealt out to the
// lanes in rank order, two per lane per step: a word with many bits (a band of a squared path, a dense
// frontier) is shared by the whole warp instead of being walked by one lane.
__device__ __forceinline__ void push_balanced(uint64_t d, int64_t w, int lane, const int64_t* __restrict__ wptr,
                                              const int32_t* __restrict__ widx, const uint64_t* __restrict__ wval,
                                              uint64_t* N, int gshift, uint64_t& tm) {
    const int c = __popcll(d);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - c;
    for (int base = 0; base < total; base += 64) {
        int64_t k[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = base + q * 32 + lane;
            int owner = 0;  // the lane whose bits hold rank r: the first with inclusive count > r
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int v = __shfl_sync(FULL, incl, owner + st - 1);
                if (v <= r) owner += st;
            }
            const uint64_t od = __shfl_sync(FULL, d, owner);
            const int64_t ow = __shfl_sync(FULL, w, owner);
            const int oex = __shfl_sync(FULL, excl, owner);
            k[q] = r < total ? ow * 64 + select_bit(od, r - oex) : -1;
        }
        push_rows<2>(k, lane, wptr, widx, wval, N, gshift, tm);
    }
}

// Algorithm 2 for one query row: the frontier expansion from the source row srcw(0 .. ) (words, bits >= n
// ignored), visited set and result in V (ldw_out words), D / N / FL / GM the warp's shared-memory arrays
// (sized for at least ldw words). Returns the levels run (the deepest BFS level + 1). Called by a whole warp.
template <class SrcWord>
__device__ __forceinline__ int smp_expand_row(SrcWord srcw, uint64_t* __restrict__ V, int64_t ldw_out, int reflexive,
                                              const int64_t* __restrict__ wptr, const int32_t* __restrict__ widx,
                                              const uint64_t* __restrict__ wval, int64_t n, int64_t ldw,
                                              int max_levels, const Deadline& dl, const int64_t* __restrict__ wptrT,
                                              const int32_t* __restrict__ widxT, const uint64_t* __restrict__ wvalT,
                                              uint64_t* D, uint64_t* N, uint16_t* FL, uint8_t* GM, int lane) {
    const unsigned lt = (1u << lane) - 1u;  // lanes below this one
    const int64_t wpr = (n + 63) / 64;
    // words of N form at most 64 groups of 2^gshift words; a push records the groups it wrote
    int gshift = 0;
    while ((int64_t(64) << gshift) < wpr) ++gshift;
    const int ngroups = static_cast<int>((wpr + (int64_t(1) << gshift) - 1) >> gshift);
    const uint64_t all_groups = ngroups >= 64 ? ~0ull : (1ull << ngroups) - 1ull;
    const float w_out = wptrT != nullptr ? static_cast<float>(wptr[n]) / static_cast<float>(n) : 0.f;
    const float w_in = wptrT != nullptr ? static_cast<float>(wptrT[n]) / static_cast<float>(n) : 0.f;
    // D = sources; FL = their nonzero words (ballot compaction); V = 0
    int fcount = 0;
    for (int64_t w0 = 0; w0 < ldw; w0 += 32) {
        const int64_t w = w0 + lane;
        uint64_t s = 0;
        if (w < wpr) {
            s = srcw(w);
            const int64_t valid = n - w * 64;
            if (valid < 64) s &= (1ull << valid) - 1ull;
        }
        if (w < ldw) {
            D[w] = s;
            N[w] = 0;
        }
        if (w < ldw_out) V[w] = 0;
        const unsigned m = __ballot_sync(FULL, s != 0ull);
        if (s) FL[fcount + __popc(m & lt)] = static_cast<uint16_t>(w);
        fcount += __popc(m);
    }
    __syncwarp();
    int lv = 0;
    bool pull = false;
    int64_t nu = n;  // unvisited constants
    while (true) {
        if (dl.budget_ns && __shfl_sync(FULL, lane == 0 ? static_cast<int>(dl.past()) : 0, 0)) break;
        uint64_t gm = all_groups;  // groups of N that may be nonzero after this expansion
        if (pull) {
            // pull: unvisited j joins the next frontier iff some word of column j (row j of R^T) meets D;
            // each lane owns whole words of N (no atomics)
            for (int64_t w = lane; w < wpr; w += 32) {
                uint64_t nw = 0;
                {
                    uint64_t u = ~V[w];
                    const int64_t valid = n - w * 64;
                    if (valid < 64) u &= (1ull << valid) - 1ull;
                    while (u) {
                        // two unvisited constants at a time: their column ranges, then the first two
                        // entries of each, all loads in flight before the first test
                        int bs[2];
                        int64_t s0[2], s1[2];
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            bs[q] = -1;
                            if (u) {
                                bs[q] = __ffsll(static_cast<long long>(u)) - 1;
                                u &= u - 1;
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int64_t j = w * 64 + (bs[q] < 0 ? 0 : bs[q]);
                            s0[q] = bs[q] < 0 ? 0 : wptrT[j];
                            s1[q] = bs[q] < 0 ? 0 : wptrT[j + 1];
                        }
                        int xi[2][2];
                        uint64_t xv[2][2];
#pragma unroll
                        for (int q = 0; q < 2; ++q)
#pragma unroll
                            for (int r = 0; r < 2; ++r) {
                                const bool in = s0[q] + r < s1[q];
                                xi[q][r] = in ? widxT[s0[q] + r] : 0;
                                xv[q][r] = in ? wvalT[s0[q] + r] : 0ull;
                            }
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            if (bs[q] < 0) continue;
                            bool hit = (xv[q][0] & D[xi[q][0]]) != 0ull || (xv[q][1] & D[xi[q][1]]) != 0ull;
                            for (int64_t e = s0[q] + 2; !hit && e < s1[q]; ++e) hit = (wvalT[e] & D[widxT[e]]) != 0ull;
                            if (hit) nw |= 1ull << bs[q];
                        }
                    }
                    N[w] = nw;
                }
            }
        } else {
            // push: OR the nonzero words of every frontier row into N (no return values, so the
            // atomics are reductions); each lane records the word groups it wrote
            uint64_t tm = 0;
            for (int i0 = 0; i0 < fcount; i0 += 32) {
                const int i = i0 + lane;
                const int64_t w = i < fcount ? FL[i] : 0;
                uint64_t d = i < fcount ? D[w] : 0ull;  // FL[i] for i < fcount <= ldw only
                // at most two constants per word: each lane takes its own; else the bits are dealt out
                if (__reduce_max_sync(FULL, static_cast<unsigned>(__popcll(d))) <= 2u)
                    push_step<2>(d, w, lane, wptr, widx, wval, N, gshift, tm);
                else
                    push_balanced(d, w, lane, wptr, widx, wval, N, gshift, tm);
            }
            gm = static_cast<uint64_t>(__reduce_or_sync(FULL, static_cast<unsigned>(tm))) |
                 (static_cast<uint64_t>(__reduce_or_sync(FULL, static_cast<unsigned>(tm >> 32))) << 32);
        }
        __syncwarp();
        // D := 0 on the old frontier words, then D := N & ~V on the touched groups (V |= D, N := 0);
        // the words that come out nonzero become the new frontier list FL
        for (int i = lane; i < fcount; i += 32) D[FL[i]] = 0;
        __syncwarp();
        int nf = 0, fnew = 0;
        // GM[r] = index of the r-th set group of gm; candidates are the words of those groups
        for (int b = lane; b < 64; b += 32)
            if ((gm >> b) & 1ull) GM[__popcll(gm & ((1ull << b) - 1ull))] = static_cast<uint8_t>(b);
        __syncwarp();
        const int cand = __popcll(gm) << gshift;
        const int gmask = (1 << gshift) - 1;
        for (int c0 = 0; c0 < cand; c0 += 32) {
            const int c = c0 + lane;
            int w = static_cast<int>(wpr);
            if (c < cand) w = (static_cast<int>(GM[c >> gshift]) << gshift) + (c & gmask);
            uint64_t nw = 0;
            if (w < wpr) {
                nw = N[w] & ~V[w];
                N[w] = 0;
                if (nw) {
                    V[w] |= nw;
                    D[w] = nw;
                }
            }
            const unsigned m = __ballot_sync(FULL, nw != 0ull);
            if (nw) FL[fnew + __popc(m & lt)] = static_cast<uint16_t>(w);
            fnew += __popc(m);
            nf += __popcll(nw);
        }
        nf = __reduce_add_sync(FULL, nf);
        fcount = fnew;
        __syncwarp();
        nu -= nf;
        ++lv;
        if (nf == 0 || lv > max_levels) break;
        // direction of the next level: the cheaper one by the words it touches (nf > 0 here)
        pull = wptrT != nullptr &&
               static_cast<float>(nf) * w_out >
                   static_cast<float>(nu) * (PULL_OVERHEAD + fminf(w_in, static_cast<float>(n) / static_cast<float>(nf)));
    }
    if (reflexive)
        for (int64_t w = lane; w < wpr; w += 32) {
            uint64_t s = srcw(w);
            const int64_t valid = n - w * 64;
            if (valid < 64) s &= (1ull << valid) - 1ull;
            V[w] |= s;
        }
    return lv;
}

__global__ void __launch_bounds__(256, 4) smp_packed_kernel(const int64_t* __restrict__ wptr, const int32_t* __restrict__ widx,
                                                         const uint64_t* __restrict__ wval, int64_t n, int64_t ldw,
                                                         const uint64_t* __restrict__ src, int64_t ldw_src, int64_t q,
                                                         uint64_t* __restrict__ out, int64_t ldw_out, int* levels_max,
                                                         unsigned long long* qcounter, int reflexive, int max_levels,
                                                         Deadline dl, const int64_t* __restrict__ wptrT,
                                                         const int32_t* __restrict__ widxT,
                                                         const uint64_t* __restrict__ wvalT) {
    extern __shared__ uint64_t sm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint64_t* D = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(sm) + wib * smp_warp_bytes(ldw));
    uint64_t* N = D + ldw;
    uint16_t* FL = reinterpret_cast<uint16_t*>(N + ldw);
    uint8_t* GM = reinterpret_cast<uint8_t*>(FL + ldw);
    while (true) {
        unsigned long long qi = 0;
        if (lane == 0) qi = atomicAdd(qcounter, 1ull);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= static_cast<unsigned long long>(q)) break;
        const uint64_t* srow = src + static_cast<int64_t>(qi) * ldw_src;
        uint64_t* V = out + static_cast<int64_t>(qi) * ldw_out;
        const int lv = smp_expand_row([srow](int64_t w) { return srow[w]; }, V, ldw_out, reflexive, wptr, widx, wval,
                                      n, ldw, max_levels, dl, wptrT, widxT, wvalT, D, N, FL, GM, lane);
        if (lane == 0) atomicMax(levels_max, lv);
        __syncwarp();
    }
}

// ---- closures by frontier expansion of many small relations in one launch (grouped batch)
// Transpose and word index of R and of R^T for every job: blockIdx.y = job; blockIdx.z = 0 builds the
// transpose, then (separate launches, stage 1-3) the word indexes of both matrices (blockIdx.z = matrix).
__global__ void __launch_bounds__(64) frontier_transpose_kernel(const FrontierJob* __restrict__ jobs) {
    __shared__ uint64_t t[64];
    const FrontierJob& J = jobs[blockIdx.y];
    const int64_t wpr = (J.n + 63) / 64;
    for (int64_t tile = blockIdx.x; tile < wpr * wpr; tile += gridDim.x)
        bit_transpose_tile(J.P, J.PT, J.n, J.ldw, tile / wpr, tile % wpr, t);
    // padding words of the transpose's rows
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < J.n;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x)
        for (int64_t w = wpr; w < J.ldw; ++w) J.PT[r * J.ldw + w] = 0ull;
}

__global__ void __launch_bounds__(256) frontier_wcsr_count_kernel(const FrontierJob* __restrict__ jobs) {
    const FrontierJob& J = jobs[blockIdx.y];
    const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    if (blockIdx.z == 0) wcsr_count_rows(J.P, J.n, J.ldw, J.wptr, warp_id, nwarps, threadIdx.x & 31);
    else wcsr_count_rows(J.PT, J.n, J.ldw, J.wptrT, warp_id, nwarps, threadIdx.x & 31);
}

__global__ void __launch_bounds__(1024) frontier_scan_kernel(const FrontierJob* __restrict__ jobs) {
    const FrontierJob& J = jobs[blockIdx.y];
    scan_block(blockIdx.z == 0 ? J.wptr : J.wptrT, J.n);
}

__global__ void __launch_bounds__(256) frontier_wcsr_fill_kernel(const FrontierJob* __restrict__ jobs) {
    const FrontierJob& J = jobs[blockIdx.y];
    const int64_t warp_id = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    if (blockIdx.z == 0) wcsr_fill_rows(J.P, J.n, J.ldw, J.wptr, J.widx, J.wval, warp_id, nwarps, threadIdx.x & 31);
    else wcsr_fill_rows(J.PT, J.n, J.ldw, J.wptrT, J.widxT, J.wvalT, warp_id, nwarps, threadIdx.x & 31);
}

// Every row of every job as one query: the rows of all jobs are numbered job by job (job j owns rows
// jobs[j].first .. jobs[j].first + n - 1), warps take them from *counter; the source of row i is constant i.
__global__ void __launch_bounds__(256, 4) frontier_group_kernel(const FrontierJob* __restrict__ jobs, int njobs,
                                                                int64_t total, int64_t ldw_max,
                                                                unsigned long long* counter) {
    extern __shared__ uint64_t sm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint64_t* D = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(sm) + wib * smp_warp_bytes(ldw_max));
    uint64_t* N = D + ldw_max;
    uint16_t* FL = reinterpret_cast<uint16_t*>(N + ldw_max);
    uint8_t* GM = reinterpret_cast<uint8_t*>(FL + ldw_max);
    const Deadline none{0, nullptr, nullptr};
    while (true) {
        unsigned long long qi = 0;
        if (lane == 0) qi = atomicAdd(counter, 1ull);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= static_cast<unsigned long long>(total)) break;
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {  // the last job whose first row is <= qi
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].first <= static_cast<int64_t>(qi)) lo = mid; else hi = mid - 1;
        }
        const FrontierJob& J = jobs[lo];
        const int64_t i = static_cast<int64_t>(qi) - J.first;
        const int64_t wi = i >> 6;
        const uint64_t bi = 1ull << (i & 63);
        const int lv = smp_expand_row([wi, bi](int64_t w) { return w == wi ? bi : 0ull; }, J.out + i * J.ldw, J.ldw, 0,
                                      J.wptr, J.widx, J.wval, J.n, J.ldw, static_cast<int>(J.n + 1), none, J.wptrT,
                                      J.widxT, J.wvalT, D, N, FL, GM, lane);
        if (lane == 0) atomicMax(J.levels, lv);
        __syncwarp();
    }
}

// ---- incremental closure: one new fact r(u, v) on a transitive R+ (packed rows)
// (R + E_uv)+ = R+ + X Y^T with X = {i : i = u or R+_iu} (the constants that
// reach u) and Y = R+_v + e_v (what v reaches, and v): every row in X gains Y.
// A warp owns each row it updates, so membership (bit u of its own row) is
// read before that row changes; row v itself only gains bit v, which every
// reader adds anyway. When R+_uv already holds, every member row already
// contains Y (transitivity) and no word is written.
__global__ void insert_fact_kernel(uint64_t* __restrict__ P, int64_t n, int64_t ldw, int64_t u, int64_t v) {
    const int lane = threadIdx.x & 31;
    const int64_t wu = u >> 6, wv = v >> 6;
    const uint64_t bu = 1ull << (u & 63), bv = 1ull << (v & 63);
    const int64_t wpr = (n + 63) >> 6;
    const uint64_t* Y = P + v * ldw;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        uint64_t* row = P + i * ldw;
        const bool member = (i == u) || (row[wu] & bu) != 0ull;  // uniform across the warp
        if (!member) continue;
        __syncwarp();
        for (int64_t w = lane; w < wpr; w += 32) {
            uint64_t y = Y[w];
            if (w == wv) y |= bv;
            const uint64_t r = row[w];
            if ((r | y) != r) row[w] = r | y;
        }
    }
}

// ---- one squaring step on packed rows through the word index of R:
// C_i = R_i | OR_{k in R_i} R_k, where row k contributes only its nonzero
// words (push_balanced), so the cost follows the index, not n / 64 words per k.
// Warp per row; the row is assembled in shared memory (ldw words per warp).
__global__ void __launch_bounds__(256) square_rows_kernel(const int64_t* __restrict__ wptr,
                                                          const int32_t* __restrict__ widx,
                                                          const uint64_t* __restrict__ wval,
                                                          const uint64_t* __restrict__ P, int64_t n, int64_t ldw,
                                                          uint64_t* __restrict__ C, int* __restrict__ changed) {
    extern __shared__ uint64_t sq_sm[];
    const int lane = threadIdx.x & 31;
    uint64_t* S = sq_sm + static_cast<int64_t>(threadIdx.x >> 5) * ldw;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        for (int64_t w = lane; w < ldw; w += 32) S[w] = P[i * ldw + w];
        __syncwarp();
        uint64_t tm = 0;  // word groups are not needed here
        const int64_t e0 = wptr[i], e1 = wptr[i + 1];
        for (int64_t b0 = e0; b0 < e1; b0 += 32) {
            const int64_t e = b0 + lane;
            const int64_t ee = e < e1 ? e : 0;
            const uint64_t d = e < e1 ? wval[ee] : 0ull;
            const int64_t w = e < e1 ? widx[ee] : 0;
            push_balanced(d, w, lane, wptr, widx, wval, S, 30, tm);
        }
        __syncwarp();
        bool grew = false;
        for (int64_t w = lane; w < ldw; w += 32) {
            const uint64_t c = S[w];
            grew |= c != P[i * ldw + w];
            C[i * ldw + w] = c;
        }
        if (changed != nullptr && __any_sync(FULL, grew) && lane == 0) atomicOr(changed, 1);
        __syncwarp();
    }
}

// ---- the work of the next squaring step through the word index: for every
// set bit k of every row, the nonzero words of row k (what square_rows_kernel
// ORs into that row). cost[0] += the total, cost[1] = max over rows (one warp
// assembles a row, so the largest row bounds the step from below). Warp per
// row, two 64-bit atomics per warp. Bits at or beyond n are zero in every
// row, so k < n.
__global__ void __launch_bounds__(256) square_cost_kernel(const int64_t* __restrict__ wptr,
                                                          const int32_t* __restrict__ widx,
                                                          const uint64_t* __restrict__ wval, int64_t n,
                                                          unsigned long long* __restrict__ cost) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    unsigned long long total = 0, top = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        unsigned long long c = 0;
        const int64_t e1 = wptr[i + 1];
        for (int64_t e = wptr[i] + lane; e < e1; e += 32) {
            uint64_t d = wval[e];
            const int64_t base = static_cast<int64_t>(widx[e]) << 6;
            while (d) {
                const int64_t k = base + (__ffsll(static_cast<long long>(d)) - 1);
                d &= d - 1ull;
                c += static_cast<unsigned long long>(wptr[k + 1] - wptr[k]);
            }
        }
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
        total += c;
        top = c > top ? c : top;
    }
    if (lane == 0 && total != 0ull) {
        atomicAdd(cost, total);
        atomicMax(cost + 1, top);
    }
}

// ---- the next squaring step's nonzero words without forming it: per row (one warp), the union of the row's own
// word indices and those of every row k it names (R + R R), in a shared-memory bitmap of ldw bits.
// out[0] += the total nonzero words of R + R R, out[1] += the word ORs the squaring would issue.
__global__ void __launch_bounds__(256) square_growth_kernel(const int64_t* __restrict__ wptr,
                                                            const int32_t* __restrict__ widx,
                                                            const uint64_t* __restrict__ wval, int64_t n, int64_t ldw,
                                                            unsigned long long* __restrict__ out,
                                                            unsigned long long* __restrict__ bits_out) {
    extern __shared__ uint32_t growth_bm[];
    const int lane = threadIdx.x & 31;
    const int bw = static_cast<int>((ldw + 31) / 32);  // bitmap words per warp
    uint32_t* bm = growth_bm + (threadIdx.x >> 5) * bw;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    unsigned long long words = 0, ors = 0, ones = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        for (int j = lane; j < bw; j += 32) bm[j] = 0u;
        __syncwarp();
        const int64_t e1 = wptr[i + 1];
        for (int64_t e = wptr[i] + lane; e < e1; e += 32) {
            const int x = widx[e];
            atomicOr(&bm[x >> 5], 1u << (x & 31));
            uint64_t d = wval[e];
            ones += static_cast<unsigned long long>(__popcll(d));
            const int64_t base = static_cast<int64_t>(x) << 6;
            while (d) {
                const int64_t k = base + (__ffsll(static_cast<long long>(d)) - 1);
                d &= d - 1ull;
                const int64_t f1 = wptr[k + 1];
                for (int64_t f = wptr[k]; f < f1; ++f) {
                    const int y = widx[f];
                    atomicOr(&bm[y >> 5], 1u << (y & 31));
                    ++ors;
                }
            }
        }
        __syncwarp();
        for (int j = lane; j < bw; j += 32) words += static_cast<unsigned long long>(__popc(bm[j]));
        __syncwarp();  // the bitmap is cleared for the next row
    }
    for (int off = 16; off > 0; off >>= 1) {
        words += __shfl_xor_sync(FULL, words, off);
        ors += __shfl_xor_sync(FULL, ors, off);
        ones += __shfl_xor_sync(FULL, ones, off);
    }
    if (lane == 0 && (words | ors) != 0ull) {
        atomicAdd(out, words);
        atomicAdd(out + 1, ors);
    }
    if (lane == 0 && bits_out != nullptr && ones != 0ull) atomicAdd(bits_out, ones);
}

// Bit rows of R^T from the word index of R (out cleared beforehand): warp per row i of R, a lane per nonzero word;
// each set bit (i, j) ORs bit i into word i / 64 of row j. Rows i of one 64-row group hit the same words of R^T,
// on different bits.
__global__ void __launch_bounds__(256) scatter_transpose_kernel(const int64_t* __restrict__ wptr,
                                                                const int32_t* __restrict__ widx,
                                                                const uint64_t* __restrict__ wval, int64_t n,
                                                                int64_t ldw, unsigned long long* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const unsigned long long bit = 1ull << (i & 63);
        const int64_t wi = i >> 6;
        const int64_t e1 = wptr[i + 1];
        for (int64_t e = wptr[i] + lane; e < e1; e += 32) {
            uint64_t d = wval[e];
            const int64_t base = static_cast<int64_t>(widx[e]) << 6;
            while (d) {
                const int64_t j = base + (__ffsll(static_cast<long long>(d)) - 1);
                d &= d - 1ull;
                if (j < n) atomicOr(out + j * ldw + wi, bit);  // a caller's bits beyond column n are not columns
            }
        }
    }
}

// ---- frontier expansion of 64 sources at once (closures whose rows reach most constants)
// Algorithm 2 for the 64 query rows e_s0 .. e_s0+63 together, bit-sliced: word w of V, D and Dn holds, in bit j,
// whether constant w is visited by / in the frontier of / in the next frontier of source s0 + j. A level pulls:
// Dn[w] = (OR of D[v] over the in-neighbours v of w, i.e. the set bits of row w of R^T) AND NOT V[w], skipping every
// w already reached from all sources whose frontier is not empty (A, the OR of all D words). One traversal of R^T
// serves 64 sources, and no word is written by two threads. V, D and Dn live in the CTA's slice of `scratch` (3 n words); the CTA takes batches from
// a global counter and, after the last level, writes its 64 output rows through 64 x 64 bit transposes (ballots).
// Threads per CTA and CTAs per SM of the sliced kernel: each CTA holds 3 n words of state, so the number of CTAs
// in flight sets the working set that has to stay in L2.
constexpr int kSlicedThreads = 1024;
constexpr int kSlicedPerSm = 1;

__global__ void __launch_bounds__(kSlicedThreads) smp_sliced_kernel(const int64_t* __restrict__ wptrT,
                                                         const int32_t* __restrict__ widxT,
                                                         const uint64_t* __restrict__ wvalT, int64_t n, int64_t nbatch,
                                                         uint64_t* __restrict__ scratch, uint64_t* __restrict__ out,
                                                         int64_t ldw_out, unsigned long long* bcounter,
                                                         int* levels_max, int max_levels, Deadline dl) {
    __shared__ unsigned long long s_batch;
    __shared__ unsigned long long s_active;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    uint64_t* const V = scratch + static_cast<int64_t>(blockIdx.x) * 3 * n;
    while (true) {
        if (tid == 0) s_batch = atomicAdd(bcounter, 1ull);
        __syncthreads();
        const int64_t b = static_cast<int64_t>(s_batch);
        __syncthreads();
        if (b >= nbatch) break;
        const int64_t s0 = b * 64;
        const int cnt = static_cast<int>(n - s0 < 64 ? n - s0 : 64);
        const uint64_t full = cnt == 64 ? ~0ull : (1ull << cnt) - 1ull;
        uint64_t* D = V + n;
        uint64_t* Dn = V + 2 * n;
        for (int64_t w = tid; w < n; w += blockDim.x) {
            V[w] = 0ull;
            D[w] = (w >= s0 && w < s0 + cnt) ? (1ull << (w - s0)) : 0ull;
        }
        if (tid == 0) s_active = 0ull;
        uint64_t act = full;  // sources whose frontier is not empty
        __syncthreads();
        int lv = 0;
        while (true) {
            int stop = 0;
            if (tid == 0 && dl.budget_ns) stop = dl.past() ? 1 : 0;
            if (__syncthreads_or(stop)) break;
            uint64_t grown = 0ull;
            // two constants per thread at a time, w and w + blockDim.x, whose in-lists are walked in lockstep so
            // that their chains of dependent loads (row range, in-word, frontier words) overlap
            const int64_t stride = blockDim.x;
            for (int64_t wa = tid; wa < n; wa += 2 * stride) {
                const int64_t wb = wa + stride;
                const bool hb = wb < n;
                const uint64_t va = V[wa];
                const uint64_t vb = hb ? V[wb] : ~0ull;
                const uint64_t needa = act & ~va;  // active sources that have not reached the constant
                const uint64_t needb = act & ~vb;
                uint64_t acca = 0ull, accb = 0ull;
                int64_t ea = 0, ea1 = 0, eb = 0, eb1 = 0;
                if (needa) {
                    ea = wptrT[wa];
                    ea1 = wptrT[wa + 1];
                }
                if (needb) {
                    eb = wptrT[wb];
                    eb1 = wptrT[wb + 1];
                }
                while (true) {
                    const bool ta = ea < ea1 && (acca & needa) != needa;
                    const bool tb = eb < eb1 && (accb & needb) != needb;
                    if (!ta && !tb) break;
                    uint64_t ba = ta ? wvalT[ea] : 0ull;
                    uint64_t bb = tb ? wvalT[eb] : 0ull;
                    const int64_t basea = ta ? static_cast<int64_t>(widxT[ea]) << 6 : 0;
                    const int64_t baseb = tb ? static_cast<int64_t>(widxT[eb]) << 6 : 0;
                    while (ba | bb) {
                        if (ba) {
                            const int64_t v = basea + (__ffsll(static_cast<long long>(ba)) - 1);
                            ba &= ba - 1ull;
                            acca |= D[v];
                        }
                        if (bb) {
                            const int64_t v = baseb + (__ffsll(static_cast<long long>(bb)) - 1);
                            bb &= bb - 1ull;
                            accb |= D[v];
                        }
                    }
                    ea += ta ? 1 : 0;
                    eb += tb ? 1 : 0;
                }
                const uint64_t nna = acca & needa;
                Dn[wa] = nna;
                if (nna) V[wa] = va | nna;
                grown |= nna;
                if (hb) {
                    const uint64_t nnb = accb & needb;
                    Dn[wb] = nnb;
                    if (nnb) V[wb] = vb | nnb;
                    grown |= nnb;
                }
            }
            const unsigned glo = __reduce_or_sync(FULL, static_cast<unsigned>(grown));
            const unsigned ghi = __reduce_or_sync(FULL, static_cast<unsigned>(grown >> 32));
            if (lane == 0 && (glo | ghi)) atomicOr(&s_active, static_cast<unsigned long long>(glo) |
                                                                (static_cast<unsigned long long>(ghi) << 32));
            __syncthreads();
            act = s_active;
            __syncthreads();
            if (tid == 0) s_active = 0ull;
            ++lv;
            uint64_t* t = D;
            D = Dn;
            Dn = t;
            if (act == 0ull || lv > max_levels) break;
        }
        if (tid == 0) atomicMax(levels_max, lv);
        // rows s0 .. s0 + cnt - 1 of the output: word wd of row s0 + j = bit j of V[64 wd .. 64 wd + 63]
        const int64_t wpr = (n + 63) >> 6;
        for (int64_t wd = tid >> 5; wd < wpr; wd += blockDim.x >> 5) {
            const int64_t w0 = wd * 64 + lane, w1 = w0 + 32;
            const uint64_t v0 = w0 < n ? V[w0] : 0ull;
            const uint64_t v1 = w1 < n ? V[w1] : 0ull;
            uint64_t mine0 = 0ull, mine1 = 0ull;
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const unsigned lo = __ballot_sync(FULL, ((v0 >> j) & 1ull) != 0ull);
                const unsigned hi = __ballot_sync(FULL, ((v1 >> j) & 1ull) != 0ull);
                if (j == lane) mine0 = static_cast<uint64_t>(lo) | (static_cast<uint64_t>(hi) << 32);
            }
#pragma unroll 8
            for (int j = 32; j < 64; ++j) {
                const unsigned lo = __ballot_sync(FULL, ((v0 >> j) & 1ull) != 0ull);
                const unsigned hi = __ballot_sync(FULL, ((v1 >> j) & 1ull) != 0ull);
                if (j - 32 == lane) mine1 = static_cast<uint64_t>(lo) | (static_cast<uint64_t>(hi) << 32);
            }
            if (lane < cnt) out[(s0 + lane) * ldw_out + wd] = mine0;
            if (lane + 32 < cnt) out[(s0 + lane + 32) * ldw_out + wd] = mine1;
        }
        __syncthreads();
    }
}

// ---- Algorithm 2 for 64 query rows at once (bit-sliced), the frontier in distributed shared memory
// A cluster of C CTAs (1..8) expands one batch of 64 rows, the query rows s0 .. s0 + 63 of src (query batches,
// which do not fill the GPU with one CTA per 64 rows as a closure's 64-source batches do, and closures with skewed
// columns, as the identity rows; the global-memory kernel above measured faster on the rest). CTA r owns the
// constants w in
// [r chunk, (r + 1) chunk) (chunk a power of two) and keeps in its shared memory their words of D (bit j: w is in
// the frontier of row j), Dn (the next frontier) and V (bit j: w reached from row j). A level pulls as the kernel
// above does, Dn[w] = (OR of D[v] over the in-neighbours v of w) AND NOT V[w] for every w that some active row has
// not reached, but D[v] comes from the shared memory of v's owner instead of L2, and a warp takes 32 consecutive
// constants at a time (from a per-level counter) and walks their in-lists together, 64 entries per step (coalesced
// index loads, no lane waiting for the longest list). One cluster barrier per level publishes Dn and each CTA's OR
// of its new words; every CTA then reads all of them, so the active rows, the level count and the stop flag (CTA
// 0's deadline check) are the same in every CTA, and all CTAs of a cluster run the same number of barriers.
constexpr int kClusterThreads = 1024;
constexpr int kClusterWarps = kClusterThreads / 32;
constexpr int kClusterMaxLog2Chunk = 13;  // 8,192 constants per CTA: D, Dn and V take 192 KiB
constexpr int kClusterMinLog2Chunk = 10;  // clusters are widened down to 1,024 constants per CTA
constexpr int kClusterMaxCtas = 8;        // portable cluster size

struct ClusterArgs {
    const int64_t* wptrT;  // word index of R^T: the in-neighbours of a constant
    const int32_t* widxT;
    const uint64_t* wvalT;
    const uint64_t* src;  // query rows (ldw_src words each)
    int64_t ldw_src;
    int64_t n;
    int64_t rows;  // query rows
    uint64_t* out;
    int64_t ldw_out;
    int* levels_max;
    int max_levels;
    int reflexive;
    int log2_chunk;
    Deadline dl;
};

__device__ __forceinline__ uint64_t or_reduce_warp(uint64_t x) {
    const unsigned lo = __reduce_or_sync(FULL, static_cast<unsigned>(x));
    const unsigned hi = __reduce_or_sync(FULL, static_cast<unsigned>(x >> 32));
    return static_cast<uint64_t>(lo) | (static_cast<uint64_t>(hi) << 32);
}

// The entries of a tile's lists, 64 per step: lane l owns cnt entries from index es on (cnt = 0: none). fn(x, e)
// gets, for this lane's two entries of the step, the owning lane (-1: past the end) and the entry index; it runs in
// every lane (shuffles inside it see the whole warp).
template <typename Fn>
__device__ __forceinline__ void walk_lists(int es, int cnt, int lane, Fn&& fn) {
    int incl = cnt;  // entries of lanes 0 .. lane
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int ebase = es - (incl - cnt);  // entry k of the warp is entry ebase(owner) + k of the index
    for (int k0 = 0; k0 < total; k0 += 64) {
        int x[2], e[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = k0 + 32 * h + lane;
            int o = 0;  // owner of entry k: the first lane whose inclusive count exceeds k
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(FULL, incl, o + step - 1) <= k) o += step;
            e[h] = __shfl_sync(FULL, ebase, o < 32 ? o : 31) + k;
            x[h] = k < total ? o : -1;
        }
        fn(x, e);
    }
}

__global__ void __launch_bounds__(kClusterThreads, 1) smp_cluster_kernel(const ClusterArgs a) {
    extern __shared__ uint64_t cl_sm[];
    __shared__ uint64_t s_grown[2];                // by level parity: the OR of this CTA's new frontier words
    __shared__ int s_stop[2];                      // by level parity, CTA 0 only: the time budget is used up
    __shared__ uint64_t s_warp[kClusterWarps];
    __shared__ uint64_t s_acc[kClusterWarps][32];  // per warp: the OR of D over each tile constant's entries
    __shared__ int s_tile[2];                      // by level parity: the next tile of 32 constants
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t rank = cluster_ctarank();
    const uint32_t ctas = cluster_nctarank();
    const int lg = a.log2_chunk;
    const int chunk = 1 << lg;
    const int n = static_cast<int>(a.n);
    const int64_t s0 = static_cast<int64_t>(cluster_id_x()) * 64;
    const int cnt = static_cast<int>(a.rows - s0 < 64 ? a.rows - s0 : 64);
    const int base = static_cast<int>(rank) * chunk;
    const int own = n - base <= 0 ? 0 : (n - base < chunk ? n - base : chunk);
    const int own_words = (own + 63) >> 6;
    const int64_t wpr = (a.n + 63) >> 6;
    uint64_t* D = cl_sm;
    uint64_t* Dn = cl_sm + chunk;
    uint64_t* V = cl_sm + 2 * chunk;
    if (tid < 2) s_tile[tid] = 0;

    // level 0 frontier of this CTA's constants: word wd of the batch's 64 query rows, transposed, D[64 wd + k]
    // bit j = bit k of word wd of row s0 + j
    for (int wl = warp; wl < own_words; wl += kClusterWarps) {
        const int64_t wd = (base >> 6) + wl;
        const int64_t valid = a.n - wd * 64;
        const uint64_t m = valid < 64 ? (1ull << valid) - 1ull : ~0ull;
        const uint64_t a0 = lane < cnt ? a.src[(s0 + lane) * a.ldw_src + wd] & m : 0ull;
        const uint64_t a1 = lane + 32 < cnt ? a.src[(s0 + lane + 32) * a.ldw_src + wd] & m : 0ull;
        uint64_t c0, c1;
        warp_transpose64(a0, a1, lane, c0, c1);
        const int i0 = wl * 64 + lane;
        if (i0 < own) {
            D[i0] = c0;
            V[i0] = 0ull;
        }
        if (i0 + 32 < own) {
            D[i0 + 32] = c1;
            V[i0 + 32] = 0ull;
        }
    }
    uint64_t act = cnt == 64 ? ~0ull : (1ull << cnt) - 1ull;  // rows whose frontier may be nonempty
    cluster_sync();  // every CTA's level 0 frontier is in place

    int lv = 0;
    while (true) {
        const int p = lv & 1;
        if (tid == 0) s_tile[p ^ 1] = 0;  // the next level's tile counter (its last use ended before the last barrier)
        if (rank == 0 && tid == 0) s_stop[p] = (a.dl.budget_ns && a.dl.past()) ? 1 : 0;
        const uint32_t d_s = smem_u32(D);
        uint64_t grown = 0ull;
        uint64_t* acc_s = s_acc[warp];
        while (true) {
            int t = 0;
            if (lane == 0) t = atomicAdd(&s_tile[p], 1);
            t = __shfl_sync(FULL, t, 0);
            if (t * 32 >= own) break;
            const int i = t * 32 + lane;
            const bool in = i < own;
            const uint64_t vw = in ? V[i] : ~0ull;
            const uint64_t need = act & ~vw;  // active rows that have not reached w = base + i
            int es = 0, c = 0;
            if (need) {
                es = static_cast<int>(a.wptrT[base + i]);
                c = static_cast<int>(a.wptrT[base + i + 1]) - es;
            }
            acc_s[lane] = 0ull;
            __syncwarp();
            walk_lists(es, c, lane, [&](const int (&x)[2], const int (&e)[2]) {
                uint64_t bits[2];
                int vb[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    bits[h] = x[h] >= 0 ? a.wvalT[e[h]] : 0ull;
                    vb[h] = x[h] >= 0 ? a.widxT[e[h]] << 6 : 0;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint64_t r = 0ull;
                    uint64_t b = bits[h];
                    while (b) {
                        const int v = vb[h] + (__ffsll(static_cast<long long>(b)) - 1);
                        b &= b - 1ull;
                        const uint32_t owner = static_cast<uint32_t>(v >> lg);
                        const uint32_t off = static_cast<uint32_t>(v & (chunk - 1));
                        r |= owner == rank ? D[off] : ld_dsmem_u64(mapa_shared(d_s + off * 8u, owner));
                    }
                    if (r) atomicOr(reinterpret_cast<unsigned long long*>(&acc_s[x[h]]), r);
                }
            });
            __syncwarp();
            const uint64_t nn = acc_s[lane] & need;
            if (in) {
                Dn[i] = nn;
                if (nn) V[i] = vw | nn;
            }
            grown |= nn;
            __syncwarp();  // acc_s is cleared for the next tile
        }
        grown = or_reduce_warp(grown);
        if (lane == 0) s_warp[warp] = grown;
        __syncthreads();
        if (warp == 0) {
            const uint64_t g = or_reduce_warp(s_warp[lane]);
            if (lane == 0) s_grown[p] = g;
        }
        cluster_sync();  // Dn and s_grown[p] of every CTA are visible cluster-wide
        act = 0ull;
        for (uint32_t c = 0; c < ctas; ++c) act |= ld_dsmem_u64(mapa_shared(smem_u32(&s_grown[p]), c));
        const int stop = ld_dsmem_s32(mapa_shared(smem_u32(&s_stop[p]), 0));
        ++lv;
        uint64_t* t = D;
        D = Dn;
        Dn = t;
        if (act == 0ull || lv > a.max_levels || stop) break;
    }
    if (rank == 0 && tid == 0) atomicMax(a.levels_max, lv);

    // output words of this CTA's constants: word wd of row s0 + j = bit j of V[64 wd .. 64 wd + 63]
    for (int wl = warp; wl < own_words; wl += kClusterWarps) {
        const int64_t wd = (base >> 6) + wl;
        const int i0 = wl * 64 + lane;
        const uint64_t v0 = i0 < own ? V[i0] : 0ull;
        const uint64_t v1 = i0 + 32 < own ? V[i0 + 32] : 0ull;
        uint64_t m0, m1;
        warp_transpose64(v0, v1, lane, m0, m1);
        if (a.reflexive) {
            const int64_t valid = a.n - wd * 64;
            const uint64_t m = valid < 64 ? (1ull << valid) - 1ull : ~0ull;
            if (lane < cnt) m0 |= a.src[(s0 + lane) * a.ldw_src + wd] & m;
            if (lane + 32 < cnt) m1 |= a.src[(s0 + lane + 32) * a.ldw_src + wd] & m;
        }
        if (lane < cnt) a.out[(s0 + lane) * a.ldw_out + wd] = m0;
        if (lane + 32 < cnt) a.out[(s0 + lane + 32) * a.ldw_out + wd] = m1;
    }
    const int64_t pad = a.ldw_out - wpr;  // words of an output row beyond n
    if (rank == ctas - 1 && pad > 0)
        for (int64_t x = tid; x < cnt * pad; x += kClusterThreads) a.out[(s0 + x / pad) * a.ldw_out + wpr + x % pad] = 0ull;
    cluster_sync();  // no CTA leaves while a peer may still read its shared memory
}

inline int warps_grid(int64_t rows, int sms) {
    int64_t blocks = (rows + 7) / 8;  // 8 warps of 256 threads
    const int64_t cap = static_cast<int64_t>(sms) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return static_cast<int>(blocks);
}

}  // namespace

cudaError_t launch_product_packed(const uint64_t* A, const uint64_t* B, uint64_t* dst, int64_t n, int64_t ldw,
                                  int or_a, int* changed, int sms, cudaStream_t s, Deadline dl,
                                  unsigned long long* pstat, bool tables) {
    if (n <= 0) return cudaSuccess;
    if (!tables) {
        const int grid = warps_grid(n, sms);
        if (ldw <= 128)
            product_gather_kernel<2><<<grid, 256, 0, s>>>(A, B, dst, n, ldw, or_a, changed, dl, pstat);
        else if (ldw <= 256)
            product_gather_kernel<4><<<grid, 256, 0, s>>>(A, B, dst, n, ldw, or_a, changed, dl, pstat);
        else
            product_gather_kernel<8><<<grid, 256, 0, s>>>(A, B, dst, n, ldw, or_a, changed, dl, pstat);
        return cudaGetLastError();
    }
    const int64_t grid = ((n + kM4Rows - 1) / kM4Rows) * ((ldw + kM4Cols - 1) / kM4Cols);
    cudaError_t e = cudaFuncSetAttribute(product_m4rm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kM4Smem));
    if (e != cudaSuccess) return e;
    product_m4rm_kernel<<<static_cast<unsigned>(grid), kM4Threads, kM4Smem, s>>>(A, B, dst, n, ldw, or_a, changed,
                                                                                   dl, pstat);
    return cudaGetLastError();
}

cudaError_t launch_insert_fact(uint64_t* P, int64_t n, int64_t ldw, int64_t u, int64_t v, int sms, cudaStream_t s) {
    insert_fact_kernel<<<warps_grid(n, sms), 256, 0, s>>>(P, n, ldw, u, v);
    return cudaGetLastError();
}

cudaError_t launch_wcsr_build(const uint64_t* P, int64_t n, int64_t ldw, int64_t* wptr, int32_t* widx, uint64_t* wval,
                              cudaStream_t s, int64_t* scan_scratch) {
    const int grid = warps_grid(n, 152);
    wcsr_count_kernel<<<grid, 256, 0, s>>>(P, n, ldw, wptr);
    const int64_t chunks = (n + kScanChunk - 1) / kScanChunk;
    if (scan_scratch != nullptr && chunks > 1 && chunks <= kScanMaxChunks) {
        scan_chunks_kernel<<<static_cast<unsigned>(chunks), 1024, 0, s>>>(wptr, n, scan_scratch, static_cast<int>(chunks));
        scan_add_kernel<<<static_cast<unsigned>(chunks), 1024, 0, s>>>(wptr, n, scan_scratch, static_cast<int>(chunks));
    } else {
        scan_kernel<<<1, 1024, 0, s>>>(wptr, n);
    }
    wcsr_fill_kernel<<<grid, 256, 0, s>>>(P, n, ldw, wptr, widx, wval);
    return cudaGetLastError();
}

int smp_packed_max_words() { return 7168; }

cudaError_t launch_square_rows(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, const uint64_t* P,
                               int64_t n, int64_t ldw, uint64_t* C, int sms, cudaStream_t s, int* changed) {
    int warps = 8;
    while (warps > 1 && warps * ldw * 8 > 32 * 1024) warps >>= 1;
    const size_t smem = static_cast<size_t>(warps) * static_cast<size_t>(ldw) * 8;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(square_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    int64_t blocks = (n + warps - 1) / warps;
    const int64_t cap = static_cast<int64_t>(sms) * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    square_rows_kernel<<<static_cast<int>(blocks), warps * 32, smem, s>>>(wptr, widx, wval, P, n, ldw, C, changed);
    return cudaGetLastError();
}

int64_t smp_sliced_grid(int64_t n, int sms) {
    const int64_t nbatch = (n + 63) / 64;
    const int64_t cap = static_cast<int64_t>(sms) * kSlicedPerSm;
    return nbatch < cap ? nbatch : cap;
}

cudaError_t launch_smp_sliced(const int64_t* wptrT, const int32_t* widxT, const uint64_t* wvalT, int64_t n,
                              uint64_t* scratch, uint64_t* out, int64_t ldw_out, unsigned long long* bcounter,
                              int* levels, int max_levels, int sms, cudaStream_t s, Deadline dl) {
    const int64_t grid = smp_sliced_grid(n, sms);
    smp_sliced_kernel<<<static_cast<int>(grid), kSlicedThreads, 0, s>>>(wptrT, widxT, wvalT, n, (n + 63) / 64, scratch, out,
                                                             ldw_out, bcounter, levels, max_levels, dl);
    return cudaGetLastError();
}

// Cluster shape of smp_cluster_kernel: the fewest CTAs whose shared memory holds the state of n constants (at most
// 8,192 per CTA), widened (down to 1,024 constants per CTA) while the batches alone leave SMs idle. False when n
// needs more than 8 CTAs.
bool smp_cluster_shape(int64_t n, int64_t batches, int sms, int* ctas, int* log2_chunk) {
    int lg = 6;
    while ((int64_t(1) << lg) < n && lg < kClusterMaxLog2Chunk) ++lg;
    int64_t c = (n + (int64_t(1) << lg) - 1) >> lg;
    if (n < 1 || c > kClusterMaxCtas) return false;
    while (lg > kClusterMinLog2Chunk && batches * c < sms) {
        const int64_t c2 = (n + (int64_t(1) << (lg - 1)) - 1) >> (lg - 1);
        if (c2 > kClusterMaxCtas) break;
        --lg;
        c = c2;
    }
    *ctas = static_cast<int>(c);
    *log2_chunk = lg;
    return true;
}

namespace {
cudaLaunchConfig_t cluster_config(int64_t clusters, int ctas, int lg, cudaStream_t s, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(clusters * ctas), 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = 3 * (size_t(8) << lg);
    cfg.stream = s;
    at->id = cudaLaunchAttributeClusterDimension;
    at->val.clusterDim.x = static_cast<unsigned>(ctas);
    at->val.clusterDim.y = 1;
    at->val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}
}  // namespace

static bool smp_cluster_fits_query(int ctas, int lg);

bool smp_cluster_fits(int64_t n, int64_t rows, int sms) {
    int ctas = 0, lg = 0;
    if (rows < 1 || !smp_cluster_shape(n, (rows + 63) / 64, sms, &ctas, &lg)) return false;
    // the answer depends on the device and the launch shape only: kept per (device, ctas, log2 chunk), since the
    // occupancy query costs far more than a launch (0: not asked yet, 1: fits, 2: does not)
    static signed char known[16][9][32] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    const bool keyed = dev >= 0 && dev < 16 && ctas >= 1 && ctas <= 8 && lg >= 0 && lg < 32;
    if (keyed && known[dev][ctas][lg] != 0) return known[dev][ctas][lg] == 1;
    const bool fits = smp_cluster_fits_query(ctas, lg);
    if (keyed) known[dev][ctas][lg] = fits ? 1 : 2;
    return fits;
}

static bool smp_cluster_fits_query(int ctas, int lg) {
    cudaLaunchAttribute at;
    const cudaLaunchConfig_t cfg = cluster_config(1, ctas, lg, nullptr, &at);
    if (cudaFuncSetAttribute(smp_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(cfg.dynamicSmemBytes)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, smp_cluster_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters > 0;
}

cudaError_t launch_smp_cluster(const int64_t* wptrT, const int32_t* widxT, const uint64_t* wvalT, int64_t n,
                               const uint64_t* src, int64_t ldw_src, int64_t rows, uint64_t* out, int64_t ldw_out,
                               int reflexive, int* levels, int max_levels, int sms, cudaStream_t s, Deadline dl) {
    const int64_t batches = (rows + 63) / 64;
    int ctas = 0, lg = 0;
    if (rows < 1 || !smp_cluster_shape(n, batches, sms, &ctas, &lg)) return cudaErrorInvalidValue;
    cudaLaunchAttribute at;
    const cudaLaunchConfig_t cfg = cluster_config(batches, ctas, lg, s, &at);
    cudaError_t e = cudaFuncSetAttribute(smp_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(cfg.dynamicSmemBytes));
    if (e != cudaSuccess) return e;
    const ClusterArgs a{wptrT, widxT, wvalT, src, ldw_src, n, rows, out, ldw_out, levels, max_levels, reflexive, lg,
                        dl};
    return cudaLaunchKernelEx(&cfg, smp_cluster_kernel, a);
}

cudaError_t launch_square_growth(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n,
                                 int64_t ldw, unsigned long long* out, int sms, cudaStream_t s,
                                 unsigned long long* bits_out) {
    const size_t smem = static_cast<size_t>(8) * ((ldw + 31) / 32) * 4;
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    square_growth_kernel<<<warps_grid(n, sms), 256, smem, s>>>(wptr, widx, wval, n, ldw, out, bits_out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_transpose(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n,
                                     int64_t ldw, uint64_t* out, int sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out, 0, static_cast<size_t>(n) * static_cast<size_t>(ldw) * 8, s);
    if (e != cudaSuccess) return e;
    scatter_transpose_kernel<<<warps_grid(n, sms), 256, 0, s>>>(wptr, widx, wval, n, ldw,
                                                                reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError();
}

cudaError_t launch_square_cost(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n,
                               unsigned long long* cost, int sms, cudaStream_t s) {
    square_cost_kernel<<<warps_grid(n, sms), 256, 0, s>>>(wptr, widx, wval, n, cost);
    return cudaGetLastError();
}

cudaError_t launch_smp_packed(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n, int64_t ldw,
                              const uint64_t* src, int64_t ldw_src, int64_t q, uint64_t* out, int64_t ldw_out,
                              int* levels, int* qcounter, int reflexive, int sms, cudaStream_t s, Deadline dl,
                              const int64_t* wptrT, const int32_t* widxT, const uint64_t* wvalT) {
    // blocks of 1-8 warps, chosen so that as many warps as possible fit an SM's shared memory
    const int64_t per_warp = smp_warp_bytes(ldw);
    if (per_warp > 200 * 1024) return cudaErrorInvalidValue;
    int warps = 8;
    while (warps > 1 && warps * per_warp > 32 * 1024) warps >>= 1;
    const size_t smem = static_cast<size_t>(warps) * per_warp;
    cudaError_t e = cudaFuncSetAttribute(smp_packed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int64_t blocks = (q + warps - 1) / warps;
    int per_sm = static_cast<int>((220 * 1024) / (smem + 1024));
    if (per_sm < 1) per_sm = 1;
    if (blocks > static_cast<int64_t>(sms) * per_sm) blocks = static_cast<int64_t>(sms) * per_sm;
    if (blocks < 1) blocks = 1;
    const int max_levels = static_cast<int>(n + 1 < 0x7FFFFFFF ? n + 1 : 0x7FFFFFFF);
    smp_packed_kernel<<<static_cast<int>(blocks), warps * 32, smem, s>>>(
        wptr, widx, wval, n, ldw, src, ldw_src, q, out, ldw_out, levels,
        reinterpret_cast<unsigned long long*>(qcounter), reflexive, max_levels, dl, wptrT, widxT, wvalT);
    return cudaGetLastError();
}

cudaError_t launch_bit_transpose(const uint64_t* in, uint64_t* out, int64_t n, int64_t ldw, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 grid(static_cast<unsigned>((ldw + kTrWords - 1) / kTrWords), static_cast<unsigned>((ldw + 3) / 4));
    bit_transpose_kernel<<<grid, 256, 0, s>>>(in, out, n, ldw);
    return cudaGetLastError();
}

cudaError_t launch_frontier_group(const FrontierJob* jobs, int njobs, int64_t max_n, int64_t max_ldw, int64_t total,
                                  unsigned long long* counter, int sms, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    const int64_t per_warp = smp_warp_bytes(max_ldw);
    if (per_warp > 200 * 1024 || njobs > 65535) return cudaErrorInvalidValue;
    const unsigned nj = static_cast<unsigned>(njobs);
    const int64_t wpr = (max_n + 63) / 64;
    int64_t tb = wpr * wpr;
    if (tb > 4096) tb = 4096;
    frontier_transpose_kernel<<<dim3(static_cast<unsigned>(tb < 1 ? 1 : tb), nj), 64, 0, s>>>(jobs);
    const int rows_grid = warps_grid(max_n, sms) / 8 + 1;  // the jobs of a launch share the GPU
    frontier_wcsr_count_kernel<<<dim3(static_cast<unsigned>(rows_grid), nj, 2), 256, 0, s>>>(jobs);
    frontier_scan_kernel<<<dim3(1, nj, 2), 1024, 0, s>>>(jobs);
    frontier_wcsr_fill_kernel<<<dim3(static_cast<unsigned>(rows_grid), nj, 2), 256, 0, s>>>(jobs);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int warps = 8;
    while (warps > 1 && warps * per_warp > 32 * 1024) warps >>= 1;
    const size_t smem = static_cast<size_t>(warps) * per_warp;
    e = cudaFuncSetAttribute(frontier_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = static_cast<int>((220 * 1024) / (smem + 1024));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (total + warps - 1) / warps;
    if (blocks > static_cast<int64_t>(sms) * per_sm) blocks = static_cast<int64_t>(sms) * per_sm;
    if (blocks < 1) blocks = 1;
    frontier_group_kernel<<<static_cast<int>(blocks), warps * 32, smem, s>>>(jobs, njobs, total, max_ldw, counter);
    return cudaGetLastError();
}

}  // namespace bmlp
