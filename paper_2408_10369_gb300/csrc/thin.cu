// A squaring R <- R + R R (Eq. 4, Algorithm 1) restricted to the entries of R that are still zero.
//
// R' = R | C with C = R R can differ from R only where R is 0. Let B be any set of columns and Rb the rows that
// have a zero outside B; every zero of R then lies in a column of B or a row of Rb, so
//     C[:, b] = OR_{k : R[k][b] = 1} R[:, k]   (b in B: row b of R'^T gains row k of R^T for each such k)
//     C[r, :] = OR_{k : R[r][k] = 1} R[k, :]   (r in Rb)
// give every entry of R' that can change. With B = the columns holding fewer than n / 2 ones, a matrix close to
// its closure (the squaring that only confirms the fixpoint, and the one before it on many graphs) has few such
// columns and rows, and they hold few ones: the step costs a few row ORs on bit rows instead of a dense product.
// The result is the same R', so the count of products and the fixpoint test are those of Algorithm 1.
//
// The tensor-core squarings keep R and R^T as packed E2M1 rows (element k of a row in byte k / 2, low nibble for
// even k, one = 0b0010); this file reads them as bit rows and ORs the new ones back into them in place.
#include "internal.h"

namespace bmlp {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// 8 E2M1 nibbles (a 32-bit word) -> 8 bits, bit k = (nibble k != 0).
__device__ __forceinline__ uint32_t nib_bits8(uint32_t w) {
    uint32_t x = w | (w >> 1);
    x |= x >> 2;
    x &= 0x11111111u;
    x = (x | (x >> 3)) & 0x03030303u;
    x = (x | (x >> 6)) & 0x000F000Fu;
    x = (x | (x >> 12)) & 0xFFu;
    return x;
}

// Bit rows (ldw words each) of the n_rows x n_cols E2M1 matrix Q (ld4 bytes per row, columns beyond n_cols zero),
// and the ones of each row into cnt. Warp per row; a lane turns 8 bytes (16 nibbles) into 16 bits at a time.
__global__ void __launch_bounds__(256) e2m1_to_bits_kernel(const uint8_t* __restrict__ Q, int64_t ld4, int64_t n_rows,
                                                           uint64_t* __restrict__ P, int64_t ldw,
                                                           int64_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_rows;
         i += warps) {
        const uint2* row = reinterpret_cast<const uint2*>(Q + i * ld4);
        uint64_t* prow = P + i * ldw;
        int64_t c = 0;
        // word w of the bit row = 64 columns = 32 bytes = 4 uint2 of nibbles
        for (int64_t w = lane; w < ldw; w += 32) {
            uint64_t bits = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t u = w * 4 + q;  // uint2 index: columns 16 u .. 16 u + 15
                uint64_t b16 = 0;
                if (u * 8 < ld4) {
                    const uint2 v = row[u];
                    b16 = static_cast<uint64_t>(nib_bits8(v.x) | (nib_bits8(v.y) << 8));
                }
                bits |= b16 << (16 * q);
            }
            prow[w] = bits;
            c += __popcll(bits);
        }
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
        if (lane == 0) cnt[i] = c;
    }
}

// The ones of each of the n_rows bit rows of P (ldw words each) into cnt (warp per row).
__global__ void __launch_bounds__(256) bits_count_kernel(const uint64_t* __restrict__ P, int64_t ldw, int64_t n_rows,
                                                         int64_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_rows;
         i += warps) {
        const uint64_t* row = P + i * ldw;
        int64_t c = 0;
        for (int64_t w = lane; w < ldw; w += 32) c += __popcll(row[w]);
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
        if (lane == 0) cnt[i] = c;
    }
}

// Columns of B: colcnt[j] < n / 2 (j < n). Bmask gets their bits, blist the columns (in no particular order);
// stat[0] += |B|, stat[2] += the ones in those columns, stat[4] = the most ones of one of them.
__global__ void thin_columns_kernel(const int64_t* __restrict__ colcnt, int64_t n, uint64_t* __restrict__ Bmask,
                                    int32_t* __restrict__ blist, unsigned long long* __restrict__ stat) {
    const int64_t wpr = (n + 63) >> 6;
    for (int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; w < wpr;
         w += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint64_t m = 0;
        unsigned long long ones = 0;
        for (int b = 0; b < 64; ++b) {
            const int64_t j = w * 64 + b;
            if (j < n && 2 * colcnt[j] < n) {
                m |= 1ull << b;
                ones += static_cast<unsigned long long>(colcnt[j]);
            }
        }
        Bmask[w] = m;
        if (m) {
            const unsigned long long at = atomicAdd(&stat[0], static_cast<unsigned long long>(__popcll(m)));
            uint64_t mm = m;
            unsigned long long top = 0;
            for (unsigned long long k = at; mm; ++k) {
                const int64_t j = w * 64 + (__ffsll(static_cast<long long>(mm)) - 1);
                blist[k] = static_cast<int32_t>(j);
                top = static_cast<unsigned long long>(colcnt[j]) > top ? static_cast<unsigned long long>(colcnt[j]) : top;
                mm &= mm - 1ull;
            }
            atomicAdd(&stat[2], ones);
            atomicMax(&stat[4], top);
        }
    }
}

// Rows of Rb: a zero at some column j < n outside B. rlist gets them; stat[1] += |Rb|, stat[3] += their ones,
// stat[5] = the most ones of one of them.
__global__ void __launch_bounds__(256) thin_rows_kernel(const uint64_t* __restrict__ P, int64_t ldw, int64_t n,
                                                        const int64_t* __restrict__ rowcnt,
                                                        const uint64_t* __restrict__ Bmask, int32_t* __restrict__ rlist,
                                                        unsigned long long* __restrict__ stat) {
    const int lane = threadIdx.x & 31;
    const int64_t wpr = (n + 63) >> 6;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        bool gap = false;
        for (int64_t w = lane; w < wpr; w += 32) {
            const int64_t valid = n - w * 64;
            const uint64_t cols = valid < 64 ? (1ull << valid) - 1ull : ~0ull;  // columns j < n of this word
            gap |= ((P[i * ldw + w] | Bmask[w]) & cols) != cols;
        }
        if (__any_sync(FULL, gap) && lane == 0) {
            rlist[atomicAdd(&stat[1], 1ull)] = static_cast<int32_t>(i);
            atomicAdd(&stat[3], static_cast<unsigned long long>(rowcnt[i]));
            atomicMax(&stat[5], static_cast<unsigned long long>(rowcnt[i]));
        }
    }
}

// Of `rows` rows of the E2M1 matrix Q spread evenly over its n rows, those with at least n / 2 ones: stat[0] = the
// most ones of one, stat[1] = the most zeros (among columns < n) of one (warp per row).
__global__ void __launch_bounds__(256) e2m1_sample_kernel(const uint8_t* __restrict__ Q, int64_t ld4, int64_t n,
                                                          int rows, unsigned long long* __restrict__ stat) {
    const int lane = threadIdx.x & 31;
    const int r = static_cast<int>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const int64_t i = static_cast<int64_t>(r) * n / rows;
    const uint4* row = reinterpret_cast<const uint4*>(Q + i * ld4);
    unsigned long long c = 0;
    for (int64_t u = lane; u * 16 < ld4; u += 32) {  // 16 bytes = 32 nibbles
        const uint4 v = row[u];
        c += __popc(nib_bits8(v.x)) + __popc(nib_bits8(v.y)) + __popc(nib_bits8(v.z)) + __popc(nib_bits8(v.w));
    }
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
    if (lane == 0 && 2 * c >= static_cast<unsigned long long>(n)) {
        atomicMax(&stat[0], c);
        atomicMax(&stat[1], static_cast<unsigned long long>(n) - c);
    }
}

// T[l] = OR of Src[k] over the set bits k of Src[list[l]] (bit rows of ldw words; warp per list entry, each lane
// ORing its own words of T[l], so one entry's work runs on one warp). With count_dev, the count is *count_dev, and
// with toff_dev, T starts *toff_dev rows further (counts known only on the device).
__global__ void __launch_bounds__(256) thin_row_or_kernel(const uint64_t* __restrict__ Src, int64_t ldw,
                                                          const int32_t* __restrict__ list, int64_t count,
                                                          uint64_t* __restrict__ T,
                                                          const unsigned long long* __restrict__ count_dev,
                                                          const unsigned long long* __restrict__ toff_dev) {
    if (count_dev != nullptr) count = static_cast<int64_t>(*count_dev);
    if (toff_dev != nullptr) T += static_cast<int64_t>(*toff_dev) * ldw;
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t l = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); l < count;
         l += warps) {
        const uint64_t* row = Src + static_cast<int64_t>(list[l]) * ldw;
        uint64_t* out = T + l * ldw;
        for (int64_t w = lane; w < ldw; w += 32) out[w] = 0ull;
        __syncwarp();
        for (int64_t wb = 0; wb < ldw; wb += 32) {
            const uint64_t x = wb + lane < ldw ? row[wb + lane] : 0ull;
            unsigned m = __ballot_sync(FULL, x != 0ull);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1u;
                uint64_t bits = __shfl_sync(FULL, x, src);
                const int64_t base = (wb + src) * 64;
                while (bits) {
                    const int64_t k = base + (__ffsll(static_cast<long long>(bits)) - 1);
                    bits &= bits - 1ull;
                    const uint64_t* rk = Src + k * ldw;
                    for (int64_t w = lane; w < ldw; w += 32) out[w] |= rk[w];  // lane-owned words
                }
            }
        }
    }
}

// One set entry (row, col) of an E2M1 matrix (ld4 bytes per row), ORed into its 32-bit word.
__device__ __forceinline__ void set_nibble(uint8_t* Q, int64_t ld4, int64_t row, int64_t col) {
    const int64_t byte = row * ld4 + (col >> 1);
    const uint32_t bit = static_cast<uint32_t>((byte & 3) * 8 + (col & 1) * 4 + 1);
    atomicOr(reinterpret_cast<unsigned int*>(Q + (byte & ~int64_t(3))), 1u << bit);
}

// New ones of a thin squaring into R (Q and the bit rows P) and R^T (QT and PT): for list entry l with index
// x = list[l] and computed row T[l], the bits of T[l] not in row x of Cur (P, or PT when transposed) are entry
// (x, j) of Cur's matrix (R[j][x] when transposed). Word w of row x is read and written by one thread only (list
// entries are distinct), and the other matrix's bits go in with atomic ORs; a one that the column pass already set
// is not new to the row pass. Raises *changed when anything is new.
__global__ void __launch_bounds__(256) thin_apply_kernel(uint64_t* P, uint64_t* PT, const uint64_t* __restrict__ T,
                                                         int64_t ldw, const int32_t* __restrict__ list, int64_t count,
                                                         int transposed, uint8_t* __restrict__ Q,
                                                         uint8_t* __restrict__ QT, int64_t ld4,
                                                         int* __restrict__ changed,
                                                         const unsigned long long* __restrict__ count_dev,
                                                         const unsigned long long* __restrict__ toff_dev) {
    if (count_dev != nullptr) count = static_cast<int64_t>(*count_dev);
    if (toff_dev != nullptr) T += static_cast<int64_t>(*toff_dev) * ldw;
    uint64_t* Cur = transposed ? PT : P;
    uint64_t* Other = transposed ? P : PT;
    const int64_t total = count * ldw;
    bool any = false;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t l = t / ldw, w = t % ldw;
        const int64_t x = list[l];
        const uint64_t old = Cur[x * ldw + w];
        uint64_t nb = T[t] & ~old;
        any |= nb != 0ull;
        if (nb) Cur[x * ldw + w] = old | nb;
        while (nb) {
            const int64_t j = w * 64 + (__ffsll(static_cast<long long>(nb)) - 1);
            nb &= nb - 1ull;
            const int64_t r = transposed ? j : x, c = transposed ? x : j;  // the new entry is R[r][c]
            set_nibble(Q, ld4, r, c);
            set_nibble(QT, ld4, c, r);
            atomicOr(reinterpret_cast<unsigned long long*>(Other + j * ldw + (x >> 6)), 1ull << (x & 63));
        }
    }
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(changed, 1);
}

int rows_grid(int64_t rows, int sms) {
    int64_t blocks = (rows + 7) / 8;
    const int64_t cap = static_cast<int64_t>(sms) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return static_cast<int>(blocks);
}

}  // namespace

cudaError_t launch_thin_sample(const uint8_t* Q, int64_t ld4, int64_t n, int rows, unsigned long long* stat,
                               cudaStream_t s) {
    if (rows < 1) return cudaSuccess;
    e2m1_sample_kernel<<<(rows + 7) / 8, 256, 0, s>>>(Q, ld4, n, rows, stat);
    return cudaGetLastError();
}

cudaError_t launch_thin_stats(const uint8_t* Q, const uint8_t* QT, int64_t ld4, int64_t n, uint64_t* P, uint64_t* PT,
                              int64_t ldw, int64_t* rowcnt, int64_t* colcnt, uint64_t* Bmask, int32_t* blist,
                              int32_t* rlist, unsigned long long* stat, bool bits_current, int sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(stat, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (bits_current) {
        bits_count_kernel<<<rows_grid(n, sms), 256, 0, s>>>(P, ldw, n, rowcnt);
        bits_count_kernel<<<rows_grid(n, sms), 256, 0, s>>>(PT, ldw, n, colcnt);
    } else {
        e2m1_to_bits_kernel<<<rows_grid(n, sms), 256, 0, s>>>(Q, ld4, n, P, ldw, rowcnt);
        e2m1_to_bits_kernel<<<rows_grid(n, sms), 256, 0, s>>>(QT, ld4, n, PT, ldw, colcnt);
    }
    const int64_t wpr = (n + 63) / 64;
    thin_columns_kernel<<<static_cast<int>((wpr + 255) / 256), 256, 0, s>>>(colcnt, n, Bmask, blist, stat);
    thin_rows_kernel<<<rows_grid(n, sms), 256, 0, s>>>(P, ldw, n, rowcnt, Bmask, rlist, stat);
    return cudaGetLastError();
}

cudaError_t launch_thin_squaring(uint64_t* P, uint64_t* PT, int64_t ldw, const int32_t* blist, int64_t nb,
                                 const int32_t* rlist, int64_t nr, uint64_t* T1, uint64_t* T2, uint8_t* Q,
                                 uint8_t* QT, int64_t ld4, int* changed, int sms, cudaStream_t s) {
    if (nb > 0) thin_row_or_kernel<<<rows_grid(nb, sms), 256, 0, s>>>(PT, ldw, blist, nb, T1, nullptr, nullptr);
    if (nr > 0) thin_row_or_kernel<<<rows_grid(nr, sms), 256, 0, s>>>(P, ldw, rlist, nr, T2, nullptr, nullptr);
    // every new one is found from the old R before any is written
    const int apply_grid = sms * 8;
    if (nb > 0)
        thin_apply_kernel<<<apply_grid, 256, 0, s>>>(P, PT, T1, ldw, blist, nb, 1, Q, QT, ld4, changed, nullptr,
                                                     nullptr);
    if (nr > 0)
        thin_apply_kernel<<<apply_grid, 256, 0, s>>>(P, PT, T2, ldw, rlist, nr, 0, Q, QT, ld4, changed, nullptr,
                                                     nullptr);
    return cudaGetLastError();
}

cudaError_t launch_thin_squaring_dev(uint64_t* P, uint64_t* PT, int64_t ldw, int64_t n, const int32_t* blist,
                                     const int32_t* rlist, const unsigned long long* stat, uint64_t* T1, uint8_t* Q,
                                     uint8_t* QT, int64_t ld4, int* changed, int sms, cudaStream_t s) {
    // |B| = stat[0] and |Rb| = stat[1] are read by the kernels; the grids cover up to n entries each
    const int g = rows_grid(n, sms);
    thin_row_or_kernel<<<g, 256, 0, s>>>(PT, ldw, blist, 0, T1, stat, nullptr);
    thin_row_or_kernel<<<g, 256, 0, s>>>(P, ldw, rlist, 0, T1, stat + 1, stat);
    const int apply_grid = sms * 8;
    thin_apply_kernel<<<apply_grid, 256, 0, s>>>(P, PT, T1, ldw, blist, 0, 1, Q, QT, ld4, changed, stat, nullptr);
    thin_apply_kernel<<<apply_grid, 256, 0, s>>>(P, PT, T1, ldw, rlist, 0, 0, Q, QT, ld4, changed, stat + 1, stat);
    return cudaGetLastError();
}

}  // namespace bmlp
