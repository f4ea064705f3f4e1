// Format converters between the caller's matrix layouts and the kernels'
// internal layouts (paper Sec. 3.2: row i of R is the bit code b_i).
//
//  * u8 / packed rows  ->  E4M3 0/1 bytes R (n_pad x n_pad) and its transpose
//    R^T, the K-major operands of the tensor-core product;
//  * E4M3 / 0-1 bytes  ->  u8 or packed rows;
//  * u8 <-> packed rows; per-block nonzero flags for frontier skipping.
//
// Padding rows and columns are written as zero: zero rows and columns add no
// paths, so padding never changes a closure.
#include "internal.h"

namespace bmlp {
namespace {

constexpr int T = 64;  // square tile edge (bytes) of the transposing encoders

__device__ __forceinline__ uint8_t e4m3_bit(bool b) { return b ? BMLP_E4M3_ONE : 0; }

// Source readers: one tile row segment of 16 logical elements as a 16-bit mask.
struct SrcU8 {
    const uint8_t* p;
    int64_t n;
    bool vec;  // rows are 16-byte aligned (n % 16 == 0 and p aligned)
    __device__ __forceinline__ uint32_t bits16(int64_t r, int64_t c0, int64_t rows) const {
        if (r >= rows || c0 >= n) return 0;
        const uint8_t* row = p + r * n;
        uint32_t m = 0;
        if (vec && c0 + 16 <= n) {
            uint4 v = *reinterpret_cast<const uint4*>(row + c0);
            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int x = 0; x < 16; ++x) m |= (((w[x >> 2] >> ((x & 3) * 8)) & 0xFFu) != 0 ? 1u : 0u) << x;
        } else {
            for (int x = 0; x < 16; ++x)
                if (c0 + x < n && row[c0 + x] != 0) m |= 1u << x;
        }
        return m;
    }
};

struct SrcPacked {
    const uint64_t* p;
    int64_t ldw;
    int64_t n;
    __device__ __forceinline__ uint32_t bits16(int64_t r, int64_t c0, int64_t rows) const {
        if (r >= rows || c0 >= n) return 0;
        uint64_t w = p[r * ldw + (c0 >> 6)];
        uint32_t m = static_cast<uint32_t>((w >> (c0 & 63)) & 0xFFFFu);
        int64_t valid = n - c0;
        if (valid < 16) m &= (1u << valid) - 1u;
        return m;
    }
};

__device__ __forceinline__ uint4 expand16(uint32_t m) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t v = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x) v |= static_cast<uint32_t>(e4m3_bit((m >> (q * 4 + x)) & 1u)) << (8 * x);
        w[q] = v;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// One 64 x 64 tile per block (256 threads, 16 elements each): writes R and,
// when RT != null, R^T. The grid covers rows_pad x n_pad.
template <class Src>
__global__ void encode_e4m3_tile(Src src, int64_t rows, uint8_t* __restrict__ R, uint8_t* __restrict__ RT,
                                 int64_t n_pad, int64_t rows_pad) {
    __shared__ uint16_t masks[T][T / 16 + 1];
    const int tid = threadIdx.x;
    const int r = tid >> 2, cseg = (tid & 3) * 16;
    const int64_t row0 = static_cast<int64_t>(blockIdx.y) * T, col0 = static_cast<int64_t>(blockIdx.x) * T;
    uint32_t m = src.bits16(row0 + r, col0 + cseg, rows);
    masks[r][tid & 3] = static_cast<uint16_t>(m);
    *reinterpret_cast<uint4*>(R + (row0 + r) * n_pad + col0 + cseg) = expand16(m);
    if (RT == nullptr) return;
    __syncthreads();
    // R^T row (col0 + r), columns row0 + cseg .. +16 = tile column r, rows cseg..cseg+15
    uint32_t t = 0;
#pragma unroll
    for (int x = 0; x < 16; ++x) t |= ((masks[cseg + x][r >> 4] >> (r & 15)) & 1u) << x;
    *reinterpret_cast<uint4*>(RT + (col0 + r) * rows_pad + row0 + cseg) = expand16(t);
}

// ---- packed E2M1 (4-bit) operands: element k of a row in byte k / 2, low
// nibble first; 0b0010 = 1.0.
// 8 bits -> 8 nibbles of {0, one}
__device__ __forceinline__ uint32_t nib_spread8(uint32_t b) {
    uint32_t t = b & 0xFFu;
    t = (t | (t << 12)) & 0x000F000Fu;
    t = (t | (t << 6)) & 0x03030303u;
    t = (t | (t << 3)) & 0x11111111u;
    return t << 1;
}
// 8 nibbles -> 8 bits (nonzero nibble = 1)
__device__ __forceinline__ uint32_t nib_gather8(uint32_t w) {
    uint32_t x = w | (w >> 1);
    x |= x >> 2;
    x &= 0x11111111u;
    x = (x | (x >> 3)) & 0x03030303u;
    x = (x | (x >> 6)) & 0x000F000Fu;
    x = (x | (x >> 12)) & 0xFFu;
    return x;
}

// One 64 x 64 tile per block (256 threads, 16 elements each): packed E2M1 R
// (row stride ld4 bytes) and R^T, as encode_e4m3_tile.
template <class Src>
__global__ void encode_e2m1_tile(Src src, int64_t rows, uint8_t* __restrict__ R, uint8_t* __restrict__ RT, int64_t ld4) {
    __shared__ uint16_t masks[T][T / 16 + 1];
    const int tid = threadIdx.x;
    const int r = tid >> 2, cseg = (tid & 3) * 16;
    const int64_t row0 = static_cast<int64_t>(blockIdx.y) * T, col0 = static_cast<int64_t>(blockIdx.x) * T;
    const uint32_t m = src.bits16(row0 + r, col0 + cseg, rows);
    masks[r][tid & 3] = static_cast<uint16_t>(m);
    *reinterpret_cast<uint2*>(R + (row0 + r) * ld4 + (col0 + cseg) / 2) = make_uint2(nib_spread8(m), nib_spread8(m >> 8));
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int x = 0; x < 16; ++x) t |= ((masks[cseg + x][r >> 4] >> (r & 15)) & 1u) << x;
    *reinterpret_cast<uint2*>(RT + (col0 + r) * ld4 + (row0 + cseg) / 2) = make_uint2(nib_spread8(t), nib_spread8(t >> 8));
}

// The 32 x 32 bit block held by a warp, one 32-bit row per lane (bit j =
// column j), transposed: lane j receives column j (bit i = row i). Five
// exchange stages, each swapping the off-diagonal s x s sub-blocks of every
// 2s x 2s block between lanes L and L ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int sh = 16 >> st;
        const uint32_t m = masks[st];  // the columns j with (j & sh) == 0
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, sh);
        x = (lane & sh) ? ((x & ~m) | ((y >> sh) & m)) : ((x & m) | ((y & m) << sh));
    }
    return x;
}

__device__ __forceinline__ uint4 nib_spread32(uint32_t b) {
    return make_uint4(nib_spread8(b), nib_spread8(b >> 8), nib_spread8(b >> 16), nib_spread8(b >> 24));
}

// Packed bit rows (ldw words per row, n x n) -> packed E2M1 R and R^T (n_pad x
// n_pad, row stride ld4 = n_pad / 2 bytes, padding zero): one 256 x 256 tile
// per block of 256 threads. Thread t reads row row0 + t (four 64-bit words);
// each warp turns its 32 rows into R^T bits as eight 32 x 32 bit blocks
// transposed in registers. Both bit tiles go through shared memory (rows of 8
// words padded to 9), so that every global store is 8 lanes x 16 bytes = one
// 128-byte line of a row of R or R^T, 4 lines per warp instruction.
__global__ void __launch_bounds__(256) packed_to_e2m1_kernel(const uint64_t* __restrict__ p, int64_t ldw, int64_t n,
                                                             uint8_t* __restrict__ R, uint8_t* __restrict__ RT,
                                                             int64_t ld4, bool vec) {
    __shared__ uint32_t sR[256][9];   // row t of the tile: bits of columns 32 w .. 32 w + 31 in word w
    __shared__ uint32_t sT[256][9];   // row c of the transposed tile: bits of rows 32 w .. 32 w + 31
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t row0 = static_cast<int64_t>(blockIdx.y) * 256, col0 = static_cast<int64_t>(blockIdx.x) * 256;
    const int64_t r = row0 + threadIdx.x;
    uint64_t w[4] = {0, 0, 0, 0};
    if (r < n) {
        const uint64_t* src = p + r * ldw + col0 / 64;
        const int64_t words = (n - col0 + 63) / 64;  // words of this row inside the tile that hold columns < n
        if (vec && words >= 4) {
            const uint4 a = reinterpret_cast<const uint4*>(src)[0], b = reinterpret_cast<const uint4*>(src)[1];
            w[0] = (static_cast<uint64_t>(a.y) << 32) | a.x;
            w[1] = (static_cast<uint64_t>(a.w) << 32) | a.z;
            w[2] = (static_cast<uint64_t>(b.y) << 32) | b.x;
            w[3] = (static_cast<uint64_t>(b.w) << 32) | b.z;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < words) w[q] = src[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t valid = n - (col0 + 64 * q);
            if (valid <= 0) w[q] = 0;
            else if (valid < 64) w[q] &= (1ull << valid) - 1ull;
        }
    }
    uint32_t x[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        x[2 * q] = static_cast<uint32_t>(w[q]);
        x[2 * q + 1] = static_cast<uint32_t>(w[q] >> 32);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        sR[threadIdx.x][k] = x[k];
        sT[32 * k + lane][warp] = warp_transpose32(x[k], lane);  // column 32 k + lane, rows 32 warp + i
    }
    __syncthreads();
    // lanes 8 q .. 8 q + 7 write the 8 pieces (16 bytes = 32 elements each) of one row
    const int piece = lane & 7;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int t = warp * 32 + i * 4 + (lane >> 3);
        *reinterpret_cast<uint4*>(R + (row0 + t) * ld4 + col0 / 2 + piece * 16) = nib_spread32(sR[t][piece]);
        *reinterpret_cast<uint4*>(RT + (col0 + t) * ld4 + row0 / 2 + piece * 16) = nib_spread32(sT[t][piece]);
    }
}

// Packed E2M1 rows -> u8 0/1 rows (n x n, + I if reflexive); 16 outputs per thread.
__global__ void e2m1_to_u8_kernel(const uint8_t* __restrict__ Q, int64_t ld4, int64_t n, uint8_t* __restrict__ out,
                                  int reflexive, bool vec_out) {
    const int64_t segs = (n + 15) / 16;
    const int64_t total = n * segs;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / segs, j0 = (t % segs) * 16;
        const uint2 v = *reinterpret_cast<const uint2*>(Q + i * ld4 + j0 / 2);
        uint32_t bits = nib_gather8(v.x) | (nib_gather8(v.y) << 8);
        if (reflexive && i >= j0 && i < j0 + 16) bits |= 1u << (i - j0);
        uint8_t* o = out + i * n + j0;
        if (vec_out && j0 + 16 <= n) {
            uint32_t q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                q[k] = ((bits >> (4 * k)) & 1u) | (((bits >> (4 * k + 1)) & 1u) << 8) |
                       (((bits >> (4 * k + 2)) & 1u) << 16) | (((bits >> (4 * k + 3)) & 1u) << 24);
            *reinterpret_cast<uint4*>(o) = make_uint4(q[0], q[1], q[2], q[3]);
        } else {
            for (int k = 0; k < 16 && j0 + k < n; ++k) o[k] = (bits >> k) & 1u;
        }
    }
}

// Packed E2M1 rows -> packed bit rows (ldw_out words, + I if reflexive); one output word per thread.
__global__ void e2m1_to_packed_kernel(const uint8_t* __restrict__ Q, int64_t ld4, int64_t n,
                                      uint64_t* __restrict__ out, int64_t ldw_out, int reflexive) {
    const int64_t wpr = (n + 63) / 64;
    const int64_t total = n * ldw_out;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / ldw_out, w = t % ldw_out;
        uint64_t bits = 0;
        if (w < wpr) {
            const uint4* src = reinterpret_cast<const uint4*>(Q + r * ld4 + w * 32);  // 64 nibbles
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const uint4 v = src[q];
                const uint64_t b = nib_gather8(v.x) | (nib_gather8(v.y) << 8) | (nib_gather8(v.z) << 16) |
                                   (static_cast<uint64_t>(nib_gather8(v.w)) << 24);
                bits |= b << (32 * q);
            }
            const int64_t valid = n - w * 64;
            if (valid < 64) bits &= (1ull << valid) - 1ull;
            if (reflexive && (r >> 6) == w) bits |= 1ull << (r & 63);
        }
        out[t] = bits;
    }
}

// 1 per nonzero 128 x 128 block of an input matrix (rows x n, padded to the block grid); one block of
// 256 threads per map entry, 16 elements per thread per pass.
template <class Src>
__global__ void input_block_flags_kernel(Src src, int64_t rows, int64_t flags_ld, uint8_t* __restrict__ flags) {
    const int64_t br = blockIdx.y, bc = blockIdx.x;
    const int tid = threadIdx.x;
    uint32_t any = 0;
#pragma unroll 4
    for (int k = 0; k < 4; ++k) {
        const int e = (k * 256 + tid) * 16;  // element offset inside the 128 x 128 block
        any |= src.bits16(br * 128 + e / 128, bc * 128 + e % 128, rows);
    }
    any = __syncthreads_or(any != 0);
    if (tid == 0) flags[br * flags_ld + bc] = any ? 1 : 0;
}

// out[i][j] = (R[i][j] != 0) | (reflexive && i == j); 16 outputs per thread.
__global__ void bytes_to_u8_kernel(const uint8_t* __restrict__ R, int64_t ld, int64_t n, uint8_t* __restrict__ out,
                                   int reflexive, bool vec_out) {
    const int64_t segs = (n + 15) / 16;
    const int64_t total = n * segs;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / segs, j0 = (t % segs) * 16;
        uint4 v = *reinterpret_cast<const uint4*>(R + i * ld + j0);
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint8_t b[16];
#pragma unroll
        for (int x = 0; x < 16; ++x) {
            b[x] = ((w[x >> 2] >> ((x & 3) * 8)) & 0xFFu) != 0;
            if (reflexive && j0 + x == i) b[x] = 1;
        }
        uint8_t* o = out + i * n + j0;
        if (vec_out && j0 + 16 <= n) {
            uint32_t q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                q[k] = b[4 * k] | (b[4 * k + 1] << 8) | (b[4 * k + 2] << 16) | (static_cast<uint32_t>(b[4 * k + 3]) << 24);
            *reinterpret_cast<uint4*>(o) = make_uint4(q[0], q[1], q[2], q[3]);
        } else {
            for (int x = 0; x < 16 && j0 + x < n; ++x) o[x] = b[x];
        }
    }
}

// One output word per thread: bits of R[r][64w .. 64w+63] != 0.
__global__ void bytes_to_packed_kernel(const uint8_t* __restrict__ R, int64_t ld, int64_t rows, int64_t n,
                                       uint64_t* __restrict__ out, int64_t ldw_out, int reflexive) {
    const int64_t wpr = (n + 63) / 64;
    const int64_t total = rows * ldw_out;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / ldw_out, w = t % ldw_out;
        uint64_t bits = 0;
        if (w < wpr) {
            const uint4* src = reinterpret_cast<const uint4*>(R + r * ld + w * 64);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 v = src[q];
                uint32_t x4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if ((x4[k >> 2] >> ((k & 3) * 8)) & 0xFFu) bits |= 1ull << (q * 16 + k);
            }
            const int64_t valid = n - w * 64;
            if (valid < 64) bits &= (1ull << valid) - 1ull;
            if (reflexive && r < n && (r >> 6) == w) bits |= 1ull << (r & 63);
        }
        out[t] = bits;
    }
}

// One output word per thread from u8 rows (ld = n).
__global__ void u8_to_packed_kernel(const uint8_t* __restrict__ in, int64_t n, uint64_t* __restrict__ out,
                                    int64_t ldw_out) {
    const int64_t wpr = (n + 63) / 64;
    const int64_t total = n * ldw_out;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / ldw_out, w = t % ldw_out;
        uint64_t bits = 0;
        if (w < wpr) {
            const uint8_t* row = in + r * n + w * 64;
            const int64_t valid = n - w * 64 < 64 ? n - w * 64 : 64;
            for (int k = 0; k < valid; ++k)
                if (row[k]) bits |= 1ull << k;
        }
        out[t] = bits;
    }
}

__global__ void packed_copy_kernel(const uint64_t* __restrict__ in, int64_t ldw_in, int64_t rows, int64_t n,
                                   uint64_t* __restrict__ out, int64_t ldw_out, int reflexive) {
    const int64_t wpr = (n + 63) / 64;
    const int64_t total = rows * ldw_out;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / ldw_out, w = t % ldw_out;
        uint64_t bits = 0;
        if (w < wpr) {
            bits = in[r * ldw_in + w];
            const int64_t valid = n - w * 64;
            if (valid < 64) bits &= (1ull << valid) - 1ull;
            if (reflexive && r < n && (r >> 6) == w) bits |= 1ull << (r & 63);
        }
        out[t] = bits;
    }
}

__global__ void packed_to_u8_kernel(const uint64_t* __restrict__ in, int64_t ldw, int64_t n, uint8_t* __restrict__ out,
                                    int reflexive) {
    const int64_t total = n * n;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / n, j = t % n;
        uint8_t b = (in[i * ldw + (j >> 6)] >> (j & 63)) & 1ull;
        if (reflexive && i == j) b = 1;
        out[t] = b;
    }
}

__global__ void packed_or_kernel(uint64_t* __restrict__ out, int64_t ldw_out, const uint64_t* __restrict__ src,
                                 int64_t ldw_src, int64_t rows, int64_t n) {
    const int64_t wpr = (n + 63) / 64;
    const int64_t total = rows * wpr;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / wpr, w = t % wpr;
        uint64_t s = src[r * ldw_src + w];
        const int64_t valid = n - w * 64;
        if (valid < 64) s &= (1ull << valid) - 1ull;
        out[r * ldw_out + w] |= s;
    }
}

__global__ void identity_packed_kernel(uint64_t* __restrict__ out, int64_t ldw, int64_t n) {
    const int64_t total = n * ldw;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / ldw, w = t % ldw;
        out[t] = ((r >> 6) == w) ? (1ull << (r & 63)) : 0ull;
    }
}

// NEG of Fig. 3 with the type literals of a stratified negation: out[i][j] =
// rows(i) AND cols(j) AND NOT in[i][j] for i, j < n; a null rows / cols
// vector admits every constant. Bits at j >= n stay zero.
__global__ void negate_restrict_kernel(const uint64_t* __restrict__ in, int64_t ldw_in, int64_t n,
                                       const uint64_t* __restrict__ rows, const uint64_t* __restrict__ cols,
                                       uint64_t* __restrict__ out, int64_t ldw_out) {
    const int64_t wpr = (n + 63) / 64;
    const int64_t total = n * ldw_out;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = t / ldw_out, w = t % ldw_out;
        uint64_t v = 0;
        if (w < wpr && (!rows || ((rows[r >> 6] >> (r & 63)) & 1ull))) {
            v = ~in[r * ldw_in + w];
            if (cols) v &= cols[w];
            const int64_t valid = n - w * 64;
            if (valid < 64) v &= (1ull << valid) - 1ull;
        }
        out[t] = v;
    }
}

// Entry (i, i) of a packed E2M1 matrix (ld bytes per row) set to one for i < n: nibble i & 1 of byte i / 2 of row i
// (each row's byte is written by one thread).
__global__ void set_diag_e2m1_kernel(uint8_t* Q, int64_t ld, int64_t n) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) Q[i * ld + (i >> 1)] |= static_cast<uint8_t>((i & 1) ? 0x20 : 0x02);
}

__global__ void set_diag_kernel(uint8_t* R, int64_t ld, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        R[i * ld + i] = BMLP_E4M3_ONE;
}

// flags[mb * kb_count + kb] = any nonzero byte in the 128 x 128 block (mb, kb).
__global__ void block_flags_kernel(const uint8_t* __restrict__ A, int64_t ld, int64_t kb_count,
                                   uint8_t* __restrict__ flags) {
    const int64_t mb = blockIdx.y, kb = blockIdx.x;
    const int r = threadIdx.x >> 1, half = threadIdx.x & 1;  // 256 threads: 128 rows x 2 halves of 64 bytes
    const uint4* p = reinterpret_cast<const uint4*>(A + (mb * 128 + r) * ld + kb * 128 + half * 64);
    uint32_t any = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 v = p[q];
        any |= v.x | v.y | v.z | v.w;
    }
    any = __syncthreads_or(any != 0);
    if (threadIdx.x == 0) flags[mb * kb_count + kb] = any ? 1 : 0;
}

inline int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

}  // namespace

void launch_u8_to_e4m3(const uint8_t* in, int64_t n, uint8_t* R, uint8_t* RT, int64_t n_pad, cudaStream_t s) {
    SrcU8 src{in, n, (n % 16 == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0)};
    dim3 grid(static_cast<unsigned>(n_pad / T), static_cast<unsigned>(n_pad / T));
    encode_e4m3_tile<SrcU8><<<grid, 256, 0, s>>>(src, n, R, RT, n_pad, n_pad);
}

void launch_packed_to_e4m3(const uint64_t* in, int64_t ldw_in, int64_t rows, int64_t n, uint8_t* R, uint8_t* RT,
                           int64_t n_pad, int64_t rows_pad, cudaStream_t s) {
    SrcPacked src{in, ldw_in, n};
    dim3 grid(static_cast<unsigned>(n_pad / T), static_cast<unsigned>(rows_pad / T));
    encode_e4m3_tile<SrcPacked><<<grid, 256, 0, s>>>(src, rows, R, RT, n_pad, rows_pad);
}

void launch_u8_to_e2m1(const uint8_t* in, int64_t n, uint8_t* R, uint8_t* RT, int64_t n_pad, cudaStream_t s) {
    SrcU8 src{in, n, (n % 16 == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0)};
    dim3 grid(static_cast<unsigned>(n_pad / T), static_cast<unsigned>(n_pad / T));
    encode_e2m1_tile<SrcU8><<<grid, 256, 0, s>>>(src, n, R, RT, n_pad / 2);
}

void launch_packed_to_e2m1(const uint64_t* in, int64_t ldw_in, int64_t n, uint8_t* R, uint8_t* RT, int64_t n_pad,
                           cudaStream_t s) {
    // n_pad is a multiple of 256 (TC_PAD); 16-byte row loads when every tile's first word is 16-byte aligned
    const bool vec = (ldw_in % 2 == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
    dim3 grid(static_cast<unsigned>(n_pad / 256), static_cast<unsigned>(n_pad / 256));
    packed_to_e2m1_kernel<<<grid, 256, 0, s>>>(in, ldw_in, n, R, RT, n_pad / 2, vec);
}

void launch_e2m1_to_u8(const uint8_t* Q, int64_t ld4, int64_t n, uint8_t* out, int reflexive, cudaStream_t s) {
    const bool vec = (n % 16 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    e2m1_to_u8_kernel<<<grid_for(n * ((n + 15) / 16), 256), 256, 0, s>>>(Q, ld4, n, out, reflexive, vec);
}

void launch_e2m1_to_packed(const uint8_t* Q, int64_t ld4, int64_t n, uint64_t* out, int64_t ldw_out, int reflexive,
                           cudaStream_t s) {
    e2m1_to_packed_kernel<<<grid_for(n * ldw_out, 256), 256, 0, s>>>(Q, ld4, n, out, ldw_out, reflexive);
}

void launch_input_block_flags(const void* in, int32_t fmt, int64_t ldw_in, int64_t n, int64_t n_pad, uint8_t* flags,
                              int64_t flags_ld, cudaStream_t s) {
    dim3 grid(static_cast<unsigned>(n_pad / 128), static_cast<unsigned>(n_pad / 128));
    if (fmt == BMLP_FMT_U8) {
        SrcU8 src{static_cast<const uint8_t*>(in), n,
                  (n % 16 == 0) && ((reinterpret_cast<uintptr_t>(in) & 15) == 0)};
        input_block_flags_kernel<SrcU8><<<grid, 256, 0, s>>>(src, n, flags_ld, flags);
    } else {
        SrcPacked src{static_cast<const uint64_t*>(in), ldw_in, n};
        input_block_flags_kernel<SrcPacked><<<grid, 256, 0, s>>>(src, n, flags_ld, flags);
    }
}

void launch_bytes_to_u8(const uint8_t* R, int64_t ld, int64_t n, uint8_t* out, int reflexive, cudaStream_t s) {
    bool vec = (n % 16 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    int64_t work = n * ((n + 15) / 16);
    bytes_to_u8_kernel<<<grid_for(work, 256), 256, 0, s>>>(R, ld, n, out, reflexive, vec);
}

void launch_bytes_to_packed(const uint8_t* R, int64_t ld, int64_t rows, int64_t n, uint64_t* out, int64_t ldw_out,
                            int reflexive, cudaStream_t s) {
    bytes_to_packed_kernel<<<grid_for(rows * ldw_out, 256), 256, 0, s>>>(R, ld, rows, n, out, ldw_out, reflexive);
}

void launch_u8_to_packed(const uint8_t* in, int64_t n, uint64_t* out, int64_t ldw_out, cudaStream_t s) {
    u8_to_packed_kernel<<<grid_for(n * ldw_out, 256), 256, 0, s>>>(in, n, out, ldw_out);
}

void launch_packed_copy(const uint64_t* in, int64_t ldw_in, int64_t rows, int64_t n, uint64_t* out, int64_t ldw_out,
                        int reflexive, cudaStream_t s) {
    packed_copy_kernel<<<grid_for(rows * ldw_out, 256), 256, 0, s>>>(in, ldw_in, rows, n, out, ldw_out, reflexive);
}

void launch_packed_to_u8(const uint64_t* in, int64_t ldw, int64_t n, uint8_t* out, int reflexive, cudaStream_t s) {
    packed_to_u8_kernel<<<grid_for(n * n, 256), 256, 0, s>>>(in, ldw, n, out, reflexive);
}

void launch_packed_or(uint64_t* out, int64_t ldw_out, const uint64_t* src, int64_t ldw_src, int64_t rows, int64_t n,
                      cudaStream_t s) {
    packed_or_kernel<<<grid_for(rows * ((n + 63) / 64), 256), 256, 0, s>>>(out, ldw_out, src, ldw_src, rows, n);
}

void launch_identity_packed(uint64_t* out, int64_t ldw, int64_t n, cudaStream_t s) {
    identity_packed_kernel<<<grid_for(n * ldw, 256), 256, 0, s>>>(out, ldw, n);
}

void launch_packed_negate(const uint64_t* in, int64_t ldw_in, int64_t n, const uint64_t* rows, const uint64_t* cols,
                          uint64_t* out, int64_t ldw_out, cudaStream_t s) {
    negate_restrict_kernel<<<grid_for(n * ldw_out, 256), 256, 0, s>>>(in, ldw_in, n, rows, cols, out, ldw_out);
}

void launch_set_diag_e4m3(uint8_t* R, int64_t ld, int64_t n, cudaStream_t s) {
    set_diag_kernel<<<grid_for(n, 256), 256, 0, s>>>(R, ld, n);
}

void launch_set_diag_e2m1(uint8_t* Q, int64_t ld4, int64_t n, cudaStream_t s) {
    set_diag_e2m1_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(Q, ld4, n);
}

void launch_block_flags(const uint8_t* A, int64_t ld, int64_t rows_pad, int64_t n_pad, uint8_t* flags,
                        cudaStream_t s, int64_t flags_ld) {
    dim3 grid(static_cast<unsigned>(n_pad / 128), static_cast<unsigned>(rows_pad / 128));
    block_flags_kernel<<<grid, 256, 0, s>>>(A, ld, flags_ld > 0 ? flags_ld : n_pad / 128, flags);
}

namespace {
__global__ void e4m3_to_01_kernel(uint8_t* __restrict__ p, int64_t bytes) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < bytes;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = (p[i] & 0x7Fu) != 0 ? 1 : 0;
}
__global__ void to_e4m3_bytes_kernel(uint8_t* __restrict__ p, int64_t bytes) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < bytes;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = p[i] != 0 ? static_cast<uint8_t>(BMLP_E4M3_ONE) : 0;
}
int byte_grid(int64_t bytes) {
    int64_t g = (bytes + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return static_cast<int>(g < 1 ? 1 : g);
}
}  // namespace

void launch_e4m3_bytes_to_01(uint8_t* p, int64_t bytes, cudaStream_t s) {
    e4m3_to_01_kernel<<<byte_grid(bytes), 256, 0, s>>>(p, bytes);
}

void launch_01_to_e4m3_bytes(uint8_t* p, int64_t bytes, cudaStream_t s) {
    to_e4m3_bytes_kernel<<<byte_grid(bytes), 256, 0, s>>>(p, bytes);
}

}  // namespace bmlp
