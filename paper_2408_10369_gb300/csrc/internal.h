// Library-internal declarations shared by the C ABI and the kernel files.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/bmlp.h"

// e4m3 encoding of 1.0 (sign 0, exponent 0111, mantissa 000) used for the
// 0/1 tensor-core operands.
#define BMLP_E4M3_ONE 0x38

namespace bmlp {

// Tile shape of the tensor-core product: BM x BN output tile, BK bytes
// (= E4M3 elements) of the reduction dimension per pipeline stage.
constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_BK = 128;
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 192;   // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int TC_PAD = 256;       // matrices are padded to a multiple of this

// Epilogue modes of the tensor-core product kernel.
enum TcMode : int {
    TC_MODE_RMS = 0,    // out = old | (C > 0), also writes out^T; changed flag
    TC_MODE_SMP = 1,    // N = (C > 0) & ~V ; V |= N ; next = N; block flags
    TC_MODE_PLAIN = 2   // out = (C > 0)
};

struct TcParams {
    int32_t m_tiles, n_tiles, k_blocks;
    int32_t mode;
    int64_t ld;                 // row stride (bytes) of every 8-bit matrix
    const uint8_t* old_r;       // RMS: R of this iteration (row-major)
    uint8_t* out_r;             // RMS: new R; SMP: next frontier; PLAIN: output
    uint8_t* out_rt;            // RMS: new R^T
    uint8_t* visited;           // SMP: V (row-major, 0 / 1 bytes)
    const uint8_t* kflags;      // SMP: nonzero flag per (M block, K block) of A, or null
    uint8_t* kflags_next;       // SMP: flags for the next frontier
    int* changed;               // set to 1 when any output bit changed / is new
    int* error;                 // set to a nonzero code when a wait timed out
    long long wait_cycles;      // bound of each in-kernel wait
    // RMS block maps (only when k_blocks <= 256): fmap[rb * fm_ld + cb] = 1 iff the 128 x 128 block (rb, cb)
    // of R is nonzero, fmapT the transpose (fmapT[cb * fm_ld + rb]); rows padded with zeros to fm_ld, a
    // multiple of 16. The epilogue fills the maps of the new R (cleared by the caller).
    const uint8_t* fmap;
    const uint8_t* fmapT;
    uint8_t* fmap_next;
    uint8_t* fmapT_next;
    int32_t fm_ld;
    unsigned long long* issued; // multiply-adds issued in units of 128 x 32 x 128 (rows x columns x K), or null
    const int* guard;           // 4-bit squaring kernel: if not null and *guard == 0 the launch does nothing (a step
                                // of a device-side loop that a decision kernel switched off)
    // squaring kernels on packed operands: if not null, the epilogue also writes R' and R'^T as bit rows of ldb
    // 32-bit words (bit j of word u = column 32 u + j), n_pad rows each
    uint32_t* out_bits;
    uint32_t* out_bits_t;
    int64_t ldb;
};

// One problem of a grouped batch (device copy; built on the host).
struct GroupProblem {  // aligned as CUtensorMap (TMA descriptors must be 64-byte aligned)
    CUtensorMap mapA[2];   // A operand: M[parity] (row-major R)
    CUtensorMap mapB[2];   // B operand: T[parity] (R^T)
    CUtensorMap mapBF;     // composition: B of the final product = R1^T
    uint8_t* M[2];         // E4M3 R ping-pong (tensor-core engine)
    uint8_t* T[2];         // E4M3 R^T ping-pong
    uint8_t* X;            // composition: final product
    uint8_t* R1T;          // composition: E4M3 R1^T
    uint64_t* P[2];        // packed ping-pong (packed engine)
    const void* in1;       // caller's R1 (closure input, or composition r1)
    const void* in2;       // caller's R2 (composition r2)
    void* out;             // caller's output
    int64_t n;
    int64_t ld;            // n_pad (tensor-core engine)
    int64_t ldw;           // words per packed row (packed engine)
    int32_t m_tiles, n_tiles, k_blocks;
    int32_t kind;          // 0 closure, 1 composition
    int32_t engine;        // 0 tensor cores, 1 packed
    int32_t fmt;           // caller's format
    int32_t reflexive;
    int32_t cap;           // iteration cap
};

// Per-problem loop state of a grouped batch (device memory).
struct GroupState {
    int* parity;     // buffer holding the current R
    int* active;     // still iterating
    int* iters;      // products issued
    int* changed;    // set by the last product
    int* notconv;    // stopped at the cap while still changing
    int* tc_offs;    // exclusive prefix of active tensor-core tiles (nprob + 1)
    int* tc_total;
    int* pk_offs;    // exclusive prefix of active packed rows (nprob + 1)
    int* pk_total;
};

// Optional time budget of a long kernel: the first warp to look records the
// start (%globaltimer) in *t0; any warp that finds more than budget_ns
// elapsed raises *hit and stops taking work. budget_ns = 0: no budget.
struct Deadline {
    unsigned long long budget_ns;
    unsigned long long* t0;
    int* hit;
#ifdef __CUDACC__
    __device__ __forceinline__ bool past() const {
        if (budget_ns == 0) return false;
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        unsigned long long s = *reinterpret_cast<volatile unsigned long long*>(t0);
        if (s == 0) {
            atomicCAS(t0, 0ull, now);
            s = *reinterpret_cast<volatile unsigned long long*>(t0);
        }
        if (now > s && now - s > budget_ns) {
            *reinterpret_cast<volatile int*>(hit) = 1;
            return true;
        }
        return false;
    }
#endif
};

// Grow-only device buffer owned by a context.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace bmlp

struct bmlp_ctx {
    int device = 0;
    int sm_count = 0;
    int clock_khz = 0;           // SM clock rate, read once (the query takes hundreds of microseconds)
    char err[512] = {0};
    bmlp::DevBuf ws[40];
    void* batch = nullptr;       // cached grouped-batch graph (batch.cu)
    int tune[32];                // autotuned engine per size bucket (-1 = unknown)
    int* d_ctl = nullptr;        // device control words (see CTL_* below)
    int* h_ctl = nullptr;        // pinned host mirror
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bmlp_stats stats{};
    void* encode_fn = nullptr;   // cuTensorMapEncodeTiled from the driver
    double t_call = 0.0;         // host time at the start of the current call (s)
    uint64_t budget_ns = 0;      // time budget of the current call (0 = none)
    void* dispatch = nullptr;    // learned dispatcher state (dispatch.cu)
};

namespace bmlp {

// CTL_QCOUNT, CTL_T0, CTL_ISSUED and CTL_BITS are 64-bit words, CTL_COST and CTL_PSTAT (the ones and nonzero words
// a bit-row squaring wrote) two of them and CTL_THIN eight (two ints each, 8-byte aligned).
enum CtlWord : int {
    CTL_CHANGED = 0, CTL_ERROR = 1, CTL_ITERS = 2, CTL_LEVELS = 3, CTL_QCOUNT = 4, CTL_T0 = 6, CTL_BUDGET = 8,
    CTL_ISSUED = 10, CTL_COST = 12, CTL_THIN = 16, CTL_BITS = 32, CTL_PSTAT = 34, CTL_WORDS = 38
};
// The pinned host mirror has two more ints: CTL_HOST_I64 is a 64-bit slot for values read from elsewhere.
constexpr int CTL_HOST_I64 = CTL_WORDS;
constexpr int CTL_HOST_WORDS = CTL_WORDS + 2;

// Workspace slots of the grouped batch and of its device-driven large problems (the others are private to api.cu).
constexpr int WS_BATCH = 15;
constexpr int WS_SOLO = 25;

// ---- grouped batch (batch.cu)
// Problems with n >= solo_n (0: none) that may use the tensor cores run as device-driven single-problem pipelines
// (bit-row squarings, then 4-bit tensor-core squarings) inside the same graph; the rest are grouped.
bmlp_status batch_run_impl(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, int variant, long long wait_cycles,
                           int32_t* iters_out, cudaStream_t s, int64_t solo_n = 0);
// The step-cost model of the bit-row squarings (api.cu): seconds of a step from its word ORs, and of a dense 4-bit
// tensor-core product of n_pad.
double bitrow_s_per_word();
double bitrow_row_s_per_word();
double bitrow_step_s();
double tc4_product_s(int64_t n_pad);
// Synchronise s on behalf of the current call (counted in bmlp_stats.host_syncs).
cudaError_t host_sync(bmlp_ctx* ctx, cudaStream_t s);
void batch_cache_free(bmlp_ctx* ctx);

// ---- learned dispatcher (dispatch.cu)
bmlp_status dispatch_features_packed(bmlp_ctx* ctx, const uint64_t* P, int64_t n, int64_t ldw, float* feat_host,
                                     cudaStream_t s);
// features and prediction on the device, one host wait: *choice = the predicted fastest bmlp_variant
bmlp_status dispatch_choose_many_packed(bmlp_ctx* ctx, const uint64_t* const* P, const int64_t* n, const int64_t* ldw,
                                        int64_t m, float* feat_host, int32_t* choice, cudaStream_t s);
bmlp_status dispatch_choose_packed(bmlp_ctx* ctx, const uint64_t* P, int64_t n, int64_t ldw, int32_t* choice,
                                   cudaStream_t s);
bool dispatch_trained(const bmlp_ctx* ctx);
bmlp_status dispatch_predict(bmlp_ctx* ctx, const float* feats, int64_t m, float* pred, int32_t* choice,
                             cudaStream_t s);
bmlp_status dispatch_set_params(bmlp_ctx* ctx, const float* params, const float* mu, const float* sig);
bmlp_status dispatch_get_params(bmlp_ctx* ctx, float* params, float* mu, float* sig);
bmlp_status dispatch_loss_grad(bmlp_ctx* ctx, const float* X, const float* Y, const uint8_t* C, int64_t m, float* loss,
                               float* grad);
bmlp_status dispatch_train(bmlp_ctx* ctx, const float* X, const float* Y, const uint8_t* C, int64_t m,
                           const bmlp_train_cfg* cfg, float* final_loss);
bmlp_status dispatch_save(bmlp_ctx* ctx, const char* path);
bmlp_status dispatch_load(bmlp_ctx* ctx, const char* path);
void dispatch_free(bmlp_ctx* ctx);

// ---- workspace / error helpers (api.cu)
bmlp_status set_err(bmlp_ctx* ctx, bmlp_status st, const char* fmt, ...);
bmlp_status cuda_err(bmlp_ctx* ctx, cudaError_t e, const char* what);
bmlp_status ws_get(bmlp_ctx* ctx, int slot, size_t bytes, void** out);

// ---- encoders / decoders (encode.cu). All launched on `s`.
// u8 (any nonzero = 1) n x n, ld = n  ->  E4M3 0/1 R and R^T, n_pad x n_pad
void launch_u8_to_e4m3(const uint8_t* in, int64_t n, uint8_t* R, uint8_t* RT, int64_t n_pad, cudaStream_t s);
// packed rows (ldw_in words) -> E4M3 R and R^T (RT may be null)
void launch_packed_to_e4m3(const uint64_t* in, int64_t ldw_in, int64_t rows, int64_t n, uint8_t* R, uint8_t* RT,
                           int64_t n_pad, int64_t rows_pad, cudaStream_t s);
// E4M3 / 0-1 bytes (ld) -> u8 n x n (diagonal forced to 1 when reflexive)
void launch_bytes_to_u8(const uint8_t* R, int64_t ld, int64_t n, uint8_t* out, int reflexive, cudaStream_t s);
// E4M3 / 0-1 bytes (ld) -> packed rows (ldw_out words), rows x n
void launch_bytes_to_packed(const uint8_t* R, int64_t ld, int64_t rows, int64_t n, uint64_t* out, int64_t ldw_out,
                            int reflexive, cudaStream_t s);
// u8 n x n -> packed rows
void launch_u8_to_packed(const uint8_t* in, int64_t n, uint64_t* out, int64_t ldw_out, cudaStream_t s);
// packed (ldw_in) -> packed (ldw_out), masking bits >= n, optional diagonal
void launch_packed_copy(const uint64_t* in, int64_t ldw_in, int64_t rows, int64_t n, uint64_t* out, int64_t ldw_out,
                        int reflexive, cudaStream_t s);
// packed -> u8 n x n
void launch_packed_to_u8(const uint64_t* in, int64_t ldw, int64_t n, uint8_t* out, int reflexive, cudaStream_t s);
// out rows |= src rows (bits < n)
void launch_packed_or(uint64_t* out, int64_t ldw_out, const uint64_t* src, int64_t ldw_src, int64_t rows, int64_t n,
                      cudaStream_t s);
// identity as packed rows: row i has only bit i
void launch_identity_packed(uint64_t* out, int64_t ldw, int64_t n, cudaStream_t s);
// caller matrix (u8 n x n or packed n x ceil(n/64)) -> packed E2M1 R and R^T (n_pad x n_pad / 2 bytes)
void launch_u8_to_e2m1(const uint8_t* in, int64_t n, uint8_t* R, uint8_t* RT, int64_t n_pad, cudaStream_t s);
void launch_packed_to_e2m1(const uint64_t* in, int64_t ldw_in, int64_t n, uint8_t* R, uint8_t* RT, int64_t n_pad,
                           cudaStream_t s);
// packed E2M1 rows (ld4 bytes) -> u8 n x n / packed rows of ldw_out words (+ I if reflexive)
void launch_e2m1_to_u8(const uint8_t* Q, int64_t ld4, int64_t n, uint8_t* out, int reflexive, cudaStream_t s);
void launch_e2m1_to_packed(const uint8_t* Q, int64_t ld4, int64_t n, uint64_t* out, int64_t ldw_out, int reflexive,
                           cudaStream_t s);
// 1 per nonzero 128 x 128 block of an n x n matrix (fmt u8 with rows of n bytes, or packed with rows of
// ldw_in words), n_pad / 128 blocks a side
void launch_input_block_flags(const void* in, int32_t fmt, int64_t ldw_in, int64_t n, int64_t n_pad, uint8_t* flags,
                              int64_t flags_ld, cudaStream_t s);
// out = rows x cols AND NOT in over n x n packed rows (null vector = all constants)
void launch_packed_negate(const uint64_t* in, int64_t ldw_in, int64_t n, const uint64_t* rows, const uint64_t* cols,
                          uint64_t* out, int64_t ldw_out, cudaStream_t s);
// E4M3 bytes -> 0 / 1 in place (0x00 and 0x80 are zero, any other byte one), and 0 / 1 -> E4M3 0x00 / 0x38
void launch_e4m3_bytes_to_01(uint8_t* p, int64_t bytes, cudaStream_t s);
void launch_01_to_e4m3_bytes(uint8_t* p, int64_t bytes, cudaStream_t s);
// set the diagonal of an n x n byte matrix (ld) to E4M3 one
void launch_set_diag_e4m3(uint8_t* R, int64_t ld, int64_t n, cudaStream_t s);
void launch_set_diag_e2m1(uint8_t* Q, int64_t ld4, int64_t n, cudaStream_t s);
// per (M block, K block) nonzero flags of a byte matrix rows_pad x n_pad
// (row stride of flags: flags_ld, default n_pad / 128)
void launch_block_flags(const uint8_t* A, int64_t ld, int64_t rows_pad, int64_t n_pad, uint8_t* flags,
                        cudaStream_t s, int64_t flags_ld = 0);

// ---- tensor-core product (tc_product.cu)
// Set up tensor maps for A (rows x K) and B^T (cols x K) byte matrices.
bmlp_status make_tmap(bmlp_ctx* ctx, CUtensorMap* map, const void* base, int64_t rows, int64_t cols_bytes,
                      int64_t ld, int box_rows);
int tc_smem_bytes();
cudaError_t launch_tc_product(const CUtensorMap& a, const CUtensorMap& b, const TcParams& p, int grid,
                              cudaStream_t s);
// squaring step (RMS mode only) on packed E2M1 operands (n_pad x n_pad / 2 bytes, p.ld = n_pad / 2,
// p.k_blocks = n_pad / 256) as M = 256 MMAs per CTA pair (tcgen05 .cta_group::2, 2-CTA clusters) on pair tiles
// of 256 rows x tc4_tile_n() columns (p.n_tiles = ceil(n_pad / tc4_tile_n())); maps over R (A, box 128 rows)
// and R^T (b0: box 128 rows; b1: box tc4_b1_rows() rows), 128 bytes wide. p.issued counts 128 x 32 x 128
// multiply-add units.
int tc4_tile_n();
int tc4_b1_rows();
// the same squaring step on E4M3 operands (n_pad x n_pad bytes, p.ld = n_pad, p.k_blocks = n_pad / 128) as
// kind::f8f6f4 M = 256 MMAs per CTA pair on pair tiles of 256 x tc8_tile_n() (p.n_tiles = ceil(n_pad / that));
// no block maps (p.fmap must be null): A box 128 rows, b_half box 128 rows of R^T
int tc8_tile_n();
cudaError_t launch_tc8_product_duo(const CUtensorMap& a, const CUtensorMap& b_half, const TcParams& p, int sms,
                                   cudaStream_t s);
cudaError_t launch_tc4_product_duo(const CUtensorMap& a, const CUtensorMap& b0, const CUtensorMap& b1,
                                   const TcParams& p, int sms, cudaStream_t s);
// E4M3 bytes <-> packed E2M1 nibbles (sizes multiples of 16 bytes)
void launch_e4m3_to_e2m1(const uint8_t* in, uint8_t* out, int64_t bytes_in, cudaStream_t s);
void launch_e2m1_to_e4m3(const uint8_t* in, uint8_t* out, int64_t bytes_out, cudaStream_t s);
// grouped form: tc_group_kernel(const GroupProblem*, const GroupState*, int nprob, int phase, int* error,
// long long wait_cycles); phase 0 = squaring step of every active problem, 1 = final products of compositions
void* tc_group_kernel_ptr();
cudaError_t prepare_tc_group();

// ---- packed kernels (packed.cu)
// dst_i = (or_a ? A_i : 0) | OR_{k : A_ik = 1} B_k over n packed rows of ldw
// words (ldw even, matrices 16-byte aligned: rows move as 128-bit words; bits
// of A at columns >= n zero); raises *changed when dst_i != A_i. With A = B and or_a = 1 this is
// one squaring step R <- R + R R. tables: the Four Russians form (shared-memory
// tables of 4-row ORs; its time does not depend on the bits per word), else one
// warp per row gathering the named rows of B (time in proportion to the ones
// of A). pstat (or nullptr): the ones and the nonzero words of dst are added
// into pstat[0] and pstat[1].
cudaError_t launch_product_packed(const uint64_t* A, const uint64_t* B, uint64_t* dst, int64_t n, int64_t ldw,
                                  int or_a, int* changed, int sms, cudaStream_t s,
                                  Deadline dl = Deadline{0, nullptr, nullptr}, unsigned long long* pstat = nullptr,
                                  bool tables = true);
// word-CSR of packed rows: counts -> (exclusive scan by caller kernel) -> fill
// (widx / wval must hold n * ldw entries: the dense worst case; wptr holds n + 2 entries, wptr[n + 1] receives
// the largest row's count)
// scan_scratch: kScanMaxChunks x 2 int64 of device memory for a prefix over many blocks (n > 4096), or nullptr
// for one block; the two may not be shared by calls that overlap in time.
constexpr int kScanMaxChunks = 512;
cudaError_t launch_wcsr_build(const uint64_t* P, int64_t n, int64_t ldw, int64_t* wptr, int32_t* widx,
                              uint64_t* wval, cudaStream_t s, int64_t* scan_scratch = nullptr);
cudaError_t launch_smp_packed(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n,
                              int64_t ldw, const uint64_t* src, int64_t ldw_src, int64_t q, uint64_t* out,
                              int64_t ldw_out, int* levels, int* qcounter, int reflexive, int sms, cudaStream_t s,
                              Deadline dl = Deadline{0, nullptr, nullptr}, const int64_t* wptrT = nullptr,
                              const int32_t* widxT = nullptr, const uint64_t* wvalT = nullptr);
// C = P | P P on packed rows through the word index (wptr, widx, wval) of P
cudaError_t launch_square_rows(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, const uint64_t* P,
                               int64_t n, int64_t ldw, uint64_t* C, int sms, cudaStream_t s, int* changed = nullptr);
// Full closure rows by 64-source bit-sliced frontier expansion over the word index of R^T (rows 0 .. n-1 of out,
// ldw_out words each). scratch: smp_sliced_grid(n, sms) x 3 n words; *bcounter = 0 and *levels = 0 beforehand.
int64_t smp_sliced_grid(int64_t n, int sms);
cudaError_t launch_smp_sliced(const int64_t* wptrT, const int32_t* widxT, const uint64_t* wvalT, int64_t n,
                              uint64_t* scratch, uint64_t* out, int64_t ldw_out, unsigned long long* bcounter,
                              int* levels, int max_levels, int sms, cudaStream_t s, Deadline dl);
// The same expansion for query rows, with the frontier of each 64-row batch in the distributed shared memory of a
// thread-block cluster (one cluster per batch, n <= 65,536): rows 0 .. rows - 1 of out (ldw_out words each) are
// v_q R+ for the query rows in src (ldw_src words each), OR-ed with v_q when reflexive. *levels = 0 beforehand
// receives the largest level count. smp_cluster_fits: the shape exists for n and the device can hold one such
// cluster.
bool smp_cluster_shape(int64_t n, int64_t batches, int sms, int* ctas, int* log2_chunk);
bool smp_cluster_fits(int64_t n, int64_t rows, int sms);
cudaError_t launch_smp_cluster(const int64_t* wptrT, const int32_t* widxT, const uint64_t* wvalT, int64_t n,
                               const uint64_t* src, int64_t ldw_src, int64_t rows, uint64_t* out, int64_t ldw_out,
                               int reflexive, int* levels, int max_levels, int sms, cudaStream_t s, Deadline dl);
// ---- a squaring restricted to the rows and columns of R that still hold zeros (thin.cu)
// launch_thin_stats: bit rows P, PT (n rows of ldw = n_pad / 64 words) of the E2M1 R, R^T (ld4 = n_pad / 2 bytes per
// row) with their ones (rowcnt, colcnt); with bits_current, P and PT already hold R and R^T (written by the squaring
// kernel's epilogue and kept by launch_thin_squaring) and only their ones are counted; B = the columns with fewer
// than n / 2 ones (Bmask, blist) and Rb = the rows with a zero outside B (rlist); stat[0..5] = |B|, |Rb|, ones in B's
// columns, ones in Rb's rows, the most ones of a column of B and of a row of Rb.
// launch_thin_sample: of `rows` rows of Q spread over its n rows, those with at least n / 2 ones: stat[0] = the most
// ones of one, stat[1] = the most zeros of one (stat[0..1] zero beforehand).
// launch_thin_squaring: R' = R + R R on those columns and rows, the new ones ORed into Q (R) and QT (R^T) and into
// the bit rows P, PT in place, *changed raised when there are any; T1, T2: nb x ldw and nr x ldw words of scratch.
cudaError_t launch_thin_stats(const uint8_t* Q, const uint8_t* QT, int64_t ld4, int64_t n, uint64_t* P, uint64_t* PT,
                              int64_t ldw, int64_t* rowcnt, int64_t* colcnt, uint64_t* Bmask, int32_t* blist,
                              int32_t* rlist, unsigned long long* stat, bool bits_current, int sms, cudaStream_t s);
cudaError_t launch_thin_sample(const uint8_t* Q, int64_t ld4, int64_t n, int rows, unsigned long long* stat,
                               cudaStream_t s);
cudaError_t launch_thin_squaring(uint64_t* P, uint64_t* PT, int64_t ldw, const int32_t* blist, int64_t nb,
                                 const int32_t* rlist, int64_t nr, uint64_t* T1, uint64_t* T2, uint8_t* Q,
                                 uint8_t* QT, int64_t ld4, int* changed, int sms, cudaStream_t s);
// The same with |B| = stat[0] and |Rb| = stat[1] read on the device (T1: 2 n x ldw words; Rb's rows after B's),
// for device-driven pipelines whose host never sees the counts.
cudaError_t launch_thin_squaring_dev(uint64_t* P, uint64_t* PT, int64_t ldw, int64_t n, const int32_t* blist,
                                     const int32_t* rlist, const unsigned long long* stat, uint64_t* T1, uint8_t* Q,
                                     uint8_t* QT, int64_t ld4, int* changed, int sms, cudaStream_t s);
double thin_fixed_seconds(int64_t n_pad);
bool thin_is_enabled();
int thin_sample_rows();
double thin_row_spread();
// nonzero words of R + R R (out[0] += their total) and the word ORs of that squaring (out[1] += their total), from
// the word index of R (ldw words per row, at most 49,152), without forming R + R R; bits_out (if not null) += the
// ones of R
cudaError_t launch_square_growth(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n,
                                 int64_t ldw, unsigned long long* out, int sms, cudaStream_t s,
                                 unsigned long long* bits_out = nullptr);
// R^T's bit rows (n x ldw words) from R's word index: cleared, then every set bit (i, j) of R sets bit i of row j
// by a 64-bit atomic OR. Work in proportion to the ones of R, against n x ldw words read and written by
// launch_bit_transpose.
cudaError_t launch_scatter_transpose(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n,
                                     int64_t ldw, uint64_t* out, int sms, cudaStream_t s);
// word ORs of the next squaring step (sum over the set bits k of a row of the nonzero words of row k):
// cost[0] += their total over all rows, cost[1] = max(cost[1], the largest row's)
cudaError_t launch_square_cost(const int64_t* wptr, const int32_t* widx, const uint64_t* wval, int64_t n,
                               unsigned long long* cost, int sms, cudaStream_t s);
// (R+ + {(u, v)})+ in place on a transitive R+ (n packed rows of ldw words)
cudaError_t launch_insert_fact(uint64_t* P, int64_t n, int64_t ldw, int64_t u, int64_t v, int sms, cudaStream_t s);
// out = in^T on n x n packed rows of ldw words (every word of out written, padding words with zeros)
cudaError_t launch_bit_transpose(const uint64_t* in, uint64_t* out, int64_t n, int64_t ldw, cudaStream_t s);
int smp_packed_max_words();
// One closure by frontier expansion inside a grouped batch (device copy): every row of R1+ as one query row.
struct FrontierJob {
    const uint64_t* P;     // R as packed rows (n x ldw words, padding bits and words zero)
    uint64_t* PT;          // R^T, written by the launch
    int64_t* wptr;         // word index of R ((n + 2) offsets; entries sized for the dense worst case)
    int32_t* widx;
    uint64_t* wval;
    int64_t* wptrT;        // word index of R^T
    int32_t* widxT;
    uint64_t* wvalT;
    uint64_t* out;         // the closure rows (n x ldw words)
    int64_t n, ldw;        // ldw even
    int64_t first;         // first row of this job in the launch's row numbering (jobs in increasing order)
    int* levels;           // receives the deepest level + 1 (atomicMax; cleared by the caller)
};
// Transposes, word indexes and the frontier expansion of every row of every job (device array `jobs`,
// `total` rows in all; max_n / max_ldw over the jobs; *counter is cleared by the launch).
cudaError_t launch_frontier_group(const FrontierJob* jobs, int njobs, int64_t max_n, int64_t max_ldw, int64_t total,
                                  unsigned long long* counter, int sms, cudaStream_t s);

}  // namespace bmlp
