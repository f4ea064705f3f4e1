// C ABI of the library (declared in include/bmlp.h): argument checks,
// host/device staging, the fixpoint drivers of BMLP-RMS (Algorithm 1),
// BMLP-SMP (Algorithm 2) and composition (Thm. 1), and the workspace.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define BMLP_HAVE_NVTX 1
#endif

using namespace bmlp;

namespace bmlp {

bmlp_status set_err(bmlp_ctx* ctx, bmlp_status st, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

bmlp_status cuda_err(bmlp_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(ctx, BMLP_ERR_OOM, "%s: out of device memory", what);
    }
    return set_err(ctx, BMLP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bmlp_status ws_get(bmlp_ctx* ctx, int slot, size_t bytes, void** out) {
    DevBuf& b = ctx->ws[slot];
    if (bytes == 0) bytes = 16;
    if (b.bytes < bytes) {
        if (b.p) {
            cudaError_t e = cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
            if (e != cudaSuccess) return cuda_err(ctx, e, "cudaFree(workspace)");
        }
        size_t want = bytes + bytes / 8;  // grow with headroom
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            b.p = nullptr;
            return cuda_err(ctx, e, "cudaMalloc(workspace)");
        }
        b.bytes = want;
    }
    *out = b.p;
    return BMLP_OK;
}

cudaError_t host_sync(bmlp_ctx* ctx, cudaStream_t s) {
    ctx->stats.host_syncs++;
    return cudaStreamSynchronize(s);
}

}  // namespace bmlp

namespace {

// A named range around a call or a phase of it, for profilers that read NVTX (ncu --nvtx, nsys); without a tool
// attached a push and a pop cost a few nanoseconds.
struct NvtxRange {
#ifdef BMLP_HAVE_NVTX
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char*) {}
#endif
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Workspace slots.
enum : int {
    WS_IN0 = 0, WS_IN1 = 1, WS_OUT = 2,
    WS_M0 = 3, WS_M1 = 4, WS_T0 = 5, WS_T1 = 6, WS_M2 = 7,
    WS_WPTR = 8, WS_WIDX = 9, WS_WVAL = 10, WS_F0 = 11, WS_F1 = 12, WS_V = 13, WS_SRC = 14,
    WS_FEAT = 16, WS_PT = 17, WS_WPTRT = 18, WS_WIDXT = 19
};
constexpr int WS_WVALT = 20;
// Relation operators and the composed isForeign program (packed buffers and type vectors).
constexpr int WS_PIPE0 = 21, WS_PIPE1 = 22, WS_PIPE2 = 23, WS_VEC0 = 24;
// R + R R and its word index, before a frontier closure of a path-like R.
constexpr int WS_SQP = 27, WS_SQPTR = 28, WS_SQIDX = 29, WS_SQVAL = 30;
// E4M3 inputs turned into 0 / 1 bytes, and the 0 / 1 result before it becomes E4M3 bytes.
constexpr int WS_E8_IN0 = 31, WS_E8_IN1 = 32, WS_E8_OUT = 33;
// Block totals of the prefix over many blocks in a word-index build.
constexpr int WS_SCAN = 34;
// Bit rows of R and R^T, their ones, the column mask and the row and column lists, and the computed rows of a
// squaring restricted to the rows and columns that still hold zeros.
constexpr int WS_THIN_P = 35, WS_THIN_AUX = 36, WS_THIN_T = 37;
constexpr int64_t kSquareMinN = 4096;
// Bits per nonzero word of R from which a whole-row bit-row squaring uses the Four Russians tables instead of
// gathering the named rows (measured at n = 8,192 and 16,384: equal times at 9.5 and 11.5 bits).
constexpr double kM4MinBitsPerWord = 10.0;
constexpr int kSquareMaxSteps = 3;  // measured: chains with 1 % shortcuts are fastest after 3 (band of 8)
// A squaring is kept while it grows the rows' nonzero words by at most this factor (path-like relations).
constexpr double kSquareMaxGrowth = 1.5;
// A full frontier closure expands 64 sources at a time when R + R R has more than this many times the nonzero
// words of R (rows that widen fast reach most constants within a few levels; measured on ER, SBM, power-law and
// grid graphs: the sliced kernel wins above about 2.8, the one-query-per-warp kernel below) ...
constexpr double kSlicedMinGrowth = 2.8;
// ... and no column of R has more than this many times the mean nonzero words of a column (a pull rescans a hub's
// in-list at every level until every active source reaches it).
constexpr double kSlicedMaxSkew = 16.0;
// Closures whose largest column holds more than this many times the mean nonzero words of a column run on the
// cluster kernel, whose warps walk many constants' in-lists together (measured on the corpus at n = 22,535-32,629:
// power-law targets, column skew 7.8-15.6, 0.71-0.93 of the global-memory kernel's time; ER and SBM, skew 2.9-5.3,
// 0.99-1.33 of it).
constexpr double kClusterClosureSkew = 6.5;
// Query batches of at least this many rows take the same test (a batch of 64 rows is one cluster's work).
constexpr int64_t kSlicedMinQueries = 64;
// Fraction of nonzero 128 x 128 blocks of R below which a squaring skips empty K blocks.
constexpr double kSkipMaxDensity = 0.5;
// Fixed device and host time of a squaring restricted to the rows and columns of R that hold zeros: the bit rows of
// R and R^T (reading both E2M1 matrices, writing both bit-row copies and reading R's again: about 1.4 bytes per
// entry at about 6 TB/s), the row and column lists and two flag read-backs; the row ORs are costed per word as the
// bit-row squarings' are.
double thin_fixed_s(int64_t n_pad) {
    return 30e-6 + static_cast<double>(n_pad) * static_cast<double>(n_pad) * 1.4 / 6.0e12;
}
// The rows and columns holding zeros are sized only after a squaring whose R, in kThinSampleRows rows spread over it,
// has its rows with at least n / 2 ones within this fraction of n of one another in count (the rows that reach most
// constants are saturated, their zeros in common columns).
constexpr double kThinRowSpread = 1.0 / 32.0;
constexpr int kThinSampleRows = 256;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, what); \
    } while (0)

#define ST(call)                                  \
    do {                                          \
        bmlp_status s_ = (call);                  \
        if (s_ != BMLP_OK) return s_;             \
    } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t words_of(int64_t n) { return (n + 63) / 64; }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t fmt_bytes(int32_t fmt, int64_t rows, int64_t n) {
    return fmt == BMLP_FMT_U8 ? static_cast<size_t>(rows) * static_cast<size_t>(n)
                              : static_cast<size_t>(rows) * static_cast<size_t>(words_of(n)) * 8;
}

// A caller's matrix: its device view (staged when the caller passed host memory).
struct Operand {
    const void* dev = nullptr;
    bool host = false;
};

bmlp_status stage_in(bmlp_ctx* ctx, const void* p, size_t bytes, int slot, cudaStream_t s, Operand* o) {
    if (is_device_ptr(p)) {
        o->dev = p;
        o->host = false;
        return BMLP_OK;
    }
    void* d = nullptr;
    ST(ws_get(ctx, slot, bytes, &d));
    CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s), "copy input to device");
    o->dev = d;
    o->host = true;
    return BMLP_OK;
}

struct OutView {
    void* dev = nullptr;
    void* host = nullptr;
    size_t bytes = 0;
};

bmlp_status stage_out(bmlp_ctx* ctx, void* p, size_t bytes, int slot, OutView* o) {
    o->bytes = bytes;
    if (is_device_ptr(p)) {
        o->dev = p;
        o->host = nullptr;
        return BMLP_OK;
    }
    void* d = nullptr;
    ST(ws_get(ctx, slot, bytes, &d));
    o->dev = d;
    o->host = p;
    return BMLP_OK;
}

bmlp_status finish_out(bmlp_ctx* ctx, const OutView& o, cudaStream_t s) {
    if (o.host) {
        CK(cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, s), "copy output to host");
        CK(host_sync(ctx, s), "synchronise output copy");
    }
    return BMLP_OK;
}

long long wait_cycles(bmlp_ctx* ctx, const bmlp_options& o) {
    const int khz = ctx->clock_khz > 0 ? ctx->clock_khz : 2100000;
    const double ns = o.timeout_ns ? static_cast<double>(o.timeout_ns) : 2.0e9;
    return static_cast<long long>(ns * static_cast<double>(khz) * 1e-6);
}

int log2_ceil(int64_t n) {
    int k = 0;
    while ((int64_t(1) << k) < n) ++k;
    return k;
}

// Reads the control words after one iteration; maps device error words.
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Start of a call: clock for the time budget, all control words cleared.
bmlp_status begin_call(bmlp_ctx* ctx, const bmlp_options& o, cudaStream_t s) {
    ctx->t_call = now_s();
    ctx->budget_ns = o.budget_ns;
    CK(cudaMemsetAsync(ctx->d_ctl, 0, CTL_WORDS * sizeof(int), s), "reset flags");
    return BMLP_OK;
}

Deadline deadline_of(bmlp_ctx* ctx) {
    return Deadline{ctx->budget_ns, reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_T0),
                    ctx->d_ctl + CTL_BUDGET};
}

bmlp_status read_ctl(bmlp_ctx* ctx, cudaStream_t s, int* changed) {
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, CTL_WORDS * sizeof(int), cudaMemcpyDeviceToHost, s), "read flags");
    CK(host_sync(ctx, s), "synchronise iteration");
    if (ctx->h_ctl[CTL_ERROR] != 0)
        return set_err(ctx, BMLP_ERR_TIMEOUT, "in-kernel wait timed out (code 0x%x)", ctx->h_ctl[CTL_ERROR]);
    if (ctx->budget_ns &&
        (ctx->h_ctl[CTL_BUDGET] != 0 || (now_s() - ctx->t_call) * 1e9 > static_cast<double>(ctx->budget_ns)))
        return set_err(ctx, BMLP_ERR_BUDGET, "time budget of %.3f ms used up", ctx->budget_ns * 1e-6);
    if (changed) *changed = ctx->h_ctl[CTL_CHANGED];
    return BMLP_OK;
}

struct ProductTimer {
    bmlp_ctx* ctx;
    bool on;
    cudaStream_t s;
    double* sink = nullptr;  // where collect() adds the time (default: stats.product_ms)
    bmlp_status begin() {
        if (on) CK(cudaEventRecord(ctx->ev[0], s), "event record");
        return BMLP_OK;
    }
    bmlp_status end() {
        if (on) CK(cudaEventRecord(ctx->ev[1], s), "event record");
        return BMLP_OK;
    }
    bmlp_status collect() {  // after the stream was synchronised
        if (!on) return BMLP_OK;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]), "event elapsed");
        *(sink ? sink : &ctx->stats.product_ms) += ms;
        return BMLP_OK;
    }
};

// 4-bit tensor-core closures try squarings restricted to the rows and columns that hold zeros unless BMLP_THIN=0.
bool thin_enabled() {
    static const bool on = [] {
        const char* v = getenv("BMLP_THIN");
        return !(v && v[0] == '0');
    }();
    return on;
}

// Full frontier closures whose first squaring widens the rows run 64 sources per CTA (bit-sliced) unless
// BMLP_SMP_SLICED=0.
bool smp_sliced_enabled() {
    static const bool on = [] {
        const char* v = getenv("BMLP_SMP_SLICED");
        return !(v && v[0] == '0');
    }();
    return on;
}

// Smallest n that a grouped batch hands to the single-problem path (BMLP_BATCH_SOLO_N, 0 = never).
int64_t batch_solo_n() {
    static const int64_t v = [] {
        const char* e = getenv("BMLP_BATCH_SOLO_N");
        return e ? static_cast<int64_t>(atoll(e)) : int64_t(4096);
    }();
    return v;
}

// K-block skipping by the block-occupancy map of R, unless BMLP_TC_SKIP=0.
bool tc_skip_enabled() {
    static const bool on = [] {
        const char* v = getenv("BMLP_TC_SKIP");
        return !(v && v[0] == '0');
    }();
    return on;
}

// ------------------------------------------------------------------------
// Tensor-core squaring fixpoint on E4M3 R / R^T buffers already encoded in
// (M[0], T[0]). On return *res points at the buffer holding R1+ (and *res_t at
// its transpose). With res_f4 set, the caller has instead encoded R / R^T as
// packed E2M1 into the halves of M[1] / T[1]; every squaring then runs on
// 4-bit operands and *res_f4 receives the E2M1 result (row stride n_pad / 2);
// the squarings also keep R as bit rows, and *res_bits receives them (n_pad
// rows of n_pad / 64 words), or null if no squaring ran.
bmlp_status rms_tc_loop(bmlp_ctx* ctx, int64_t n, int64_t n_pad, uint8_t* M[2], uint8_t* T[2], int max_iters,
                        const bmlp_options& o, cudaStream_t s, int* iters, uint8_t** res, uint8_t** res_t,
                        const uint8_t** res_f4 = nullptr, const uint64_t** res_bits = nullptr) {
    NvtxRange nvtx_("tensor-core squarings");
    CUtensorMap mapA[2], mapB[2], mapBh[2];
    for (int b = 0; b < 2; ++b) {
        ST(make_tmap(ctx, &mapA[b], M[b], n_pad, n_pad, n_pad, TC_BM));
        ST(make_tmap(ctx, &mapB[b], T[b], n_pad, n_pad, n_pad, TC_BN));
        ST(make_tmap(ctx, &mapBh[b], T[b], n_pad, n_pad, n_pad, TC_BN / 2));
    }
    TcParams p{};
    p.m_tiles = static_cast<int32_t>(n_pad / TC_BM);
    p.n_tiles = static_cast<int32_t>(n_pad / TC_BN);
    p.k_blocks = static_cast<int32_t>(n_pad / TC_BK);
    p.mode = TC_MODE_RMS;
    p.ld = n_pad;
    p.changed = ctx->d_ctl + CTL_CHANGED;
    p.error = ctx->d_ctl + CTL_ERROR;
    p.wait_cycles = wait_cycles(ctx, o);
    const int tiles = p.m_tiles * p.n_tiles;
    const int grid = tiles < ctx->sm_count ? tiles : ctx->sm_count;
    // 128 x 128 block-occupancy maps of R (this iteration's and the next): K blocks whose A or B^T block
    // is empty are skipped, which removes most of the work of the early, block-sparse squarings
    // (maps F[b] and their transposes FT[b], rows padded to fm_ld bytes; up to 256 x 256 blocks)
    uint8_t* F[2] = {nullptr, nullptr};
    uint8_t* FT[2] = {nullptr, nullptr};
    p.fm_ld = static_cast<int32_t>(round_up(p.k_blocks, 16));
    const size_t fbytes = static_cast<size_t>(p.k_blocks) * static_cast<size_t>(p.fm_ld);
    if (tc_skip_enabled() && p.k_blocks <= 256 && res_f4 == nullptr) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        ST(ws_get(ctx, WS_F0, 2 * fbytes, &f0));
        ST(ws_get(ctx, WS_F1, 2 * fbytes, &f1));
        F[0] = static_cast<uint8_t*>(f0);
        FT[0] = F[0] + fbytes;
        F[1] = static_cast<uint8_t*>(f1);
        FT[1] = F[1] + fbytes;
        CK(cudaMemsetAsync(F[0], 0, 2 * fbytes, s), "clear block map");
        launch_block_flags(M[0], n_pad, n_pad, n_pad, F[0], s, p.fm_ld);
        launch_block_flags(T[0], n_pad, n_pad, n_pad, FT[0], s, p.fm_ld);
        CK(cudaGetLastError(), "block map");
        ctx->stats.launches += 2;
    }
    // Skipping pays only while many blocks are empty; R only gains bits, so once the map is dense it stays
    // dense and the maps are dropped for the rest of the closure.
    std::vector<uint8_t> hmap;
    auto sparse_map = [&](const uint8_t* dmap, bool* sparse) -> bmlp_status {
        hmap.resize(fbytes);
        CK(cudaMemcpyAsync(hmap.data(), dmap, fbytes, cudaMemcpyDeviceToHost, s), "read block map");
        CK(host_sync(ctx, s), "read block map");
        size_t nz = 0;
        for (size_t i = 0; i < fbytes; ++i) nz += hmap[i] != 0;
        *sparse = static_cast<double>(nz) < kSkipMaxDensity * double(p.k_blocks) * double(p.k_blocks);
        return BMLP_OK;
    };
    bool use_maps = false;
    if (F[0] != nullptr) ST(sparse_map(F[0], &use_maps));
    ProductTimer tm{ctx, o.profile != 0, s};
    p.issued = reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_ISSUED);
    CK(cudaMemsetAsync(p.issued, 0, sizeof(unsigned long long), s), "reset issued counter");
    // Once R is dense, the squarings continue on packed E2M1 operands (half the bytes per Boolean operation):
    // R, R^T are converted into the halves of the free E4M3 buffer pair (index sw ^ 1) and ping-pong there;
    // the result is converted back into the E4M3 pair sw.
    const bool fp4 = o.e4m3_only == 0;
    bool on_f4 = false;
    int sw = 0, qcur = 0;
    uint8_t* Q[2] = {nullptr, nullptr};
    uint8_t* QT[2] = {nullptr, nullptr};
    CUtensorMap mapA4[2], mapB4[2], mapB4x[2];
    const int64_t ld4 = n_pad / 2;
    auto finish_f4 = [&](uint8_t** r, uint8_t** rt) -> bmlp_status {
        launch_e2m1_to_e4m3(Q[qcur], M[sw], n_pad * n_pad, s);
        launch_e2m1_to_e4m3(QT[qcur], T[sw], n_pad * n_pad, s);
        CK(cudaGetLastError(), "E2M1 decode");
        ctx->stats.launches += 2;
        *r = M[sw];
        *rt = T[sw];
        return BMLP_OK;
    };
    // Once a 4-bit squaring has run, the next one is first sized on the rows and columns of R that still hold
    // zeros (thin.cu); when those hold few ones, it runs there, on bit rows, at a fraction of a dense product.
    const int64_t ldw_t = n_pad / 64;
    const bool thin_on = !o.tc_only && thin_enabled() && thin_fixed_s(n_pad) < tc4_product_s(n_pad);
    bool thin_try = false;  // the last 4-bit squaring left R dense enough (sampled) to size the next one
    // bit rows of R and R^T (n_pad rows each): written by every 4-bit squaring's epilogue when the caller takes the
    // result from them (res_bits), kept by the restricted squarings; bits_current once a squaring has written them
    uint64_t* P = nullptr;
    uint64_t* PT = nullptr;
    bool bits_current = false;
    if (thin_on || res_bits != nullptr) {
        void* pp = nullptr;
        ST(ws_get(ctx, WS_THIN_P, static_cast<size_t>(2 * n_pad * ldw_t * 8), &pp));
        P = static_cast<uint64_t*>(pp);
        PT = P + n_pad * ldw_t;
    }
    if (res_bits != nullptr) *res_bits = nullptr;
    auto thin_step = [&](bool* ran, int* changed) -> bmlp_status {
        *ran = false;
        void* aux = nullptr;
        const size_t aux_bytes = static_cast<size_t>(2 * n * 8 + (ldw_t + 1) * 8 + 2 * n * 4);
        ST(ws_get(ctx, WS_THIN_AUX, aux_bytes, &aux));
        int64_t* rowcnt = static_cast<int64_t*>(aux);
        int64_t* colcnt = rowcnt + n;
        uint64_t* Bmask = reinterpret_cast<uint64_t*>(colcnt + n);
        int32_t* blist = reinterpret_cast<int32_t*>(Bmask + ldw_t + 1);
        int32_t* rlist = blist + n;
        auto* stat = reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_THIN);
        CK(launch_thin_stats(Q[qcur], QT[qcur], ld4, n, P, PT, ldw_t, rowcnt, colcnt, Bmask, blist, rlist, stat,
                             bits_current, ctx->sm_count, s),
           "thin squaring statistics");
        bits_current = true;  // P, PT hold R, R^T from here on (converted, or already there)
        ctx->stats.launches += 4;
        ST(read_ctl(ctx, s, nullptr));
        unsigned long long st[6];
        memcpy(st, ctx->h_ctl + CTL_THIN, sizeof(st));
        // the word ORs over the GPU, or one warp's list entry with the most ones, whichever takes longer
        const double words = static_cast<double>(st[2] + st[3]) * static_cast<double>(ldw_t);
        const double row_words = static_cast<double>(st[4] > st[5] ? st[4] : st[5]) * static_cast<double>(ldw_t);
        const double t = thin_fixed_s(n_pad) + std::max(words * bitrow_s_per_word(), row_words * bitrow_row_s_per_word());
        if (t >= tc4_product_s(n_pad)) return BMLP_OK;
        const int64_t nb = static_cast<int64_t>(st[0]), nr = static_cast<int64_t>(st[1]);
        void* tt = nullptr;
        ST(ws_get(ctx, WS_THIN_T, static_cast<size_t>((nb + nr + 1) * ldw_t * 8), &tt));
        uint64_t* T1 = static_cast<uint64_t*>(tt);
        CK(launch_thin_squaring(P, PT, ldw_t, blist, nb, rlist, nr, T1, T1 + nb * ldw_t, Q[qcur], QT[qcur], ld4,
                                ctx->d_ctl + CTL_CHANGED, ctx->sm_count, s),
           "thin squaring");
        ctx->stats.launches += 4;
        ctx->stats.thin_squarings++;
        ST(read_ctl(ctx, s, changed));
        *ran = true;
        return BMLP_OK;
    };
    int cur = 0;
    *iters = 0;
    if (res_f4 != nullptr) {
        // the caller encoded R, R^T as packed E2M1 into the halves of M[1], T[1]: 4-bit squarings from the start
        const size_t half = static_cast<size_t>(n_pad) * static_cast<size_t>(ld4);
        sw = 0;
        Q[0] = M[1];
        Q[1] = M[1] + half;
        QT[0] = T[1];
        QT[1] = T[1] + half;
        for (int b = 0; b < 2; ++b) {
            ST(make_tmap(ctx, &mapA4[b], Q[b], n_pad, ld4, ld4, TC_BM));
            ST(make_tmap(ctx, &mapB4[b], QT[b], n_pad, ld4, ld4, TC_BN / 2));
            ST(make_tmap(ctx, &mapB4x[b], QT[b], n_pad, ld4, ld4, tc4_b1_rows()));
        }
        on_f4 = true;
        qcur = 0;
    }
    for (int it = 0; it < max_iters; ++it) {
        const int nxt = cur ^ 1;
        CK(cudaMemsetAsync(ctx->d_ctl, 0, 2 * sizeof(int), s), "reset flags");
        if (fp4 && !use_maps && !on_f4) {
            sw = cur;
            const size_t half = static_cast<size_t>(n_pad) * static_cast<size_t>(ld4);
            Q[0] = M[nxt];
            Q[1] = M[nxt] + half;
            QT[0] = T[nxt];
            QT[1] = T[nxt] + half;
            launch_e4m3_to_e2m1(M[cur], Q[0], n_pad * n_pad, s);
            launch_e4m3_to_e2m1(T[cur], QT[0], n_pad * n_pad, s);
            CK(cudaGetLastError(), "E2M1 encode");
            ctx->stats.launches += 2;
            for (int b = 0; b < 2; ++b) {
                ST(make_tmap(ctx, &mapA4[b], Q[b], n_pad, ld4, ld4, TC_BM));
                ST(make_tmap(ctx, &mapB4[b], QT[b], n_pad, ld4, ld4, TC_BN / 2));
                ST(make_tmap(ctx, &mapB4x[b], QT[b], n_pad, ld4, ld4, tc4_b1_rows()));
            }
            on_f4 = true;
            qcur = 0;
        }
        if (on_f4 && thin_try) {
            bool ran = false;
            int changed = 0;
            ST(thin_step(&ran, &changed));
            if (ran) {
                *iters = it + 1;
                if (!changed) {  // R is its closure; Q[qcur], QT[qcur] hold it
                    if (res_f4 != nullptr) {
                        *res_f4 = Q[qcur];
                        if (res_bits != nullptr && bits_current) *res_bits = P;
                        *res = *res_t = nullptr;
                        return BMLP_OK;
                    }
                    return finish_f4(res, res_t);
                }
                continue;
            }
        }
        if (on_f4) {
            TcParams p4 = p;
            p4.ld = ld4;
            p4.k_blocks = static_cast<int32_t>(n_pad / 256);
            p4.n_tiles = static_cast<int32_t>((n_pad + tc4_tile_n() - 1) / tc4_tile_n());
            p4.fmap = p4.fmapT = p4.fmap_next = p4.fmapT_next = nullptr;
            p4.old_r = Q[qcur];
            p4.out_r = Q[qcur ^ 1];
            p4.out_rt = QT[qcur ^ 1];
            // the epilogue writes the bit rows too when the result leaves from them, or a restricted squaring may
            // follow (which then needs no conversion from E2M1)
            const bool bits_out = P != nullptr && (res_bits != nullptr || thin_on);
            if (bits_out) {
                p4.out_bits = reinterpret_cast<uint32_t*>(P);
                p4.out_bits_t = reinterpret_cast<uint32_t*>(PT);
                p4.ldb = 2 * ldw_t;
            }
            ST(tm.begin());
            CK(launch_tc4_product_duo(mapA4[qcur], mapB4[qcur], mapB4x[qcur], p4, ctx->sm_count, s),
               "tensor-core product launch");
            ST(tm.end());
            ctx->stats.product_launches++;
            ctx->stats.e2m1_products++;
            ctx->stats.launches += 2;
            bits_current = bits_out;
            auto* sample = reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_THIN) + 6;
            if (thin_on) {
                // whether the rows of the new R that reach most constants are saturated (a sample of 256 rows),
                // read back with the changed flag
                CK(cudaMemsetAsync(sample, 0, 2 * sizeof(unsigned long long), s), "reset row sample");
                CK(launch_thin_sample(Q[qcur ^ 1], ld4, n, kThinSampleRows, sample, s), "row sample");
                ctx->stats.launches++;
            }
            int changed = 0;
            ST(read_ctl(ctx, s, &changed));
            ST(tm.collect());
            unsigned long long kbs = 0;
            memcpy(&kbs, ctx->h_ctl + CTL_ISSUED, sizeof(kbs));
            ctx->stats.issued_ops = 2.0 * TC_BM * 32.0 * TC_BK * static_cast<double>(kbs);
            *iters = it + 1;
            qcur ^= 1;
            if (!changed) {
                if (res_f4 != nullptr) {
                    *res_f4 = Q[qcur];
                    if (res_bits != nullptr && bits_current) *res_bits = P;
                    *res = *res_t = nullptr;
                    return BMLP_OK;
                }
                return finish_f4(res, res_t);
            }
            if (thin_on) {
                // every zero of a row that reaches most constants must lie in the few columns of B: such rows have
                // (nearly) the same count
                unsigned long long smp[2];
                memcpy(smp, ctx->h_ctl + CTL_THIN + 12, sizeof(smp));
                const double spread = static_cast<double>(smp[0]) - (static_cast<double>(n) - static_cast<double>(smp[1]));
                thin_try = smp[0] > 0 && spread <= kThinRowSpread * static_cast<double>(n);
            }
            continue;
        }
        if (use_maps) {
            CK(cudaMemsetAsync(F[nxt], 0, 2 * fbytes, s), "clear block map");
            p.fmap = F[cur];
            p.fmapT = FT[cur];
            p.fmap_next = F[nxt];
            p.fmapT_next = FT[nxt];
        } else {
            p.fmap = p.fmapT = nullptr;
            p.fmap_next = p.fmapT_next = nullptr;
        }
        p.old_r = M[cur];
        p.out_r = M[nxt];
        p.out_rt = T[nxt];
        ST(tm.begin());
        if (use_maps) {
            // block-sparse R: one CTA per SM, empty K blocks skipped, block maps of the new R
            CK(launch_tc_product(mapA[cur], mapB[cur], p, grid, s), "tensor-core product launch");
        } else {
            // dense R on E4M3 operands: M = 256 MMAs per CTA pair on 256 x 512 pair tiles
            TcParams p8 = p;
            p8.n_tiles = static_cast<int32_t>((n_pad + tc8_tile_n() - 1) / tc8_tile_n());
            CK(launch_tc8_product_duo(mapA[cur], mapBh[cur], p8, ctx->sm_count, s), "tensor-core product launch");
        }
        ST(tm.end());
        ctx->stats.product_launches++;
        ctx->stats.launches += 2;
        int changed = 0;
        ST(read_ctl(ctx, s, &changed));
        ST(tm.collect());
        // multiply-adds actually issued (units of 128 x 32 x 128), times 2
        unsigned long long kbs = 0;
        memcpy(&kbs, ctx->h_ctl + CTL_ISSUED, sizeof(kbs));
        ctx->stats.issued_ops = 2.0 * TC_BM * 32.0 * TC_BK * static_cast<double>(kbs);
        *iters = it + 1;
        cur = nxt;
        if (!changed) {
            *res = M[cur];
            *res_t = T[cur];
            return BMLP_OK;
        }
        if (use_maps) ST(sparse_map(F[cur], &use_maps));
    }
    if (on_f4 && res_f4 != nullptr) {
        *res_f4 = Q[qcur];
        if (res_bits != nullptr && bits_current) *res_bits = P;
        *res = *res_t = nullptr;
    } else if (on_f4) {
        ST(finish_f4(res, res_t));
    } else {
        *res = M[cur];
        *res_t = T[cur];
    }
    return set_err(ctx, BMLP_ERR_NOT_CONVERGED, "no fixpoint within %d products", max_iters);
}

// Device scratch for the prefix of a word-index build (kScanMaxChunks x 2 words).
int64_t* scan_scratch(bmlp_ctx* ctx) {
    void* p = nullptr;
    return ws_get(ctx, WS_SCAN, static_cast<size_t>(kScanMaxChunks) * 2 * sizeof(int64_t), &p) == BMLP_OK
               ? static_cast<int64_t*>(p)
               : nullptr;
}

// Packed squaring fixpoint on P[0] (n rows x ldw words). *res = R1+. While fewer than half of R's words are
// nonzero a squaring runs through R's word index (square_rows_kernel: only the nonzero words of the named rows are
// ORed in, and the step streams R in and R' out), after that as the whole-row product (product_packed_kernel); a
// squaring that widens the rows past half their words hands the next ones to the whole-row product.
bmlp_status rms_packed_loop(bmlp_ctx* ctx, int64_t n, int64_t ldw, uint64_t* P[2], int max_iters,
                            const bmlp_options& o, cudaStream_t s, int* iters, uint64_t** res) {
    ProductTimer tm{ctx, o.profile != 0, s};
    void *wptr = nullptr, *widx = nullptr, *wval = nullptr;
    ST(ws_get(ctx, WS_WPTR, static_cast<size_t>((n + 2) * 8), &wptr));
    ST(ws_get(ctx, WS_WIDX, static_cast<size_t>(n * ldw * 4), &widx));
    ST(ws_get(ctx, WS_WVAL, static_cast<size_t>(n * ldw * 8), &wval));
    const bool index_fits = ldw * 8 <= 200 * 1024;  // square_rows_kernel assembles a row in shared memory
    bool sparse = index_fits;
    auto index_of = [&](const uint64_t* Pm) -> bmlp_status {
        CK(launch_wcsr_build(Pm, n, ldw, static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx),
                             static_cast<uint64_t*>(wval), s, scan_scratch(ctx)),
           "word index build");
        CK(cudaMemcpyAsync(ctx->h_ctl + CTL_HOST_I64, static_cast<const int64_t*>(wptr) + n, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s),
           "read word count");
        ctx->stats.launches += 3;
        return BMLP_OK;
    };
    auto half_full = [&]() {
        int64_t W = 0;
        memcpy(&W, ctx->h_ctl + CTL_HOST_I64, sizeof(W));
        return 2 * W >= n * ldw;
    };
    int cur = 0;
    *iters = 0;
    if (sparse) {
        ST(index_of(P[0]));
        CK(host_sync(ctx, s), "read word count");
        sparse = !half_full();
    }
    // ones and nonzero words of the current R, counted by the whole-row step that wrote it (-1: not counted, as
    // after a word-indexed step)
    auto* pstat = reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_PSTAT);
    int64_t ones = -1, words = -1;
    for (int it = 0; it < max_iters; ++it) {
        const int nxt = cur ^ 1;
        CK(cudaMemsetAsync(ctx->d_ctl, 0, 2 * sizeof(int), s), "reset flags");
        CK(cudaMemsetAsync(pstat, 0, 2 * sizeof(unsigned long long), s), "reset counts");
        ST(tm.begin());
        if (sparse) {
            CK(launch_square_rows(static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx),
                                  static_cast<uint64_t*>(wval), P[cur], n, ldw, P[nxt], ctx->sm_count, s,
                                  ctx->d_ctl + CTL_CHANGED),
               "word-indexed squaring launch");
            ctx->stats.sparse_squarings++;
        } else {
            // whole rows: the Four Russians tables once the nonzero words of R carry many bits (their cost does not
            // depend on the bits; gathering the named rows costs one row of R per one)
            const bool tables = ones < 0 || static_cast<double>(ones) >= kM4MinBitsPerWord * static_cast<double>(words);
            CK(launch_product_packed(P[cur], P[cur], P[nxt], n, ldw, 1, ctx->d_ctl + CTL_CHANGED, ctx->sm_count, s,
                                     deadline_of(ctx), pstat, tables),
               "packed product launch");
            if (tables) ctx->stats.table_squarings++;
        }
        ST(tm.end());
        ctx->stats.product_launches++;
        ctx->stats.launches += 2;
        if (sparse) ST(index_of(P[nxt]));  // the next step's index, read back with the flag
        int changed = 0;
        ST(read_ctl(ctx, s, &changed));
        ST(tm.collect());
        if (sparse) {
            ones = words = -1;
        } else {
            unsigned long long cnt[2];
            memcpy(cnt, ctx->h_ctl + CTL_PSTAT, sizeof(cnt));
            ones = static_cast<int64_t>(cnt[0]);
            words = static_cast<int64_t>(cnt[1]);
        }
        *iters = it + 1;
        cur = nxt;
        if (!changed) {
            *res = P[cur];
            return BMLP_OK;
        }
        if (sparse) sparse = !half_full();
    }
    *res = P[cur];
    return set_err(ctx, BMLP_ERR_NOT_CONVERGED, "no fixpoint within %d products", max_iters);
}

// Whether R (format fmt; packed rows of ldw words) is dense by its 128 x 128 block map: then a closure starts on
// 4-bit operands and leaves from them, else on E4M3 with empty K blocks skipped.
bmlp_status dense_by_blocks(bmlp_ctx* ctx, const Operand& src, int32_t fmt, int64_t ldw, int64_t n, int64_t n_pad,
                            cudaStream_t s, bool* dense) {
    const int64_t kb = n_pad / 128;
    *dense = !tc_skip_enabled() || kb > 256;
    if (*dense) return BMLP_OK;
    void* f = nullptr;
    ST(ws_get(ctx, WS_F0, static_cast<size_t>(kb * kb), &f));
    launch_input_block_flags(src.dev, fmt, ldw, n, n_pad, static_cast<uint8_t*>(f), kb, s);
    CK(cudaGetLastError(), "input block map");
    ctx->stats.launches++;
    std::vector<uint8_t> h(static_cast<size_t>(kb * kb));
    CK(cudaMemcpyAsync(h.data(), f, h.size(), cudaMemcpyDeviceToHost, s), "read input block map");
    CK(host_sync(ctx, s), "read input block map");
    size_t nz = 0;
    for (uint8_t x : h) nz += x != 0;
    *dense = static_cast<double>(nz) >= kSkipMaxDensity * static_cast<double>(kb * kb);
    return BMLP_OK;
}

// The caller's rows themselves when they are packed bit rows on the device with ldw words per row (words_of(n) even),
// no padding bits (n a multiple of 64: a caller's bits at columns >= n are to be ignored, and the copy clears them)
// and 16-byte aligned, so that a read-only pass can use them without a copy; else null.
const uint64_t* in_place_packed(const Operand& in, int32_t fmt, int64_t n, int64_t ldw) {
    if (fmt != BMLP_FMT_PACKED64 || in.host || words_of(n) != ldw || n % 64 != 0) return nullptr;
    if ((reinterpret_cast<uintptr_t>(in.dev) & 15) != 0) return nullptr;
    return static_cast<const uint64_t*>(in.dev);
}

// Packed copy of a caller matrix (any format) into n x ldw words.
bmlp_status to_packed(bmlp_ctx* ctx, const Operand& in, int32_t fmt, int64_t n, uint64_t* P, int64_t ldw,
                      cudaStream_t s) {
    if (fmt == BMLP_FMT_U8)
        launch_u8_to_packed(static_cast<const uint8_t*>(in.dev), n, P, ldw, s);
    else
        launch_packed_copy(static_cast<const uint64_t*>(in.dev), words_of(n), n, n, P, ldw, 0, s);
    ctx->stats.launches++;
    CK(cudaGetLastError(), "encode launch");
    return BMLP_OK;
}

// E4M3 R and R^T (n_pad) of a caller matrix (packed rows of ldw_in words; 0 = ceil(n / 64)).
bmlp_status to_e4m3(bmlp_ctx* ctx, const Operand& in, int32_t fmt, int64_t n, uint8_t* R, uint8_t* RT, int64_t n_pad,
                    cudaStream_t s, int64_t ldw_in = 0) {
    if (fmt == BMLP_FMT_U8)
        launch_u8_to_e4m3(static_cast<const uint8_t*>(in.dev), n, R, RT, n_pad, s);
    else
        launch_packed_to_e4m3(static_cast<const uint64_t*>(in.dev), ldw_in > 0 ? ldw_in : words_of(n), n, n, R, RT,
                              n_pad, n_pad, s);
    ctx->stats.launches++;
    CK(cudaGetLastError(), "encode launch");
    return BMLP_OK;
}

bmlp_status bytes_out(bmlp_ctx* ctx, const uint8_t* R, int64_t ld, int64_t n, int32_t fmt, void* out, int reflexive,
                      cudaStream_t s) {
    if (fmt == BMLP_FMT_U8)
        launch_bytes_to_u8(R, ld, n, static_cast<uint8_t*>(out), reflexive, s);
    else
        launch_bytes_to_packed(R, ld, n, n, static_cast<uint64_t*>(out), words_of(n), reflexive, s);
    ctx->stats.launches++;
    CK(cudaGetLastError(), "decode launch");
    return BMLP_OK;
}

bmlp_status packed_out(bmlp_ctx* ctx, const uint64_t* P, int64_t ldw, int64_t n, int32_t fmt, void* out, int reflexive,
                       cudaStream_t s) {
    if (fmt == BMLP_FMT_U8)
        launch_packed_to_u8(P, ldw, n, static_cast<uint8_t*>(out), reflexive, s);
    else
        launch_packed_copy(P, ldw, n, n, static_cast<uint64_t*>(out), words_of(n), reflexive, s);
    ctx->stats.launches++;
    CK(cudaGetLastError(), "decode launch");
    return BMLP_OK;
}

// ---- engine switch inside one closure (squaring on bit rows, then on the tensor cores)
// Smallest n whose tensor-core closures start on bit rows: below it a tensor-core product takes microseconds and
// the word index, the cost pass and one host round trip per step cost more than they save.
constexpr int64_t kSparseMinN = 4096;
// Fixed device and host time of one bit-row step besides its word ORs: word index, cost pass, flag read-back.
constexpr double kSparseStepS = 20e-6;

// Device seconds per word OR of square_rows_kernel over the whole GPU, and per word OR of the one warp that
// assembles a row (BMLP_SPARSE_PS_PER_WORD / BMLP_SPARSE_ROW_PS_PER_WORD in picoseconds override them).
double sparse_s_per_word() {
    static const double v = [] {
        const char* e = getenv("BMLP_SPARSE_PS_PER_WORD");
        return (e ? atof(e) : 10.0) * 1e-12;
    }();
    return v;
}
double sparse_row_s_per_word() {
    static const double v = [] {
        const char* e = getenv("BMLP_SPARSE_ROW_PS_PER_WORD");
        return (e ? atof(e) : 10000.0) * 1e-12;
    }();
    return v;
}

// Device seconds of one dense tensor-core squaring of an n_pad x n_pad matrix (2 n_pad^3 Boolean multiply-adds at
// the 4-bit kernel's measured rate, plus launch and flag read-back).
double tc_product_s(int64_t n_pad) {
    const double n3 = static_cast<double>(n_pad) * static_cast<double>(n_pad) * static_cast<double>(n_pad);
    return 2.0 * n3 / 7.0e15 + 20e-6;
}

struct SparseStart {
    uint64_t* P = nullptr;  // packed rows after the squarings on bit rows (nullptr: none ran)
    int64_t ldw = 0;
    int iters = 0;          // squarings run on bit rows
    bool done = false;      // the last of them changed nothing: P is the closure
};

// Squarings R <- R + R R on word-indexed bit rows (square_rows_kernel) for as long as the next one costs less than a
// tensor-core product. Each step is the squaring the tensor cores would run, so the fixpoint and the count of
// products are the same (R_k covers the paths of length 1 .. 2^k whichever engine squared it); the cost of a step is
// the word ORs it will issue, summed on the GPU from the word index, and only grows as R gains bits, so the switch
// goes one way. Leaves at least one product to the caller's loop unless the fixpoint was reached here.
bmlp_status sparse_squarings(bmlp_ctx* ctx, const Operand& in, int32_t fmt, int64_t n, int64_t n_pad, int max_iters,
                             const bmlp_options& o, cudaStream_t s, SparseStart* out) {
    NvtxRange nvtx_("bit-row squarings");
    const int64_t ldw = round_up(words_of(n), 2);
    if (n < kSparseMinN || ldw > 2048 || max_iters < 2) return BMLP_OK;
    void *pa = nullptr, *pb = nullptr, *wptr = nullptr, *widx = nullptr, *wval = nullptr;
    ST(ws_get(ctx, WS_SQP, static_cast<size_t>(n * ldw * 8), &pa));
    ST(ws_get(ctx, WS_PT, static_cast<size_t>(n * ldw * 8), &pb));
    ST(ws_get(ctx, WS_SQPTR, static_cast<size_t>((n + 2) * 8), &wptr));
    ST(ws_get(ctx, WS_SQIDX, static_cast<size_t>(n * ldw * 4), &widx));
    ST(ws_get(ctx, WS_SQVAL, static_cast<size_t>(n * ldw * 8), &wval));
    uint64_t* P[2] = {static_cast<uint64_t*>(pa), static_cast<uint64_t*>(pb)};
    // the first pass reads the caller's rows in place when they already have this layout (never written)
    const uint64_t* R0 = in_place_packed(in, fmt, n, ldw);
    if (R0 == nullptr) {
        ST(to_packed(ctx, in, fmt, n, P[0], ldw, s));
        R0 = P[0];
    }
    auto* cost = reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_COST);
    const double limit = tc_product_s(n_pad);
    ProductTimer tm{ctx, o.profile != 0, s, &ctx->stats.sparse_ms};
    int cur = 0;
    for (;;) {
        const uint64_t* Rc = out->iters == 0 ? R0 : P[cur];
        CK(launch_wcsr_build(Rc, n, ldw, static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx),
                             static_cast<uint64_t*>(wval), s, scan_scratch(ctx)),
           "word index build");
        CK(cudaMemsetAsync(cost, 0, 2 * sizeof(unsigned long long), s), "reset cost");
        CK(launch_square_cost(static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx), static_cast<uint64_t*>(wval),
                              n, cost, ctx->sm_count, s),
           "squaring cost launch");
        ctx->stats.launches += 4;
        int changed = 1;
        ST(read_ctl(ctx, s, &changed));
        if (out->iters > 0) ST(tm.collect());  // the squaring recorded in the previous pass
        if (out->iters > 0 && !changed) {
            out->done = true;
            break;
        }
        unsigned long long words = 0, row_words = 0;
        memcpy(&words, ctx->h_ctl + CTL_COST, sizeof(words));
        memcpy(&row_words, ctx->h_ctl + CTL_COST + 2, sizeof(row_words));
        const double t = kSparseStepS + std::max(static_cast<double>(words) * sparse_s_per_word(),
                                                 static_cast<double>(row_words) * sparse_row_s_per_word());
        if (out->iters + 1 >= max_iters || t > limit) break;
        CK(cudaMemsetAsync(ctx->d_ctl + CTL_CHANGED, 0, sizeof(int), s), "reset flag");
        ST(tm.begin());
        CK(launch_square_rows(static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx), static_cast<uint64_t*>(wval),
                              Rc, n, ldw, P[cur ^ 1], ctx->sm_count, s, ctx->d_ctl + CTL_CHANGED),
           "squaring launch");
        ST(tm.end());
        ctx->stats.launches++;
        ctx->stats.sparse_squarings++;
        ctx->stats.sparse_words += static_cast<double>(words);
        out->iters++;
        cur ^= 1;
    }
    if (out->iters > 0) {
        out->P = P[cur];
        out->ldw = ldw;
    }
    return BMLP_OK;
}

// X = A B thresholded to 0/1 for packed E2M1 operands (A row-major, B given as B^T, both n_pad x n_pad / 2 bytes), on
// the 4-bit squaring kernel with a zero old R (Z, cleared here), so that its R' is the product; its R'^T goes to XT
// (scratch). Raises the call's error on an in-kernel timeout.
bmlp_status e2m1_product(bmlp_ctx* ctx, const uint8_t* A, const uint8_t* BT, int64_t n_pad, uint8_t* Z, uint8_t* X,
                         uint8_t* XT, const bmlp_options& o, cudaStream_t s) {
    const int64_t ld4 = n_pad / 2;
    CK(cudaMemsetAsync(Z, 0, static_cast<size_t>(n_pad) * static_cast<size_t>(ld4), s), "clear old R");
    CUtensorMap fa, fb0, fb1;
    ST(make_tmap(ctx, &fa, A, n_pad, ld4, ld4, TC_BM));
    ST(make_tmap(ctx, &fb0, BT, n_pad, ld4, ld4, TC_BN / 2));
    ST(make_tmap(ctx, &fb1, BT, n_pad, ld4, ld4, tc4_b1_rows()));
    TcParams pp{};
    pp.m_tiles = static_cast<int32_t>(n_pad / TC_BM);
    pp.n_tiles = static_cast<int32_t>((n_pad + tc4_tile_n() - 1) / tc4_tile_n());
    pp.k_blocks = static_cast<int32_t>(n_pad / 256);
    pp.mode = TC_MODE_RMS;
    pp.ld = ld4;
    pp.old_r = Z;
    pp.out_r = X;
    pp.out_rt = XT;
    pp.changed = ctx->d_ctl + CTL_CHANGED;
    pp.error = ctx->d_ctl + CTL_ERROR;
    pp.wait_cycles = wait_cycles(ctx, o);
    CK(launch_tc4_product_duo(fa, fb0, fb1, pp, ctx->sm_count, s), "4-bit product launch");
    ctx->stats.product_launches++;
    ctx->stats.e2m1_products++;
    ctx->stats.launches += 2;
    return read_ctl(ctx, s, nullptr);
}

// X = A B for E4M3 0/1 operands on the tensor cores: A row-major, B given as B^T (both n_pad x n_pad); one plain
// product (no OR with an old R) with exact FP32 counts thresholded to 0/1.
bmlp_status tc_plain_product(bmlp_ctx* ctx, const uint8_t* A, const uint8_t* BT, int64_t n_pad, uint8_t* X,
                             const bmlp_options& o, cudaStream_t s) {
    CUtensorMap mapA, mapB;
    ST(make_tmap(ctx, &mapA, A, n_pad, n_pad, n_pad, TC_BM));
    ST(make_tmap(ctx, &mapB, BT, n_pad, n_pad, n_pad, TC_BN));
    TcParams p{};
    p.m_tiles = static_cast<int32_t>(n_pad / TC_BM);
    p.n_tiles = static_cast<int32_t>(n_pad / TC_BN);
    p.k_blocks = static_cast<int32_t>(n_pad / TC_BK);
    p.mode = TC_MODE_PLAIN;
    p.ld = n_pad;
    p.out_r = X;
    p.changed = ctx->d_ctl + CTL_CHANGED;
    p.error = ctx->d_ctl + CTL_ERROR;
    p.wait_cycles = wait_cycles(ctx, o);
    const int tiles = p.m_tiles * p.n_tiles;
    CK(cudaMemsetAsync(ctx->d_ctl, 0, 2 * sizeof(int), s), "reset flags");
    CK(launch_tc_product(mapA, mapB, p, tiles < ctx->sm_count ? tiles : ctx->sm_count, s), "product launch");
    ctx->stats.product_launches++;
    ctx->stats.launches += 2;
    return read_ctl(ctx, s, nullptr);
}

bmlp_options resolve(const bmlp_options* o) {
    bmlp_options r;
    bmlp_default_options(&r);
    if (o) r = *o;
    return r;
}

void reset_stats(bmlp_ctx* ctx, int variant, int64_t n_pad) {
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.variant = variant;
    ctx->stats.n_pad = n_pad;
}

// Without a trained dispatcher the fixed choice is squaring on the tensor cores.
int pick_variant_rms(int64_t) { return BMLP_RMS_TC; }

// Frontier expansion (Algorithm 2) on packed rows for the sources `src`
// (device, q x ldw_src words). out: device, q x ldw_out words. square_first:
// a full closure (src = the identity, q = n), which may square R first
// (path-like R) or expand 64 sources at a time (rows that widen fast).
bmlp_status smp_packed_run(bmlp_ctx* ctx, const Operand& R, int32_t fmt, int64_t n, const uint64_t* src,
                           int64_t ldw_src, int64_t q, uint64_t* out, int64_t ldw_out, const bmlp_options& o,
                           cudaStream_t s, int* levels, bool square_first = false) {
    NvtxRange nvtx_("frontier expansion");
    const int64_t ldw = round_up(words_of(n), 2);
    if (ldw > smp_packed_max_words())
        return set_err(ctx, BMLP_ERR_UNSUPPORTED, "packed frontier path supports n <= %d", smp_packed_max_words() * 64);
    void *P = nullptr, *wptr = nullptr, *widx = nullptr, *wval = nullptr;
    ST(ws_get(ctx, WS_WPTR, static_cast<size_t>((n + 2) * 8), &wptr));
    ST(ws_get(ctx, WS_WIDX, static_cast<size_t>(n * ldw * 4), &widx));
    ST(ws_get(ctx, WS_WVAL, static_cast<size_t>(n * ldw * 8), &wval));
    if (!square_first && fmt == BMLP_FMT_PACKED64 && words_of(n) == ldw && n % 64 == 0) {
        // query rows: R is only read, so packed rows of the working width without padding bits are used where
        // they are
        P = const_cast<void*>(R.dev);
    } else {
        ST(ws_get(ctx, WS_M0, static_cast<size_t>(n * ldw * 8), &P));
        ST(to_packed(ctx, R, fmt, n, static_cast<uint64_t*>(P), ldw, s));
    }
    CK(launch_wcsr_build(static_cast<uint64_t*>(P), n, ldw, static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx),
                         static_cast<uint64_t*>(wval), s, scan_scratch(ctx)),
       "word index build");
    ctx->stats.launches += 3;
    // nonzero words of R (W) and of R + R R (W2, counted from the word index of R without forming R + R R)
    int64_t ones = -1;  // ones of the current R (with its word index), when a growth test has counted them
    auto growth = [&](int64_t* W, int64_t* W2) -> bmlp_status {
        auto* cnt = reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_COST);
        auto* bits = reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_BITS);
        CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s), "reset counts");
        CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s), "reset ones");
        CK(launch_square_growth(static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx),
                                static_cast<uint64_t*>(wval), n, ldw, cnt, ctx->sm_count, s, bits),
           "squaring growth launch");
        CK(cudaMemcpyAsync(ctx->h_ctl + CTL_HOST_I64, static_cast<const int64_t*>(wptr) + n, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s),
           "read word count");
        ST(read_ctl(ctx, s, nullptr));
        ctx->stats.launches++;
        unsigned long long w2 = 0, b = 0;
        memcpy(&w2, ctx->h_ctl + CTL_COST, sizeof(w2));
        memcpy(&b, ctx->h_ctl + CTL_BITS, sizeof(b));
        memcpy(W, ctx->h_ctl + CTL_HOST_I64, sizeof(int64_t));
        *W2 = static_cast<int64_t>(w2);
        ones = static_cast<int64_t>(b);
        return BMLP_OK;
    };
    bool dense_reach = false;
    if (square_first && n >= kSquareMinN && ldw <= 2048) {
        // Long shortest paths make the frontier latency-bound (one level per path step). closure(R + R R) =
        // closure(R) with half the levels, so R is squared while that keeps its rows within ~1.5x the nonzero
        // words (path-like structure); once the words grow faster, the frontier would pay more per level than
        // it saves in levels, and that squaring is not formed.
        for (int k = 0; k < kSquareMaxSteps; ++k) {
            int64_t W = 0, W2 = 0;
            ST(growth(&W, &W2));
            if (static_cast<double>(W2) > kSquareMaxGrowth * static_cast<double>(W)) {
                // the first squaring widens the rows fast: closure rows fill up within a few levels
                dense_reach = k == 0 && static_cast<double>(W2) > kSlicedMinGrowth * static_cast<double>(W);
                break;
            }
            void *P2 = nullptr, *wptr2 = nullptr, *widx2 = nullptr, *wval2 = nullptr;
            ST(ws_get(ctx, WS_SQP, static_cast<size_t>(n * ldw * 8), &P2));
            ST(ws_get(ctx, WS_SQPTR, static_cast<size_t>((n + 2) * 8), &wptr2));
            ST(ws_get(ctx, WS_SQIDX, static_cast<size_t>(n * ldw * 4), &widx2));
            ST(ws_get(ctx, WS_SQVAL, static_cast<size_t>(n * ldw * 8), &wval2));
            CK(launch_square_rows(static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx),
                                  static_cast<uint64_t*>(wval), static_cast<uint64_t*>(P), n, ldw,
                                  static_cast<uint64_t*>(P2), ctx->sm_count, s),
               "squaring launch");
            CK(launch_wcsr_build(static_cast<uint64_t*>(P2), n, ldw, static_cast<int64_t*>(wptr2),
                                 static_cast<int32_t*>(widx2), static_cast<uint64_t*>(wval2), s, scan_scratch(ctx)),
               "word index build");
            ctx->stats.launches += 4;
            std::swap(P, P2);
            std::swap(wptr, wptr2);
            std::swap(widx, widx2);
            std::swap(wval, wval2);
            ones = -1;  // counted for the R before this squaring
            ctx->stats.frontier_squarings++;
        }
    }
    if (!square_first && q >= kSlicedMinQueries && n >= kSquareMinN && ldw <= 2048 && smp_sliced_enabled()) {
        // query rows 64 at a time (bit-sliced) when the rows of R widen fast, the closures' test; R itself is used
        // as it is (the levels stay those of R)
        int64_t W = 0, W2 = 0;
        ST(growth(&W, &W2));
        dense_reach = W > 0 && static_cast<double>(W2) > kSlicedMinGrowth * static_cast<double>(W);
    }
    // transposed word index for the pull direction (levels whose frontier is large)
    void *PT = nullptr, *wptrT = nullptr, *widxT = nullptr, *wvalT = nullptr;
    ST(ws_get(ctx, WS_PT, static_cast<size_t>(n * ldw * 8), &PT));
    ST(ws_get(ctx, WS_WPTRT, static_cast<size_t>((n + 2) * 8), &wptrT));
    ST(ws_get(ctx, WS_WIDXT, static_cast<size_t>(n * ldw * 4), &widxT));
    ST(ws_get(ctx, WS_WVALT, static_cast<size_t>(n * ldw * 8), &wvalT));
    if (ones >= 0 && ones * 16 <= n * ldw) {
        // few ones: R^T scattered from R's word index (clearing n x ldw words and one atomic OR per one) instead
        // of reading and writing every word
        CK(launch_scatter_transpose(static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx),
                                    static_cast<uint64_t*>(wval), n, ldw, static_cast<uint64_t*>(PT), ctx->sm_count,
                                    s),
           "scatter transpose");
    } else {
        CK(launch_bit_transpose(static_cast<uint64_t*>(P), static_cast<uint64_t*>(PT), n, ldw, s), "bit transpose");
    }
    CK(launch_wcsr_build(static_cast<uint64_t*>(PT), n, ldw, static_cast<int64_t*>(wptrT),
                         static_cast<int32_t*>(widxT), static_cast<uint64_t*>(wvalT), s, scan_scratch(ctx)),
       "transposed word index build");
    ctx->stats.launches += 4;
    CK(cudaMemsetAsync(ctx->d_ctl + CTL_LEVELS, 0, 3 * sizeof(int), s), "reset level and query counters");
    ProductTimer tm{ctx, o.profile != 0, s};
    double skew = 0.0;  // largest column's nonzero words over the mean
    if (dense_reach && smp_sliced_enabled()) {
        // no hubs among the columns: a pull scans a hub's whole in-list at every level until all active sources
        // reach it (power-law targets), which the one-query-per-warp kernel avoids
        int64_t wt[2] = {0, 0};
        CK(cudaMemcpyAsync(wt, static_cast<const int64_t*>(wptrT) + n, sizeof(wt), cudaMemcpyDeviceToHost, s),
           "read column word counts");
        CK(host_sync(ctx, s), "read column word counts");
        skew = static_cast<double>(wt[1]) * static_cast<double>(n) / static_cast<double>(wt[0] > 0 ? wt[0] : 1);
        dense_reach = skew <= kSlicedMaxSkew;
    }
    if (dense_reach && smp_sliced_enabled() && (!square_first || skew > kClusterClosureSkew) &&
        smp_cluster_fits(n, q, ctx->sm_count)) {
        // 64 rows per thread-block cluster with the frontier in the cluster's shared memory: query rows, or the
        // closure's identity rows
        ST(tm.begin());
        CK(launch_smp_cluster(static_cast<int64_t*>(wptrT), static_cast<int32_t*>(widxT),
                              static_cast<uint64_t*>(wvalT), n, src, ldw_src, q, out, ldw_out,
                              square_first ? 0 : o.reflexive,
                              ctx->d_ctl + CTL_LEVELS,
                              static_cast<int>(n + 1 < 0x7FFFFFFF ? n + 1 : 0x7FFFFFFF), ctx->sm_count, s,
                              deadline_of(ctx)),
           "cluster frontier kernel launch");
        ST(tm.end());
        ctx->stats.product_launches++;
        ctx->stats.launches++;
        ctx->stats.sliced_closures++;
        ctx->stats.cluster_frontiers++;
        ST(read_ctl(ctx, s, nullptr));
        ST(tm.collect());
        *levels = ctx->h_ctl[CTL_LEVELS];
        const int cap = o.max_iters > 0 ? o.max_iters : static_cast<int>(n + 1);
        if (*levels > cap) return set_err(ctx, BMLP_ERR_NOT_CONVERGED, "frontier did not empty within %d levels", cap);
        return BMLP_OK;
    }
    if (dense_reach && smp_sliced_enabled() && square_first) {
        // every row of the closure (src = the identity), 64 sources per CTA over the word index of R^T
        void* scratch = nullptr;
        ST(ws_get(ctx, WS_V, static_cast<size_t>(smp_sliced_grid(n, ctx->sm_count) * 3 * n * 8), &scratch));
        ST(tm.begin());
        CK(launch_smp_sliced(static_cast<int64_t*>(wptrT), static_cast<int32_t*>(widxT), static_cast<uint64_t*>(wvalT),
                             n, static_cast<uint64_t*>(scratch), out, ldw_out,
                             reinterpret_cast<unsigned long long*>(ctx->d_ctl + CTL_QCOUNT), ctx->d_ctl + CTL_LEVELS,
                             static_cast<int>(n + 1 < 0x7FFFFFFF ? n + 1 : 0x7FFFFFFF), ctx->sm_count, s,
                             deadline_of(ctx)),
           "sliced frontier kernel launch");
        ST(tm.end());
        ctx->stats.product_launches++;
        ctx->stats.launches++;
        ctx->stats.sliced_closures++;
        ST(read_ctl(ctx, s, nullptr));
        ST(tm.collect());
        *levels = ctx->h_ctl[CTL_LEVELS];
        return BMLP_OK;
    }
    ST(tm.begin());
    CK(launch_smp_packed(static_cast<int64_t*>(wptr), static_cast<int32_t*>(widx), static_cast<uint64_t*>(wval), n, ldw,
                         src, ldw_src, q, out, ldw_out, ctx->d_ctl + CTL_LEVELS, ctx->d_ctl + CTL_QCOUNT, o.reflexive,
                         ctx->sm_count, s, deadline_of(ctx), static_cast<int64_t*>(wptrT),
                         static_cast<int32_t*>(widxT), static_cast<uint64_t*>(wvalT)),
       "frontier kernel launch");
    ST(tm.end());
    ctx->stats.product_launches++;
    ctx->stats.launches++;
    ST(read_ctl(ctx, s, nullptr));
    ST(tm.collect());
    *levels = ctx->h_ctl[CTL_LEVELS];
    const int cap = o.max_iters > 0 ? o.max_iters : static_cast<int>(n + 1);
    if (*levels > cap) return set_err(ctx, BMLP_ERR_NOT_CONVERGED, "frontier did not empty within %d levels", cap);
    return BMLP_OK;
}

// Frontier expansion with the tensor-core frontier product. src/out packed.
bmlp_status smp_tc_run(bmlp_ctx* ctx, const Operand& R, int32_t fmt, int64_t n, const uint64_t* src, int64_t ldw_src,
                       int64_t q, uint64_t* out, int64_t ldw_out, const bmlp_options& o, cudaStream_t s, int* levels) {
    const int64_t n_pad = round_up(n, TC_PAD);
    const int64_t q_pad = round_up(q, TC_BM);
    ctx->stats.n_pad = n_pad;
    void *Rs = nullptr, *RT = nullptr, *D0 = nullptr, *D1 = nullptr, *V = nullptr, *F0 = nullptr, *F1 = nullptr;
    ST(ws_get(ctx, WS_M0, static_cast<size_t>(n_pad * n_pad), &Rs));
    ST(ws_get(ctx, WS_T0, static_cast<size_t>(n_pad * n_pad), &RT));
    ST(ws_get(ctx, WS_M1, static_cast<size_t>(q_pad * n_pad), &D0));
    ST(ws_get(ctx, WS_T1, static_cast<size_t>(q_pad * n_pad), &D1));
    ST(ws_get(ctx, WS_V, static_cast<size_t>(q_pad * n_pad), &V));
    const int64_t kb = n_pad / TC_BK, mbs = q_pad / TC_BM;
    ST(ws_get(ctx, WS_F0, static_cast<size_t>(mbs * kb), &F0));
    ST(ws_get(ctx, WS_F1, static_cast<size_t>(mbs * kb), &F1));
    ST(to_e4m3(ctx, R, fmt, n, static_cast<uint8_t*>(Rs), static_cast<uint8_t*>(RT), n_pad, s));
    launch_packed_to_e4m3(src, ldw_src, q, n, static_cast<uint8_t*>(D0), nullptr, n_pad, q_pad, s);
    CK(cudaMemsetAsync(V, 0, static_cast<size_t>(q_pad * n_pad), s), "clear visited");
    launch_block_flags(static_cast<uint8_t*>(D0), n_pad, q_pad, n_pad, static_cast<uint8_t*>(F0), s);
    ctx->stats.launches += 2;
    CK(cudaGetLastError(), "frontier encode");
    uint8_t* D[2] = {static_cast<uint8_t*>(D0), static_cast<uint8_t*>(D1)};
    uint8_t* F[2] = {static_cast<uint8_t*>(F0), static_cast<uint8_t*>(F1)};
    CUtensorMap mapA[2], mapB;
    ST(make_tmap(ctx, &mapA[0], D[0], q_pad, n_pad, n_pad, TC_BM));
    ST(make_tmap(ctx, &mapA[1], D[1], q_pad, n_pad, n_pad, TC_BM));
    ST(make_tmap(ctx, &mapB, RT, n_pad, n_pad, n_pad, TC_BN));
    TcParams p{};
    p.m_tiles = static_cast<int32_t>(mbs);
    p.n_tiles = static_cast<int32_t>(n_pad / TC_BN);
    p.k_blocks = static_cast<int32_t>(kb);
    p.mode = TC_MODE_SMP;
    p.ld = n_pad;
    p.visited = static_cast<uint8_t*>(V);
    p.changed = ctx->d_ctl + CTL_CHANGED;
    p.error = ctx->d_ctl + CTL_ERROR;
    p.wait_cycles = wait_cycles(ctx, o);
    const int tiles = p.m_tiles * p.n_tiles;
    const int grid = tiles < ctx->sm_count ? tiles : ctx->sm_count;
    const int cap = o.max_iters > 0 ? o.max_iters : static_cast<int>(n + 1);
    ProductTimer tm{ctx, o.profile != 0, s};
    int cur = 0;
    *levels = 0;
    bool converged = false;
    for (int lv = 0; lv < cap + 1; ++lv) {
        const int nxt = cur ^ 1;
        CK(cudaMemsetAsync(ctx->d_ctl, 0, 2 * sizeof(int), s), "reset flags");
        CK(cudaMemsetAsync(F[nxt], 0, static_cast<size_t>(mbs * kb), s), "reset block flags");
        p.kflags = F[cur];
        p.kflags_next = F[nxt];
        p.out_r = D[nxt];
        ST(tm.begin());
        CK(launch_tc_product(mapA[cur], mapB, p, grid, s), "tensor-core frontier launch");
        ST(tm.end());
        ctx->stats.product_launches++;
        ctx->stats.launches += 3;
        int changed = 0;
        ST(read_ctl(ctx, s, &changed));
        ST(tm.collect());
        *levels = lv + 1;
        cur = nxt;
        if (!changed) {
            converged = true;
            break;
        }
    }
    launch_bytes_to_packed(static_cast<uint8_t*>(V), n_pad, q, n, out, ldw_out, 0, s);
    ctx->stats.launches++;
    if (o.reflexive) launch_packed_or(out, ldw_out, src, ldw_src, q, n, s);
    CK(cudaGetLastError(), "decode launch");
    if (!converged) return set_err(ctx, BMLP_ERR_NOT_CONVERGED, "frontier did not empty within %d levels", cap);
    return BMLP_OK;
}

}  // namespace

// ============================================================== C ABI ===
extern "C" {

void bmlp_default_options(bmlp_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->variant = BMLP_AUTO;
    o->loop = BMLP_LOOP_HOST;
}

bmlp_status bmlp_ctx_create(bmlp_ctx** out, int32_t device) {
    if (!out) return BMLP_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return BMLP_ERR_INVALID_ARG;
    }
    bmlp_ctx* ctx = new (std::nothrow) bmlp_ctx();
    if (!ctx) return BMLP_ERR_OOM;
    ctx->device = device;
    for (int& t : ctx->tune) t = -1;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    // the clock rate bounds every in-kernel wait; its query is slow (about 0.7 ms), so it is read here only
    cudaDeviceGetAttribute(&ctx->clock_khz, cudaDevAttrClockRate, device);
    if (cudaMalloc(&ctx->d_ctl, CTL_WORDS * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ctl, CTL_HOST_WORDS * sizeof(int)) != cudaSuccess ||
        cudaEventCreate(&ctx->ev[0]) != cudaSuccess || cudaEventCreate(&ctx->ev[1]) != cudaSuccess) {
        cudaGetLastError();
        bmlp_ctx_destroy(ctx);
        return BMLP_ERR_OOM;
    }
    cudaMemset(ctx->d_ctl, 0, CTL_WORDS * sizeof(int));
    *out = ctx;
    return BMLP_OK;
}

bmlp_status bmlp_ctx_destroy(bmlp_ctx* ctx) {
    if (!ctx) return BMLP_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    batch_cache_free(ctx);
    dispatch_free(ctx);
    for (auto& b : ctx->ws)
        if (b.p) cudaFree(b.p);
    if (ctx->d_ctl) cudaFree(ctx->d_ctl);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
    return BMLP_OK;
}

const char* bmlp_last_error(const bmlp_ctx* ctx) { return ctx ? ctx->err : "null context"; }

bmlp_status bmlp_get_stats(const bmlp_ctx* ctx, bmlp_stats* out) {
    if (!ctx || !out) return BMLP_ERR_INVALID_ARG;
    *out = ctx->stats;
    return BMLP_OK;
}

static bmlp_status core_rms(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out, const bmlp_options* opts,
                     int32_t* iters_out, cudaStream_t s) {
    NvtxRange nvtx_("bmlp_rms");
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (iters_out) *iters_out = 0;
    if (n < 0) return set_err(ctx, BMLP_ERR_INVALID_ARG, "n < 0");
    if (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    if (n == 0) return BMLP_OK;
    if (!R || !out) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null matrix pointer");
    if (n > (int64_t(1) << 20)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "n > 2^20");
    DeviceGuard g(ctx->device);
    bmlp_options o = resolve(opts);
    int variant = o.variant == BMLP_AUTO ? pick_variant_rms(n) : o.variant;
    reset_stats(ctx, variant, n);
    ST(begin_call(ctx, o, s));
    const int max_iters = o.max_iters > 0 ? o.max_iters : log2_ceil(n) + 2;
    Operand in;
    OutView ov;
    ST(stage_in(ctx, R, fmt_bytes(fmt, n, n), WS_IN0, s, &in));
    ST(stage_out(ctx, out, fmt_bytes(fmt, n, n), WS_OUT, &ov));
    if (o.variant == BMLP_AUTO && dispatch_trained(ctx)) {
        // learned choice: features on the GPU, MLP prediction, argmin
        const int64_t ldw = round_up(words_of(n), 2);
        const uint64_t* Pin = in_place_packed(in, fmt, n, ldw);
        if (Pin == nullptr) {
            void* P = nullptr;
            ST(ws_get(ctx, WS_FEAT, static_cast<size_t>(n * ldw * 8), &P));
            ST(to_packed(ctx, in, fmt, n, static_cast<uint64_t*>(P), ldw, s));
            Pin = static_cast<const uint64_t*>(P);
        }
        int32_t choice = BMLP_RMS_TC;
        ST(dispatch_choose_packed(ctx, Pin, n, ldw, &choice, s));
        variant = choice;
        ctx->stats.variant = variant;
    }
    int iters = 0;
    bmlp_status st = BMLP_OK;
    if (o.loop == BMLP_LOOP_GRAPH && (variant == BMLP_RMS_TC || variant == BMLP_RMS_PACKED)) {
        // device-side loop: a batch of one problem inside the graph WHILE node
        bmlp_problem pr{};
        pr.kind = BMLP_PROBLEM_CLOSURE;
        pr.fmt = fmt;
        pr.reflexive = o.reflexive;
        pr.n = n;
        pr.R1 = in.dev;
        pr.out = ov.dev;
        int32_t it = 0;
        st = batch_run_impl(ctx, &pr, 1, variant, wait_cycles(ctx, o), &it, s, batch_solo_n());
        iters = it;
    } else if (variant == BMLP_RMS_TC) {
        const int64_t n_pad = round_up(n, TC_PAD);
        ctx->stats.n_pad = n_pad;
        void* b[4];
        const size_t bytes = static_cast<size_t>(n_pad * n_pad);
        ST(ws_get(ctx, WS_M0, bytes, &b[0]));
        ST(ws_get(ctx, WS_M1, bytes, &b[1]));
        ST(ws_get(ctx, WS_T0, bytes, &b[2]));
        ST(ws_get(ctx, WS_T1, bytes, &b[3]));
        uint8_t* M[2] = {static_cast<uint8_t*>(b[0]), static_cast<uint8_t*>(b[1])};
        uint8_t* T[2] = {static_cast<uint8_t*>(b[2]), static_cast<uint8_t*>(b[3])};
        uint8_t *res = nullptr, *res_t = nullptr;
        // while R is sparse, the squarings run on word-indexed bit rows; the tensor cores take over from their result
        SparseStart sp;
        if (!o.tc_only) ST(sparse_squarings(ctx, in, fmt, n, n_pad, max_iters, o, s, &sp));
        if (sp.done) {
            ctx->stats.iterations = iters = sp.iters;
            if (iters_out) *iters_out = iters;
            ST(packed_out(ctx, sp.P, sp.ldw, n, fmt, ov.dev, o.reflexive, s));
            return finish_out(ctx, ov, s);
        }
        Operand src = in;
        int32_t sfmt = fmt;
        int64_t sldw = words_of(n);
        if (sp.P) {
            src.dev = sp.P;
            src.host = false;
            sfmt = BMLP_FMT_PACKED64;
            sldw = sp.ldw;
        }
        bool direct = false;
        if (o.e4m3_only == 0) ST(dense_by_blocks(ctx, src, sfmt, sldw, n, n_pad, s, &direct));
        if (direct) {
            const int64_t ld4 = n_pad / 2;
            if (sfmt == BMLP_FMT_U8)
                launch_u8_to_e2m1(static_cast<const uint8_t*>(src.dev), n, M[1], T[1], n_pad, s);
            else
                launch_packed_to_e2m1(static_cast<const uint64_t*>(src.dev), sldw, n, M[1], T[1], n_pad, s);
            CK(cudaGetLastError(), "E2M1 encode");
            ctx->stats.launches++;
            const uint8_t* q = nullptr;
            const uint64_t* qb = nullptr;
            st = rms_tc_loop(ctx, n, n_pad, M, T, max_iters - sp.iters, o, s, &iters, &res, &res_t, &q, &qb);
            if ((st == BMLP_OK || st == BMLP_ERR_NOT_CONVERGED) && qb != nullptr) {
                // the squarings kept R as bit rows: the result leaves from them
                ST(packed_out(ctx, qb, n_pad / 64, n, fmt, ov.dev, o.reflexive, s));
            } else if (st == BMLP_OK || st == BMLP_ERR_NOT_CONVERGED) {
                if (fmt == BMLP_FMT_U8)
                    launch_e2m1_to_u8(q, ld4, n, static_cast<uint8_t*>(ov.dev), o.reflexive, s);
                else
                    launch_e2m1_to_packed(q, ld4, n, static_cast<uint64_t*>(ov.dev), words_of(n), o.reflexive, s);
                CK(cudaGetLastError(), "E2M1 decode");
                ctx->stats.launches++;
            }
        } else {
            ST(to_e4m3(ctx, src, sfmt, n, M[0], T[0], n_pad, s, sldw));
            st = rms_tc_loop(ctx, n, n_pad, M, T, max_iters - sp.iters, o, s, &iters, &res, &res_t);
            if (st == BMLP_OK || st == BMLP_ERR_NOT_CONVERGED)
                ST(bytes_out(ctx, res, n_pad, n, fmt, ov.dev, o.reflexive, s));
        }
        iters += sp.iters;
    } else if (variant == BMLP_RMS_PACKED) {
        const int64_t ldw = round_up(words_of(n), 2);
        ctx->stats.n_pad = ldw * 64;
        void* b[2];
        ST(ws_get(ctx, WS_M0, static_cast<size_t>(n * ldw * 8), &b[0]));
        ST(ws_get(ctx, WS_M1, static_cast<size_t>(n * ldw * 8), &b[1]));
        uint64_t* P[2] = {static_cast<uint64_t*>(b[0]), static_cast<uint64_t*>(b[1])};
        ST(to_packed(ctx, in, fmt, n, P[0], ldw, s));
        uint64_t* res = nullptr;
        st = rms_packed_loop(ctx, n, ldw, P, max_iters, o, s, &iters, &res);
        if (st == BMLP_OK || st == BMLP_ERR_NOT_CONVERGED) ST(packed_out(ctx, res, ldw, n, fmt, ov.dev, o.reflexive, s));
    } else if (variant == BMLP_SMP_PACKED || variant == BMLP_SMP_TC) {
        // the full closure as n selective queries, one per constant
        const int64_t ldw_src = words_of(n);
        void *src = nullptr, *dst = nullptr;
        ST(ws_get(ctx, WS_SRC, static_cast<size_t>(n * ldw_src * 8), &src));
        launch_identity_packed(static_cast<uint64_t*>(src), ldw_src, n, s);
        ctx->stats.launches++;
        uint64_t* outp = nullptr;
        if (fmt == BMLP_FMT_PACKED64) {
            outp = static_cast<uint64_t*>(ov.dev);
        } else {
            ST(ws_get(ctx, WS_M2, static_cast<size_t>(n * ldw_src * 8), &dst));
            outp = static_cast<uint64_t*>(dst);
        }
        bmlp_options o2 = o;
        o2.reflexive = 0;
        o2.max_iters = 0;
        if (variant == BMLP_SMP_PACKED)
            st = smp_packed_run(ctx, in, fmt, n, static_cast<uint64_t*>(src), ldw_src, n, outp, ldw_src, o2, s, &iters,
                                true);
        else
            st = smp_tc_run(ctx, in, fmt, n, static_cast<uint64_t*>(src), ldw_src, n, outp, ldw_src, o2, s, &iters);
        if (st == BMLP_OK) {
            if (fmt == BMLP_FMT_U8)
                launch_packed_to_u8(outp, ldw_src, n, static_cast<uint8_t*>(ov.dev), o.reflexive, s);
            else if (o.reflexive)
                launch_packed_copy(outp, ldw_src, n, n, outp, ldw_src, 1, s);
            ctx->stats.launches++;
            CK(cudaGetLastError(), "decode launch");
        }
    } else {
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "variant %d is not a closure variant", variant);
    }
    ctx->stats.iterations = iters;
    if (iters_out) *iters_out = iters;
    if (st != BMLP_OK) return st;
    return finish_out(ctx, ov, s);
}

static bmlp_status core_insert(bmlp_ctx* ctx, void* closure, int64_t n, int32_t fmt, const int32_t* pairs, int64_t m,
                        cudaStream_t s) {
    NvtxRange nvtx_("bmlp_insert");
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (n < 0 || m < 0) return set_err(ctx, BMLP_ERR_INVALID_ARG, "n < 0 or m < 0");
    if (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    if (n == 0 || m == 0) return BMLP_OK;
    if (!closure || !pairs) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null pointer");
    if (n > (int64_t(1) << 20)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "n > 2^20");
    DeviceGuard g(ctx->device);
    reset_stats(ctx, 0, n);
    // the facts are read on the host (they steer one launch each) and checked there
    std::vector<int32_t> hp(static_cast<size_t>(2 * m));
    if (is_device_ptr(pairs)) {
        CK(cudaMemcpyAsync(hp.data(), pairs, hp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read facts");
        CK(host_sync(ctx, s), "read facts");
    } else {
        memcpy(hp.data(), pairs, hp.size() * sizeof(int32_t));
    }
    for (int64_t k = 0; k < 2 * m; ++k)
        if (hp[k] < 0 || hp[k] >= n) return set_err(ctx, BMLP_ERR_INVALID_ARG, "fact %lld names constant %d outside [0, n)",
                                                    static_cast<long long>(k / 2), hp[k]);
    const int64_t ldw = words_of(n);
    const bool dev_packed = fmt == BMLP_FMT_PACKED64 && is_device_ptr(closure);
    uint64_t* P = nullptr;
    Operand in;
    if (dev_packed) {
        P = static_cast<uint64_t*>(closure);
    } else {
        ST(stage_in(ctx, closure, fmt_bytes(fmt, n, n), WS_IN0, s, &in));
        void* p = nullptr;
        ST(ws_get(ctx, WS_PIPE0, static_cast<size_t>(n * ldw * 8), &p));
        P = static_cast<uint64_t*>(p);
        ST(to_packed(ctx, in, fmt, n, P, ldw, s));
    }
    for (int64_t k = 0; k < m; ++k) {
        CK(launch_insert_fact(P, n, ldw, hp[2 * k], hp[2 * k + 1], ctx->sm_count, s), "insert launch");
        ctx->stats.launches++;
    }
    ctx->stats.iterations = static_cast<int32_t>(m);
    if (!dev_packed) {
        OutView ov;
        ST(stage_out(ctx, closure, fmt_bytes(fmt, n, n), WS_OUT, &ov));
        ST(packed_out(ctx, P, ldw, n, fmt, ov.dev, 0, s));
        return finish_out(ctx, ov, s);
    }
    return BMLP_OK;
}

static bmlp_status core_smp(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, const uint64_t* src_rows, int64_t q,
                     uint64_t* out_rows, const bmlp_options* opts, int32_t* iters_out, cudaStream_t s) {
    NvtxRange nvtx_("bmlp_smp");
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (iters_out) *iters_out = 0;
    if (n < 0 || q < 0) return set_err(ctx, BMLP_ERR_INVALID_ARG, "negative size");
    if (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    if (n == 0 || q == 0) return BMLP_OK;
    if (!R || !src_rows || !out_rows) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null pointer");
    if (n > (int64_t(1) << 20)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "n > 2^20");
    DeviceGuard g(ctx->device);
    bmlp_options o = resolve(opts);
    int variant = o.variant == BMLP_AUTO ? BMLP_SMP_PACKED : o.variant;
    if (variant != BMLP_SMP_PACKED && variant != BMLP_SMP_TC)
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "variant %d is not a frontier variant", variant);
    reset_stats(ctx, variant, n);
    ST(begin_call(ctx, o, s));
    const int64_t ldw = words_of(n);
    Operand in, src;
    OutView ov;
    ST(stage_in(ctx, R, fmt_bytes(fmt, n, n), WS_IN0, s, &in));
    ST(stage_in(ctx, src_rows, static_cast<size_t>(q * ldw * 8), WS_IN1, s, &src));
    ST(stage_out(ctx, out_rows, static_cast<size_t>(q * ldw * 8), WS_OUT, &ov));
    int levels = 0;
    bmlp_status st;
    if (variant == BMLP_SMP_PACKED)
        st = smp_packed_run(ctx, in, fmt, n, static_cast<const uint64_t*>(src.dev), ldw, q,
                            static_cast<uint64_t*>(ov.dev), ldw, o, s, &levels);
    else
        st = smp_tc_run(ctx, in, fmt, n, static_cast<const uint64_t*>(src.dev), ldw, q, static_cast<uint64_t*>(ov.dev),
                        ldw, o, s, &levels);
    ctx->stats.iterations = levels;
    if (iters_out) *iters_out = levels;
    if (st != BMLP_OK) return st;
    return finish_out(ctx, ov, s);
}

static bmlp_status core_compose(bmlp_ctx* ctx, const void* R1, const void* R2, int64_t n, int32_t fmt, void* out,
                         const bmlp_options* opts, int32_t* iters_out, cudaStream_t s) {
    NvtxRange nvtx_("bmlp_compose");
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (iters_out) *iters_out = 0;
    if (n < 0) return set_err(ctx, BMLP_ERR_INVALID_ARG, "n < 0");
    if (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    if (n == 0) return BMLP_OK;
    if (!R1 || !R2 || !out) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null matrix pointer");
    if (n > (int64_t(1) << 20)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "n > 2^20");
    DeviceGuard g(ctx->device);
    bmlp_options o = resolve(opts);
    int variant = o.variant == BMLP_AUTO ? pick_variant_rms(n) : o.variant;
    if (variant != BMLP_RMS_TC && variant != BMLP_RMS_PACKED)
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "variant %d is not a composition variant", variant);
    reset_stats(ctx, variant, n);
    ST(begin_call(ctx, o, s));
    const int max_iters = o.max_iters > 0 ? o.max_iters : log2_ceil(n) + 2;
    Operand a, b;
    OutView ov;
    ST(stage_in(ctx, R1, fmt_bytes(fmt, n, n), WS_IN0, s, &a));
    ST(stage_in(ctx, R2, fmt_bytes(fmt, n, n), WS_IN1, s, &b));
    ST(stage_out(ctx, out, fmt_bytes(fmt, n, n), WS_OUT, &ov));
    int iters = 0;
    bmlp_status st;
    if (variant == BMLP_RMS_TC) {
        const int64_t n_pad = round_up(n, TC_PAD);
        ctx->stats.n_pad = n_pad;
        const size_t bytes = static_cast<size_t>(n_pad * n_pad);
        void* bb[5];
        ST(ws_get(ctx, WS_M0, bytes, &bb[0]));
        ST(ws_get(ctx, WS_M1, bytes, &bb[1]));
        ST(ws_get(ctx, WS_T0, bytes, &bb[2]));
        ST(ws_get(ctx, WS_T1, bytes, &bb[3]));
        ST(ws_get(ctx, WS_M2, bytes, &bb[4]));
        uint8_t* M[2] = {static_cast<uint8_t*>(bb[0]), static_cast<uint8_t*>(bb[1])};
        uint8_t* T[2] = {static_cast<uint8_t*>(bb[2]), static_cast<uint8_t*>(bb[3])};
        uint8_t* X = static_cast<uint8_t*>(bb[4]);
        // R2+ as in bmlp_rms: squarings on bit rows while R2 is sparse, then on the tensor cores
        SparseStart sp;
        if (!o.tc_only) ST(sparse_squarings(ctx, b, fmt, n, n_pad, max_iters, o, s, &sp));
        Operand src = b;
        int32_t sfmt = fmt;
        int64_t sldw = words_of(n);
        if (sp.P) {
            src.dev = sp.P;
            src.host = false;
            sfmt = BMLP_FMT_PACKED64;
            sldw = sp.ldw;
        }
        bool direct = false;
        if (o.e4m3_only == 0) ST(dense_by_blocks(ctx, src, sfmt, sldw, n, n_pad, s, &direct));
        if (direct) {
            // dense R2: its closure on packed E2M1 operands in the halves of M[1], T[1] (as bmlp_rms), then
            // (I + R2+) R1 on the same 4-bit squaring kernel: A = I + R2+ (diagonal set in place), B^T = R1^T
            // (R1 and R1^T encoded into the first halves of M[0], T[0]) and a zero old R (M[0]'s second half), so
            // that the kernel's R' is C > 0 (into X; R'^T into T[0]'s second half)
            const int64_t ld4 = n_pad / 2;
            const size_t half = static_cast<size_t>(n_pad) * static_cast<size_t>(ld4);
            if (sfmt == BMLP_FMT_U8)
                launch_u8_to_e2m1(static_cast<const uint8_t*>(src.dev), n, M[1], T[1], n_pad, s);
            else
                launch_packed_to_e2m1(static_cast<const uint64_t*>(src.dev), sldw, n, M[1], T[1], n_pad, s);
            CK(cudaGetLastError(), "E2M1 encode");
            ctx->stats.launches++;
            const uint8_t* q = M[1];  // the closure already, when the bit-row squarings reached it
            st = BMLP_OK;
            if (!sp.done) {
                uint8_t *res = nullptr, *res_t = nullptr;
                st = rms_tc_loop(ctx, n, n_pad, M, T, max_iters - sp.iters, o, s, &iters, &res, &res_t, &q);
            }
            iters += sp.iters;
            if (st != BMLP_OK) return st;
            uint8_t* A = const_cast<uint8_t*>(q);  // a half of M[1], this call's workspace
            launch_set_diag_e2m1(A, ld4, n, s);
            if (fmt == BMLP_FMT_U8)
                launch_u8_to_e2m1(static_cast<const uint8_t*>(a.dev), n, M[0], T[0], n_pad, s);
            else
                launch_packed_to_e2m1(static_cast<const uint64_t*>(a.dev), words_of(n), n, M[0], T[0], n_pad, s);
            CK(cudaGetLastError(), "E2M1 encode of R1");
            ctx->stats.launches += 2;
            ST(e2m1_product(ctx, A, T[0], n_pad, M[0] + half, X, T[0] + half, o, s));
            if (fmt == BMLP_FMT_U8)
                launch_e2m1_to_u8(X, ld4, n, static_cast<uint8_t*>(ov.dev), 0, s);
            else
                launch_e2m1_to_packed(X, ld4, n, static_cast<uint64_t*>(ov.dev), words_of(n), 0, s);
            CK(cudaGetLastError(), "E2M1 decode");
            ctx->stats.launches++;
        } else {
            if (sp.P) {
                Operand pk;
                pk.dev = sp.P;
                ST(to_e4m3(ctx, pk, BMLP_FMT_PACKED64, n, M[0], T[0], n_pad, s, sp.ldw));
            } else {
                ST(to_e4m3(ctx, b, fmt, n, M[0], T[0], n_pad, s));
            }
            uint8_t *res = nullptr, *res_t = nullptr;
            if (sp.done) {
                res = M[0];
                res_t = T[0];
                st = BMLP_OK;
            } else {
                st = rms_tc_loop(ctx, n, n_pad, M, T, max_iters - sp.iters, o, s, &iters, &res, &res_t);
            }
            iters += sp.iters;
            if (st != BMLP_OK) return st;
            // A = I + R2+ (row-major, in res); B^T = R1^T (written into the other R^T buffer)
            launch_set_diag_e4m3(res, n_pad, n, s);
            ctx->stats.launches++;
            uint8_t* r1t = (res_t == T[0]) ? T[1] : T[0];
            uint8_t* r1 = (res == M[0]) ? M[1] : M[0];
            ST(to_e4m3(ctx, a, fmt, n, r1, r1t, n_pad, s));
            ST(tc_plain_product(ctx, res, r1t, n_pad, X, o, s));
            ST(bytes_out(ctx, X, n_pad, n, fmt, ov.dev, 0, s));
        }
    } else {
        const int64_t ldw = round_up(words_of(n), 2);
        ctx->stats.n_pad = ldw * 64;
        const size_t bytes = static_cast<size_t>(n * ldw * 8);
        void* bb[4];
        ST(ws_get(ctx, WS_M0, bytes, &bb[0]));
        ST(ws_get(ctx, WS_M1, bytes, &bb[1]));
        ST(ws_get(ctx, WS_T0, bytes, &bb[2]));
        ST(ws_get(ctx, WS_T1, bytes, &bb[3]));
        uint64_t* P[2] = {static_cast<uint64_t*>(bb[0]), static_cast<uint64_t*>(bb[1])};
        uint64_t* A1 = static_cast<uint64_t*>(bb[2]);
        uint64_t* X = static_cast<uint64_t*>(bb[3]);
        ST(to_packed(ctx, b, fmt, n, P[0], ldw, s));
        uint64_t* res = nullptr;
        st = rms_packed_loop(ctx, n, ldw, P, max_iters, o, s, &iters, &res);
        if (st != BMLP_OK) return st;
        launch_packed_copy(res, ldw, n, n, res, ldw, 1, s);  // I + R2+
        ST(to_packed(ctx, a, fmt, n, A1, ldw, s));
        CK(cudaMemsetAsync(ctx->d_ctl, 0, 2 * sizeof(int), s), "reset flags");
        CK(launch_product_packed(res, A1, X, n, ldw, 0, ctx->d_ctl + CTL_CHANGED, ctx->sm_count, s), "product launch");
        ctx->stats.product_launches++;
        ctx->stats.launches += 2;
        ST(read_ctl(ctx, s, nullptr));
        ST(packed_out(ctx, X, ldw, n, fmt, ov.dev, 0, s));
    }
    ctx->stats.iterations = iters;
    if (iters_out) *iters_out = iters;
    return finish_out(ctx, ov, s);
}

// Algorithm 1 as printed: R* = (I + R1)^(2^k) by squaring until a squaring changes nothing, then one product
// R* R1 = R1+. With I inside R the squaring step R <- R + R R is R <- R R, so the squaring loop of bmlp_rms run on
// I + R1 is Algorithm 1's loop (same engines and switches); the last product runs on the tensor cores.
static bmlp_status core_rms_alg1(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out, const bmlp_options* opts,
                          int32_t* iters_out, cudaStream_t s) {
    NvtxRange nvtx_("bmlp_rms_alg1");
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (iters_out) *iters_out = 0;
    if (n < 0) return set_err(ctx, BMLP_ERR_INVALID_ARG, "n < 0");
    if (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    if (n == 0) return BMLP_OK;
    if (!R || !out) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null matrix pointer");
    if (n > (int64_t(1) << 20)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "n > 2^20");
    DeviceGuard g(ctx->device);
    bmlp_options o = resolve(opts);
    if (o.variant != BMLP_AUTO && o.variant != BMLP_RMS_TC)
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "Algorithm 1 runs as tensor-core squaring (variant %d)", o.variant);
    reset_stats(ctx, BMLP_RMS_TC, n);
    ST(begin_call(ctx, o, s));
    Operand a;
    OutView ov;
    ST(stage_in(ctx, R, fmt_bytes(fmt, n, n), WS_IN0, s, &a));
    ST(stage_out(ctx, out, fmt_bytes(fmt, n, n), WS_OUT, &ov));
    // I + R1 as packed rows
    const int64_t ldw = words_of(n);
    void *p0 = nullptr, *q = nullptr;
    ST(ws_get(ctx, WS_PIPE0, static_cast<size_t>(n * ldw * 8), &p0));
    ST(ws_get(ctx, WS_PIPE1, static_cast<size_t>(n * ldw * 8), &q));
    if (fmt == BMLP_FMT_U8) {
        launch_u8_to_packed(static_cast<const uint8_t*>(a.dev), n, static_cast<uint64_t*>(p0), ldw, s);
        launch_packed_copy(static_cast<uint64_t*>(p0), ldw, n, n, static_cast<uint64_t*>(p0), ldw, 1, s);
    } else {
        launch_packed_copy(static_cast<const uint64_t*>(a.dev), ldw, n, n, static_cast<uint64_t*>(p0), ldw, 1, s);
    }
    CK(cudaGetLastError(), "encode launch");
    // squarings of I + R1 until one changes nothing: q = I + R1+
    bmlp_options o2 = o;
    o2.variant = BMLP_RMS_TC;
    o2.reflexive = 0;
    o2.loop = BMLP_LOOP_HOST;
    int32_t squarings = 0;
    ST(core_rms(ctx, p0, n, BMLP_FMT_PACKED64, q, &o2, &squarings, s));
    ctx->stats.launches += fmt == BMLP_FMT_U8 ? 2 : 1;
    // R1+ = (I + R1+) R1 on the tensor cores
    const int64_t n_pad = round_up(n, TC_PAD);
    const size_t bytes = static_cast<size_t>(n_pad * n_pad);
    void* bb[5];
    ST(ws_get(ctx, WS_M0, bytes, &bb[0]));
    ST(ws_get(ctx, WS_M1, bytes, &bb[1]));
    ST(ws_get(ctx, WS_T0, bytes, &bb[2]));
    ST(ws_get(ctx, WS_T1, bytes, &bb[3]));
    ST(ws_get(ctx, WS_M2, bytes, &bb[4]));
    uint8_t* B8[5];
    for (int k = 0; k < 5; ++k) B8[k] = static_cast<uint8_t*>(bb[k]);
    if (o.e4m3_only == 0) {
        // on 4-bit operands: A = I + R1+ and R1 (with R1^T) as packed E2M1 in the first halves of the buffers
        const int64_t ld4 = n_pad / 2;
        const size_t half = static_cast<size_t>(n_pad) * static_cast<size_t>(ld4);
        launch_packed_to_e2m1(static_cast<const uint64_t*>(q), ldw, n, B8[0], B8[2], n_pad, s);
        if (fmt == BMLP_FMT_U8)
            launch_u8_to_e2m1(static_cast<const uint8_t*>(a.dev), n, B8[1], B8[3], n_pad, s);
        else
            launch_packed_to_e2m1(static_cast<const uint64_t*>(a.dev), ldw, n, B8[1], B8[3], n_pad, s);
        CK(cudaGetLastError(), "E2M1 encode");
        ctx->stats.launches += 2;
        ST(e2m1_product(ctx, B8[0], B8[3], n_pad, B8[0] + half, B8[4], B8[2] + half, o, s));
        if (fmt == BMLP_FMT_U8)
            launch_e2m1_to_u8(B8[4], ld4, n, static_cast<uint8_t*>(ov.dev), o.reflexive, s);
        else
            launch_e2m1_to_packed(B8[4], ld4, n, static_cast<uint64_t*>(ov.dev), words_of(n), o.reflexive, s);
        CK(cudaGetLastError(), "E2M1 decode");
        ctx->stats.launches++;
    } else {
        Operand qs;
        qs.dev = q;
        ST(to_e4m3(ctx, qs, BMLP_FMT_PACKED64, n, B8[0], B8[2], n_pad, s, ldw));
        ST(to_e4m3(ctx, a, fmt, n, B8[1], B8[3], n_pad, s));
        ST(tc_plain_product(ctx, B8[0], B8[3], n_pad, B8[4], o, s));
        ST(bytes_out(ctx, B8[4], n_pad, n, fmt, ov.dev, o.reflexive, s));
    }
    ctx->stats.iterations = squarings + 1;
    if (iters_out) *iters_out = squarings + 1;
    return finish_out(ctx, ov, s);
}

// ---- relation operators of Sec. 3.4 (Fig. 3) on packed rows of words_of(n) words
static bmlp_status op_args(bmlp_ctx* ctx, int64_t n, int32_t fmt) {
    if (n < 0) return set_err(ctx, BMLP_ERR_INVALID_ARG, "n < 0");
    if (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    if (n > (int64_t(1) << 20)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "n > 2^20");
    return BMLP_OK;
}

// A packed workspace copy of a caller matrix (staged through `stage_slot` when it is host memory).
static bmlp_status packed_operand(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, int stage_slot, int slot,
                                  cudaStream_t s, uint64_t** P) {
    Operand in;
    ST(stage_in(ctx, R, fmt_bytes(fmt, n, n), stage_slot, s, &in));
    void* p = nullptr;
    ST(ws_get(ctx, slot, static_cast<size_t>(n * words_of(n) * 8), &p));
    *P = static_cast<uint64_t*>(p);
    return to_packed(ctx, in, fmt, n, *P, words_of(n), s);
}

static bmlp_status core_transpose(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out, cudaStream_t s) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    ST(op_args(ctx, n, fmt));
    if (n == 0) return BMLP_OK;
    if (!R || !out) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null matrix pointer");
    DeviceGuard g(ctx->device);
    reset_stats(ctx, 0, n);
    const int64_t ldw = words_of(n);
    uint64_t *P = nullptr, *PT = nullptr;
    ST(packed_operand(ctx, R, n, fmt, WS_IN0, WS_PIPE0, s, &P));
    void* pt = nullptr;
    ST(ws_get(ctx, WS_PIPE1, static_cast<size_t>(n * ldw * 8), &pt));
    PT = static_cast<uint64_t*>(pt);
    CK(launch_bit_transpose(P, PT, n, ldw, s), "transpose launch");
    ctx->stats.launches++;
    OutView ov;
    ST(stage_out(ctx, out, fmt_bytes(fmt, n, n), WS_OUT, &ov));
    ST(packed_out(ctx, PT, ldw, n, fmt, ov.dev, 0, s));
    return finish_out(ctx, ov, s);
}

static bmlp_status core_union(bmlp_ctx* ctx, const void* A, const void* B, int64_t n, int32_t fmt, void* out, cudaStream_t s) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    ST(op_args(ctx, n, fmt));
    if (n == 0) return BMLP_OK;
    if (!A || !B || !out) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null matrix pointer");
    DeviceGuard g(ctx->device);
    reset_stats(ctx, 0, n);
    const int64_t ldw = words_of(n);
    uint64_t *PA = nullptr, *PB = nullptr;
    ST(packed_operand(ctx, A, n, fmt, WS_IN0, WS_PIPE0, s, &PA));
    ST(packed_operand(ctx, B, n, fmt, WS_IN1, WS_PIPE1, s, &PB));
    launch_packed_or(PA, ldw, PB, ldw, n, n, s);
    ctx->stats.launches++;
    CK(cudaGetLastError(), "union launch");
    OutView ov;
    ST(stage_out(ctx, out, fmt_bytes(fmt, n, n), WS_OUT, &ov));
    ST(packed_out(ctx, PA, ldw, n, fmt, ov.dev, 0, s));
    return finish_out(ctx, ov, s);
}

// Device view of an optional packed type vector (null = every constant).
static bmlp_status type_vector(bmlp_ctx* ctx, const uint64_t* v, int64_t n, int slot, cudaStream_t s,
                               const uint64_t** dv) {
    *dv = nullptr;
    if (!v) return BMLP_OK;
    Operand o;
    ST(stage_in(ctx, v, static_cast<size_t>(words_of(n) * 8), slot, s, &o));
    *dv = static_cast<const uint64_t*>(o.dev);
    return BMLP_OK;
}

static bmlp_status core_negate(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, const uint64_t* rows,
                        const uint64_t* cols, void* out, cudaStream_t s) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    ST(op_args(ctx, n, fmt));
    if (n == 0) return BMLP_OK;
    if (!R || !out) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null matrix pointer");
    DeviceGuard g(ctx->device);
    reset_stats(ctx, 0, n);
    const int64_t ldw = words_of(n);
    uint64_t* P = nullptr;
    ST(packed_operand(ctx, R, n, fmt, WS_IN0, WS_PIPE0, s, &P));
    const uint64_t *dr = nullptr, *dc = nullptr;
    ST(type_vector(ctx, rows, n, WS_SRC, s, &dr));
    ST(type_vector(ctx, cols, n, WS_VEC0, s, &dc));
    launch_packed_negate(P, ldw, n, dr, dc, P, ldw, s);
    ctx->stats.launches++;
    CK(cudaGetLastError(), "negate launch");
    OutView ov;
    ST(stage_out(ctx, out, fmt_bytes(fmt, n, n), WS_OUT, &ov));
    ST(packed_out(ctx, P, ldw, n, fmt, ov.dev, 0, s));
    return finish_out(ctx, ov, s);
}

static bmlp_status core_is_foreign(bmlp_ctx* ctx, const void* contains, const void* adjoins, const uint64_t* location,
                            int64_t n, int32_t fmt, void* out, const bmlp_options* opts, int32_t* iters_out,
                            cudaStream_t s) {
    NvtxRange nvtx_("bmlp_is_foreign");
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (iters_out) iters_out[0] = iters_out[1] = 0;
    ST(op_args(ctx, n, fmt));
    if (n == 0) return BMLP_OK;
    if (!contains || !adjoins || !out) return set_err(ctx, BMLP_ERR_INVALID_ARG, "null matrix pointer");
    DeviceGuard g(ctx->device);
    const bmlp_options o = resolve(opts);
    const int64_t ldw = words_of(n);
    const size_t pbytes = static_cast<size_t>(n * ldw * 8);
    // PA = adjoins, PC = contains (packed); PH receives hasPlace = contains+ (P3)
    uint64_t *PA = nullptr, *PC = nullptr, *PH = nullptr;
    ST(packed_operand(ctx, adjoins, n, fmt, WS_IN1, WS_PIPE0, s, &PA));
    ST(packed_operand(ctx, contains, n, fmt, WS_IN0, WS_PIPE2, s, &PC));
    void* ph = nullptr;
    ST(ws_get(ctx, WS_PIPE1, pbytes, &ph));
    PH = static_cast<uint64_t*>(ph);
    bmlp_options oc = o;
    oc.reflexive = 0;
    int32_t it0 = 0, it1 = 0;
    ST(core_rms(ctx, PC, n, BMLP_FMT_PACKED64, PH, &oc, &it0, s));
    bmlp_stats acc = ctx->stats;
    // P4: indirectlyPartOf = adjoins u adjoins^T u hasPlace^T . indirectlyPartOf = (I + (hasPlace^T)+) B
    CK(launch_bit_transpose(PH, PC, n, ldw, s), "transpose launch");  // PC := hasPlace^T
    CK(launch_bit_transpose(PA, PH, n, ldw, s), "transpose launch");  // PH := adjoins^T
    launch_packed_or(PH, ldw, PA, ldw, n, n, s);                     // PH := B = adjoins u adjoins^T
    CK(cudaGetLastError(), "union launch");
    oc.variant = (o.variant == BMLP_RMS_TC || o.variant == BMLP_SMP_TC) ? BMLP_RMS_TC : BMLP_RMS_PACKED;
    ST(core_compose(ctx, PH, PC, n, BMLP_FMT_PACKED64, PA, &oc, &it1, s));  // PA := indirectlyPartOf
    // P5: isForeign = location x location AND NOT indirectlyPartOf
    const uint64_t* loc = nullptr;
    ST(type_vector(ctx, location, n, WS_VEC0, s, &loc));
    launch_packed_negate(PA, ldw, n, loc, loc, PA, ldw, s);
    CK(cudaGetLastError(), "negate launch");
    OutView ov;
    ST(stage_out(ctx, out, fmt_bytes(fmt, n, n), WS_OUT, &ov));
    ST(packed_out(ctx, PA, ldw, n, fmt, ov.dev, 0, s));
    acc.product_launches += ctx->stats.product_launches;
    acc.launches += ctx->stats.launches + 5;
    acc.product_ms += ctx->stats.product_ms;
    acc.issued_ops += ctx->stats.issued_ops;
    acc.iterations = it0 + it1;
    ctx->stats = acc;
    if (iters_out) {
        iters_out[0] = it0;
        iters_out[1] = it1;
    }
    return finish_out(ctx, ov, s);
}

bmlp_status bmlp_batch_run(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, const bmlp_options* opts,
                           int32_t* iters_out, cudaStream_t s) {
    NvtxRange nvtx_("bmlp_batch_run");
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (count < 0 || (count > 0 && !probs)) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad problem list");
    if (count == 0) return BMLP_OK;
    DeviceGuard g(ctx->device);
    bmlp_options o = resolve(opts);
    if (o.variant != BMLP_AUTO && o.variant != BMLP_RMS_TC && o.variant != BMLP_RMS_PACKED &&
        o.variant != BMLP_SMP_PACKED)
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "variant %d is not a batch variant", o.variant);
    for (int64_t i = 0; i < count; ++i)
        if (probs[i].variant < 0 || probs[i].variant > BMLP_SMP_PACKED)
            return set_err(ctx, BMLP_ERR_INVALID_ARG, "problem %lld: bad variant %d", static_cast<long long>(i),
                           probs[i].variant);
    // Problems large enough to fill the GPU on their own (n >= batch_solo_n()) and not forced onto packed rows run
    // inside the same graph as device-driven single-problem pipelines (squarings on bit rows while R is sparse, then
    // on 4-bit operands on the tensor cores); the rest run together as one grouped batch. One graph launch, one
    // read of the results.
    // I8 problems are read and written as U8
    std::vector<bmlp_problem> canon;
    for (int64_t i = 0; i < count; ++i)
        if (probs[i].fmt == BMLP_FMT_I8) {
            canon.assign(probs, probs + count);
            for (bmlp_problem& q : canon)
                if (q.fmt == BMLP_FMT_I8) q.fmt = BMLP_FMT_U8;
            probs = canon.data();
            break;
        }
    reset_stats(ctx, o.variant, 0);
    ProductTimer tm{ctx, o.profile != 0, s};
    ST(tm.begin());
    bmlp_status st = batch_run_impl(ctx, probs, count, o.variant, wait_cycles(ctx, o), iters_out, s, batch_solo_n());
    ST(tm.end());
    if (o.profile) {
        CK(cudaEventSynchronize(ctx->ev[1]), "synchronise batch timer");
        ST(tm.collect());
    }
    return st;
}

bmlp_status bmlp_batch_autotune(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, const char* cache_path,
                                cudaStream_t s) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (count < 0 || (count > 0 && !probs)) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad problem list");
    DeviceGuard g(ctx->device);
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, ctx->device), "device properties");
    std::string gpu(prop.name);
    for (char& ch : gpu)
        if (ch == ' ') ch = '_';
    bool from_file = false;
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            char name[256];
            int b = 0, eng = 0;
            double t0 = 0, t1 = 0;
            while (fscanf(f, "%255s %d %d %lf %lf", name, &b, &eng, &t0, &t1) == 5)
                if (gpu == name && b >= 0 && b < 32 && (eng == 0 || eng == 1)) {
                    ctx->tune[b] = eng;
                    from_file = true;
                }
            fclose(f);
        }
    }
    if (from_file) return BMLP_OK;
    bmlp_options o;
    bmlp_default_options(&o);
    const long long wc = wait_cycles(ctx, o);
    std::vector<std::string> lines;
    for (int b = 0; b < 32; ++b) {
        std::vector<bmlp_problem> sub;
        for (int64_t i = 0; i < count; ++i)
            if (probs[i].kind == BMLP_PROBLEM_CLOSURE && probs[i].n > 0 && (int64_t(1) << b) >= probs[i].n &&
                (b == 0 || (int64_t(1) << (b - 1)) < probs[i].n))
                sub.push_back(probs[i]);
        if (sub.empty()) continue;
        double ms[2] = {0, 0};
        for (int eng = 0; eng < 2; ++eng) {
            const int variant = eng == 0 ? BMLP_RMS_TC : BMLP_RMS_PACKED;
            bmlp_status st = batch_run_impl(ctx, sub.data(), static_cast<int64_t>(sub.size()), variant, wc, nullptr, s);
            if (st != BMLP_OK && st != BMLP_ERR_NOT_CONVERGED) return st;
            CK(cudaEventRecord(ctx->ev[0], s), "event");
            st = batch_run_impl(ctx, sub.data(), static_cast<int64_t>(sub.size()), variant, wc, nullptr, s);
            if (st != BMLP_OK && st != BMLP_ERR_NOT_CONVERGED) return st;
            CK(cudaEventRecord(ctx->ev[1], s), "event");
            CK(cudaEventSynchronize(ctx->ev[1]), "event");
            float t = 0;
            CK(cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]), "event");
            ms[eng] = t;
        }
        ctx->tune[b] = ms[1] < ms[0] ? 1 : 0;
        char buf[512];
        snprintf(buf, sizeof(buf), "%s %d %d %.6f %.6f\n", gpu.c_str(), b, ctx->tune[b], ms[0], ms[1]);
        lines.push_back(buf);
    }
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            for (auto& l : lines) fputs(l.c_str(), f);
            fclose(f);
        }
    }
    return BMLP_OK;
}

static bmlp_status core_dispatch_features(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, float* feats, cudaStream_t s) {
    if (!ctx || !feats) return BMLP_ERR_INVALID_ARG;
    if (n <= 0 || !R) return set_err(ctx, BMLP_ERR_INVALID_ARG, "features need n > 0 and a matrix");
    if (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    DeviceGuard g(ctx->device);
    Operand in;
    ST(stage_in(ctx, R, fmt_bytes(fmt, n, n), WS_IN0, s, &in));
    const int64_t ldw = round_up(words_of(n), 2);
    const uint64_t* Pin = in_place_packed(in, fmt, n, ldw);
    if (Pin == nullptr) {
        void* P = nullptr;
        ST(ws_get(ctx, WS_FEAT, static_cast<size_t>(n * ldw * 8), &P));
        ST(to_packed(ctx, in, fmt, n, static_cast<uint64_t*>(P), ldw, s));
        Pin = static_cast<const uint64_t*>(P);
    }
    return dispatch_features_packed(ctx, Pin, n, ldw, feats, s);
}

bmlp_status bmlp_dispatch_train(bmlp_ctx* ctx, const float* feats, const float* log2_ms, const uint8_t* censored,
                                int64_t m, const bmlp_train_cfg* cfg, float* final_loss) {
    if (!ctx || !cfg) return BMLP_ERR_INVALID_ARG;
    if (m <= 0 || !feats || !log2_ms || !censored) return set_err(ctx, BMLP_ERR_INVALID_ARG, "empty training set");
    if (cfg->epochs < 0 || cfg->batch < 0 || m > (int64_t(1) << 26))
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad training configuration");
    DeviceGuard g(ctx->device);
    return dispatch_train(ctx, feats, log2_ms, censored, m, cfg, final_loss);
}

bmlp_status bmlp_dispatch_predict(bmlp_ctx* ctx, const float* feats, int64_t m, float* pred, int32_t* choice) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (m < 0 || (m > 0 && !feats)) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad feature rows");
    DeviceGuard g(ctx->device);
    return dispatch_predict(ctx, feats, m, pred, choice, nullptr);
}

bmlp_status bmlp_dispatch_loss_grad(bmlp_ctx* ctx, const float* feats, const float* log2_ms, const uint8_t* censored,
                                    int64_t m, float* loss, float* grad) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (m <= 0 || !feats || !log2_ms || !censored || !loss || !grad)
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad arguments");
    DeviceGuard g(ctx->device);
    return dispatch_loss_grad(ctx, feats, log2_ms, censored, m, loss, grad);
}

bmlp_status bmlp_dispatch_set_params(bmlp_ctx* ctx, const float* params, const float* mu, const float* sigma) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return dispatch_set_params(ctx, params, mu, sigma);
}

bmlp_status bmlp_dispatch_get_params(bmlp_ctx* ctx, float* params, float* mu, float* sigma) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return dispatch_get_params(ctx, params, mu, sigma);
}

bmlp_status bmlp_dispatch_save(bmlp_ctx* ctx, const char* path) {
    if (!ctx || !path) return BMLP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return dispatch_save(ctx, path);
}

bmlp_status bmlp_dispatch_load(bmlp_ctx* ctx, const char* path) {
    if (!ctx || !path) return BMLP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return dispatch_load(ctx, path);
}


// ---- byte formats: I8 is read and written as U8 (nonzero = 1, outputs 0 / 1); E4M3 inputs are turned into 0 / 1
// bytes (0x00 and 0x80 are zero, any other byte is one) in a context buffer, the U8 path runs, and the 0 / 1
// result becomes E4M3 bytes (0x00 / 0x38) in the caller's buffer.
#define FMT_WRAP_CHECK(fmt)                                                                       \
    do {                                                                                          \
        if ((fmt) == BMLP_FMT_I8) (fmt) = BMLP_FMT_U8;                                            \
    } while (0)

static bmlp_status e4m3_in(bmlp_ctx* ctx, const void* p, int64_t n, int slot, cudaStream_t s, const void** out) {
    if (!p) {
        *out = nullptr;
        return BMLP_OK;
    }
    const size_t bytes = static_cast<size_t>(n) * static_cast<size_t>(n);
    void* d = nullptr;
    ST(ws_get(ctx, slot, bytes, &d));
    CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyDefault, s), "copy E4M3 input");
    launch_e4m3_bytes_to_01(static_cast<uint8_t*>(d), static_cast<int64_t>(bytes), s);
    CK(cudaGetLastError(), "E4M3 input");
    *out = d;
    return BMLP_OK;
}

static bmlp_status e4m3_out_buf(bmlp_ctx* ctx, int64_t n, void** out) {
    return ws_get(ctx, WS_E8_OUT, static_cast<size_t>(n) * static_cast<size_t>(n), out);
}

static bmlp_status e4m3_out_done(bmlp_ctx* ctx, const void* tmp, void* out, int64_t n, cudaStream_t s) {
    const size_t bytes = static_cast<size_t>(n) * static_cast<size_t>(n);
    launch_01_to_e4m3_bytes(static_cast<uint8_t*>(const_cast<void*>(tmp)), static_cast<int64_t>(bytes), s);
    CK(cudaGetLastError(), "E4M3 output");
    CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDefault, s), "copy E4M3 output");
    if (!is_device_ptr(out)) CK(host_sync(ctx, s), "synchronise E4M3 output");
    return BMLP_OK;
}

bmlp_status bmlp_rms(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out, const bmlp_options* opts,
                     int32_t* iters_out, cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !R || !out) return core_rms(ctx, R, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, out, opts, iters_out, s);
    DeviceGuard g(ctx->device);
    const void* r = nullptr;
    void* t = nullptr;
    ST(e4m3_in(ctx, R, n, WS_E8_IN0, s, &r));
    ST(e4m3_out_buf(ctx, n, &t));
    ST(core_rms(ctx, r, n, BMLP_FMT_U8, t, opts, iters_out, s));
    return e4m3_out_done(ctx, t, out, n, s);
}

bmlp_status bmlp_rms_alg1(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out, const bmlp_options* opts,
                          int32_t* iters_out, cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !R || !out) return core_rms_alg1(ctx, R, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, out, opts, iters_out, s);
    DeviceGuard g(ctx->device);
    const void* r = nullptr;
    void* t = nullptr;
    ST(e4m3_in(ctx, R, n, WS_E8_IN0, s, &r));
    ST(e4m3_out_buf(ctx, n, &t));
    ST(core_rms_alg1(ctx, r, n, BMLP_FMT_U8, t, opts, iters_out, s));
    return e4m3_out_done(ctx, t, out, n, s);
}

bmlp_status bmlp_smp(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, const uint64_t* src_rows, int64_t q,
                     uint64_t* out_rows, const bmlp_options* opts, int32_t* iters_out, cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !R) return core_smp(ctx, R, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, src_rows, q, out_rows, opts, iters_out, s);
    DeviceGuard g(ctx->device);
    const void* r = nullptr;
    ST(e4m3_in(ctx, R, n, WS_E8_IN0, s, &r));
    return core_smp(ctx, r, n, BMLP_FMT_U8, src_rows, q, out_rows, opts, iters_out, s);
}

bmlp_status bmlp_compose(bmlp_ctx* ctx, const void* R1, const void* R2, int64_t n, int32_t fmt, void* out,
                         const bmlp_options* opts, int32_t* iters_out, cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !R1 || !R2 || !out) return core_compose(ctx, R1, R2, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, out, opts, iters_out, s);
    DeviceGuard g(ctx->device);
    const void *a = nullptr, *b = nullptr;
    void* t = nullptr;
    ST(e4m3_in(ctx, R1, n, WS_E8_IN0, s, &a));
    ST(e4m3_in(ctx, R2, n, WS_E8_IN1, s, &b));
    ST(e4m3_out_buf(ctx, n, &t));
    ST(core_compose(ctx, a, b, n, BMLP_FMT_U8, t, opts, iters_out, s));
    return e4m3_out_done(ctx, t, out, n, s);
}

bmlp_status bmlp_insert(bmlp_ctx* ctx, void* closure, int64_t n, int32_t fmt, const int32_t* pairs, int64_t m,
                        cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !closure) return core_insert(ctx, closure, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, pairs, m, s);
    DeviceGuard g(ctx->device);
    const void* c = nullptr;
    ST(e4m3_in(ctx, closure, n, WS_E8_IN0, s, &c));
    ST(core_insert(ctx, const_cast<void*>(c), n, BMLP_FMT_U8, pairs, m, s));
    return e4m3_out_done(ctx, c, closure, n, s);
}

bmlp_status bmlp_transpose(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out, cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !R || !out) return core_transpose(ctx, R, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, out, s);
    DeviceGuard g(ctx->device);
    const void* r = nullptr;
    void* t = nullptr;
    ST(e4m3_in(ctx, R, n, WS_E8_IN0, s, &r));
    ST(e4m3_out_buf(ctx, n, &t));
    ST(core_transpose(ctx, r, n, BMLP_FMT_U8, t, s));
    return e4m3_out_done(ctx, t, out, n, s);
}

bmlp_status bmlp_union(bmlp_ctx* ctx, const void* A, const void* B, int64_t n, int32_t fmt, void* out,
                       cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !A || !B || !out) return core_union(ctx, A, B, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, out, s);
    DeviceGuard g(ctx->device);
    const void *a = nullptr, *b = nullptr;
    void* t = nullptr;
    ST(e4m3_in(ctx, A, n, WS_E8_IN0, s, &a));
    ST(e4m3_in(ctx, B, n, WS_E8_IN1, s, &b));
    ST(e4m3_out_buf(ctx, n, &t));
    ST(core_union(ctx, a, b, n, BMLP_FMT_U8, t, s));
    return e4m3_out_done(ctx, t, out, n, s);
}

bmlp_status bmlp_negate(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, const uint64_t* rows,
                        const uint64_t* cols, void* out, cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !R || !out) return core_negate(ctx, R, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, rows, cols, out, s);
    DeviceGuard g(ctx->device);
    const void* r = nullptr;
    void* t = nullptr;
    ST(e4m3_in(ctx, R, n, WS_E8_IN0, s, &r));
    ST(e4m3_out_buf(ctx, n, &t));
    ST(core_negate(ctx, r, n, BMLP_FMT_U8, rows, cols, t, s));
    return e4m3_out_done(ctx, t, out, n, s);
}

bmlp_status bmlp_is_foreign(bmlp_ctx* ctx, const void* contains, const void* adjoins, const uint64_t* location,
                            int64_t n, int32_t fmt, void* out, const bmlp_options* opts, int32_t* iters_out,
                            cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !contains || !adjoins || !out)
        return core_is_foreign(ctx, contains, adjoins, location, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, out, opts, iters_out, s);
    DeviceGuard g(ctx->device);
    const void *c = nullptr, *a = nullptr;
    void* t = nullptr;
    ST(e4m3_in(ctx, contains, n, WS_E8_IN0, s, &c));
    ST(e4m3_in(ctx, adjoins, n, WS_E8_IN1, s, &a));
    ST(e4m3_out_buf(ctx, n, &t));
    ST(core_is_foreign(ctx, c, a, location, n, BMLP_FMT_U8, t, opts, iters_out, s));
    return e4m3_out_done(ctx, t, out, n, s);
}

bmlp_status bmlp_dispatch_choose_many(bmlp_ctx* ctx, const void* const* R, const int64_t* n, int64_t m, int32_t fmt,
                                      int32_t* choice, float* feats, cudaStream_t s) {
    if (!ctx) return BMLP_ERR_INVALID_ARG;
    if (m < 0 || (m > 0 && (!R || !n || !choice))) return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad matrix list");
    const bool e4m3 = fmt == BMLP_FMT_E4M3;
    FMT_WRAP_CHECK(fmt);
    if (!e4m3 && fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64)
        return set_err(ctx, BMLP_ERR_INVALID_ARG, "bad format %d", fmt);
    for (int64_t i = 0; i < m; ++i)
        if (!R[i] || n[i] <= 0) return set_err(ctx, BMLP_ERR_INVALID_ARG, "matrix %lld: null or n <= 0", (long long)i);
    DeviceGuard g(ctx->device);
    if (!dispatch_trained(ctx)) return set_err(ctx, BMLP_ERR_UNSUPPORTED, "no dispatcher model (train, load or set one)");
    if (m == 0) return BMLP_OK;
    std::vector<const uint64_t*> P(static_cast<size_t>(m), nullptr);
    std::vector<int64_t> ldw(static_cast<size_t>(m));
    size_t need = 0;  // 64-bit words of the matrices that are converted
    for (int64_t i = 0; i < m; ++i) {
        ldw[i] = round_up(words_of(n[i]), 2);
        if (!e4m3 && is_device_ptr(R[i])) P[i] = in_place_packed(Operand{R[i], false}, fmt, n[i], ldw[i]);
        if (P[i] == nullptr) need += static_cast<size_t>(n[i] * ldw[i]);
    }
    uint64_t* buf = nullptr;
    if (need > 0) {
        void* b = nullptr;
        ST(ws_get(ctx, WS_FEAT, need * 8, &b));
        buf = static_cast<uint64_t*>(b);
    }
    // converted one after another in stream order, so the staging slots may be reused from one matrix to the next
    size_t off = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (P[i] != nullptr) continue;
        Operand in;
        int32_t f = fmt;
        if (e4m3) {
            const void* r = nullptr;
            ST(e4m3_in(ctx, R[i], n[i], WS_E8_IN0, s, &r));
            in.dev = r;
            f = BMLP_FMT_U8;
        } else {
            ST(stage_in(ctx, R[i], fmt_bytes(fmt, n[i], n[i]), WS_IN0, s, &in));
        }
        ST(to_packed(ctx, in, f, n[i], buf + off, ldw[i], s));
        P[i] = buf + off;
        off += static_cast<size_t>(n[i] * ldw[i]);
    }
    return dispatch_choose_many_packed(ctx, P.data(), n, ldw.data(), m, feats, choice, s);
}

bmlp_status bmlp_dispatch_features(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, float* feats, cudaStream_t s) {
    FMT_WRAP_CHECK(fmt);
    if (fmt != BMLP_FMT_E4M3 || !ctx || n <= 0 || !R) return core_dispatch_features(ctx, R, n, fmt == BMLP_FMT_E4M3 ? BMLP_FMT_U8 : fmt, feats, s);
    DeviceGuard g(ctx->device);
    const void* r = nullptr;
    ST(e4m3_in(ctx, R, n, WS_E8_IN0, s, &r));
    return core_dispatch_features(ctx, r, n, BMLP_FMT_U8, feats, s);
}
#undef FMT_WRAP_CHECK
}  // extern "C"

namespace bmlp {
// The bit-row step-cost model, for the device-driven large problems of a grouped batch.
double bitrow_s_per_word() { return sparse_s_per_word(); }
double bitrow_row_s_per_word() { return sparse_row_s_per_word(); }
double bitrow_step_s() { return kSparseStepS; }
double tc4_product_s(int64_t n_pad) { return tc_product_s(n_pad); }
// The restricted squaring's fixed cost, switch, sampled rows and row-count spread, for the device-driven pipelines.
double thin_fixed_seconds(int64_t n_pad) { return thin_fixed_s(n_pad); }
bool thin_is_enabled() { return thin_enabled(); }
int thin_sample_rows() { return kThinSampleRows; }
double thin_row_spread() { return kThinRowSpread; }
}  // namespace bmlp
