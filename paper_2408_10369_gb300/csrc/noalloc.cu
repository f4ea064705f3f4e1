// bmlp_rms_tc_noalloc: the tensor-core squaring closure for callers that may
// not allocate device memory. Its scratch (the ping-pong E4M3 R / R^T
// matrices and the control words) lives in one file-scope __device__ array of
// fixed size, so the call itself never allocates.
#include <cstring>
#include <cudaTypedefs.h>
#include <mutex>

#include "internal.h"

namespace bmlp {
namespace {

constexpr int64_t NA_MAX_N = BMLP_NOALLOC_MAX_N;                 // largest padded n
constexpr size_t NA_MAT = static_cast<size_t>(NA_MAX_N) * NA_MAX_N;
constexpr size_t NA_CTL = 256;                                  // control words
constexpr size_t NA_BYTES = 4 * NA_MAT + NA_CTL;                // 16 MiB + 256 B

// The scratch every call on a device shares; each GPU that loads the library
// holds it until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[NA_BYTES];

std::mutex g_mu;
void* g_encode = nullptr;                      // cuTensorMapEncodeTiled

// Device address of the scratch on the current device. In host code the
// array's name is only a handle, so the address comes from
// cudaGetSymbolAddress with the device current. It is looked up on every
// call: the lookup allocates nothing once the module is loaded (the first
// call on a device loads it), and an address kept from an earlier call would
// be stale if the caller had torn down and recreated the device's context.
bmlp_status scratch_on_current_device(int* dev_out, uint8_t** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return BMLP_ERR_CUDA;
    }
    void* addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || addr == nullptr) {
        cudaGetLastError();
        return BMLP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_encode == nullptr) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr) {
            cudaGetLastError();
            return BMLP_ERR_CUDA;
        }
        g_encode = fn;
    }
    *dev_out = dev;
    *out = static_cast<uint8_t*>(addr);
    return BMLP_OK;
}

bool tmap(CUtensorMap* map, const void* base, int64_t n_pad, int box_rows) {
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(g_encode);
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(n_pad), static_cast<cuuint64_t>(n_pad)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(n_pad)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(TC_BK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Device memory of device `dev` (or managed memory): the kernels read and
// write it directly, so host memory and another GPU's memory are refused.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
}  // namespace bmlp

using namespace bmlp;

extern "C" bmlp_status bmlp_rms_tc_noalloc(const void* R, int64_t n, int32_t fmt, void* out, int32_t reflexive,
                                           int32_t max_iters, int32_t* iters_out, cudaStream_t s) {
    if (iters_out) *iters_out = 0;
    if (fmt == BMLP_FMT_I8) fmt = BMLP_FMT_U8;  // same bytes, same meaning
    if (n < 0 || (fmt != BMLP_FMT_U8 && fmt != BMLP_FMT_PACKED64)) return BMLP_ERR_INVALID_ARG;
    if (n == 0) return BMLP_OK;
    if (R == nullptr || out == nullptr) return BMLP_ERR_INVALID_ARG;
    if (n > NA_MAX_N) return BMLP_ERR_UNSUPPORTED;
    int dev = 0;
    uint8_t* base = nullptr;
    bmlp_status st = scratch_on_current_device(&dev, &base);
    if (st != BMLP_OK) return st;
    if (!on_device(R, dev) || !on_device(out, dev)) return BMLP_ERR_INVALID_ARG;
    // SM count and clock rate per device, queried once (the clock-rate query takes about 0.7 ms); concurrent first
    // calls may both query and store the same values
    static int dev_sms[64] = {0}, dev_khz[64] = {0};
    int sms = dev < 64 ? dev_sms[dev] : 0, khz = dev < 64 ? dev_khz[dev] : 0;
    if (sms <= 0 || khz <= 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        if (khz <= 0) khz = 2100000;
        if (dev < 64 && sms > 0) {
            dev_sms[dev] = sms;
            dev_khz[dev] = khz;
        }
    }

    const int64_t n_pad = (n + TC_PAD - 1) / TC_PAD * TC_PAD;
    const size_t mat = static_cast<size_t>(n_pad * n_pad);
    uint8_t* M[2] = {base, base + mat};
    uint8_t* T[2] = {base + 2 * mat, base + 3 * mat};
    int* ctl = reinterpret_cast<int*>(base + 4 * NA_MAT);

    // the encoder writes every byte of R and R^T (padding included)
    if (fmt == BMLP_FMT_U8)
        launch_u8_to_e4m3(static_cast<const uint8_t*>(R), n, M[0], T[0], n_pad, s);
    else
        launch_packed_to_e4m3(static_cast<const uint64_t*>(R), (n + 63) / 64, n, n, M[0], T[0], n_pad, n_pad, s);
    if (cudaGetLastError() != cudaSuccess) return BMLP_ERR_CUDA;

    CUtensorMap mapA[2], mapB[2];
    for (int b = 0; b < 2; ++b)
        if (!tmap(&mapA[b], M[b], n_pad, TC_BM) || !tmap(&mapB[b], T[b], n_pad, TC_BN)) return BMLP_ERR_CUDA;
    TcParams p{};
    p.m_tiles = static_cast<int32_t>(n_pad / TC_BM);
    p.n_tiles = static_cast<int32_t>(n_pad / TC_BN);
    p.k_blocks = static_cast<int32_t>(n_pad / TC_BK);
    p.mode = TC_MODE_RMS;
    p.ld = n_pad;
    p.changed = ctl;
    p.error = ctl + 1;
    p.wait_cycles = static_cast<long long>(2.0e9 * static_cast<double>(khz) * 1e-6);
    const int tiles = p.m_tiles * p.n_tiles;
    const int grid = tiles < sms ? tiles : sms;
    int cap = max_iters;
    if (cap <= 0) {
        cap = 2;
        while ((int64_t(1) << (cap - 2)) < n) ++cap;   // ceil(log2 n) + 2
    }
    int cur = 0, iters = 0;
    bool converged = false;
    for (int it = 0; it < cap; ++it) {
        const int nxt = cur ^ 1;
        int h[2] = {0, 0};
        if (cudaMemsetAsync(ctl, 0, 2 * sizeof(int), s) != cudaSuccess) return BMLP_ERR_CUDA;
        p.old_r = M[cur];
        p.out_r = M[nxt];
        p.out_rt = T[nxt];
        if (launch_tc_product(mapA[cur], mapB[cur], p, grid, s) != cudaSuccess) return BMLP_ERR_CUDA;
        if (cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BMLP_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return BMLP_ERR_CUDA;
        if (h[1] != 0) return BMLP_ERR_TIMEOUT;
        iters = it + 1;
        cur = nxt;
        if (!h[0]) {
            converged = true;
            break;
        }
    }
    if (iters_out) *iters_out = iters;
    if (fmt == BMLP_FMT_U8)
        launch_bytes_to_u8(M[cur], n_pad, n, static_cast<uint8_t*>(out), reflexive, s);
    else
        launch_bytes_to_packed(M[cur], n_pad, n, n, static_cast<uint64_t*>(out), (n + 63) / 64, reflexive, s);
    if (cudaGetLastError() != cudaSuccess) return BMLP_ERR_CUDA;
    return converged ? BMLP_OK : BMLP_ERR_NOT_CONVERGED;
}
