// Tensor-core issue-rate probe: one CTA per SM issues back-to-back tcgen05.mma
// instructions on fixed shared-memory tiles (all zero) into TMEM, with no
// operand traffic. Its FLOP rate is the ceiling the squaring kernels are
// measured against besides the nominal peaks: it shows what this part issues
// for the operand kind the kernel uses (kind::f8f6f4 E4M3, M128 N256 K32, or
// kind::mxf4 E2M1 with unit UE8M0 scales, M128 N256 K64).
#include "internal.h"
#include "ptx.cuh"

namespace bmlp {
namespace {

constexpr int PROBE_SMEM = 130 * 1024;  // forces one CTA per SM (the operand tiles use 48 KB)

template <int KIND>
__global__ void __launch_bounds__(128, 1) mma_rate_kernel(int iters, int* err) {
    extern __shared__ uint8_t raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    __shared__ int abort_flag;
    for (int i = threadIdx.x; i < 48 * 1024 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        tmem_alloc(&slot, 512);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zero tiles are visible to the MMA
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t base = slot;
    {
        const uint32_t lanes = static_cast<uint32_t>(warp * 32) << 16;
        const uint32_t ones[8] = {0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu,
                                  0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu};
        tmem_st_32x32b_x8(base + lanes + 256, ones);
        tmem_st_32x32b_x8(base + lanes + 384, ones);
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t a0 = smem_u32(sm), b0 = smem_u32(sm + 16384);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t da = smem_desc_kmajor_sw128(a0 + k * 32), db = smem_desc_kmajor_sw128(b0 + k * 32);
                if (KIND == 0)
                    tc_mma_f8(base, da, db, idesc_e4m3_f32(128, 256), 1);
                else
                    tc_mma_mxf4(base, da, db, idesc_mxf4_ue8m0(128, 256), base + 256, base + 384, 1);
            }
        }
        tc_commit(&bar);
        if (!mbar_wait_bounded(&bar, 0, &abort_flag, 8000000000LL)) atomicAdd(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(base, 512);
    }
}

template <int KIND>
bmlp_status run_probe(bmlp_ctx* ctx, int iters, double* tflops) {
    void* e = nullptr;
    const bmlp_status ws = ws_get(ctx, 26, 16, &e);  // workspace slot of the probe's error word
    if (ws != BMLP_OK) return ws;
    int* err = static_cast<int*>(e);
    if (cudaFuncSetAttribute(mma_rate_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM) !=
        cudaSuccess)
        return cuda_err(ctx, cudaGetLastError(), "probe attribute");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemset(err, 0, sizeof(int));
    mma_rate_kernel<KIND><<<ctx->sm_count, 128, PROBE_SMEM>>>(50, err);  // warm-up
    cudaEventRecord(e0);
    mma_rate_kernel<KIND><<<ctx->sm_count, 128, PROBE_SMEM>>>(iters, err);
    cudaEventRecord(e1);
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    int herr = 0;
    if (ce == cudaSuccess) ce = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return cuda_err(ctx, ce, "probe launch");
    if (herr) return set_err(ctx, BMLP_ERR_TIMEOUT, "probe wait timed out");
    const double k = KIND == 0 ? 32.0 : 64.0;
    const double flop = static_cast<double>(ctx->sm_count) * iters * 4.0 * 2.0 * 128.0 * 256.0 * k;
    *tflops = flop / (static_cast<double>(ms) * 1e-3) / 1e12;
    return BMLP_OK;
}

}  // namespace
}  // namespace bmlp

extern "C" bmlp_status bmlp_mma_issue_rate(bmlp_ctx* ctx, int32_t kind, int32_t iters, double* tflops) {
    if (!ctx || !tflops || iters <= 0 || (kind != 0 && kind != 1)) return BMLP_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const bmlp_status st = kind == 0 ? bmlp::run_probe<0>(ctx, iters, tflops) : bmlp::run_probe<1>(ctx, iters, tflops);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return st;
}
