// Issue-rate probes, the ceilings the kernels are measured against besides
// the nominal peaks. Tensor cores: one CTA per SM (or one CTA pair per two
// SMs) issues back-to-back tcgen05.mma instructions on fixed shared-memory
// tiles (all zero) into TMEM, with no operand traffic, for the operand kind a
// squaring kernel uses (kind::f8f6f4 E4M3 M128 N256 K32; kind::mxf4 E2M1 with
// unit UE8M0 scales M128 N256 K64; the same as one M256 N256 K64
// .cta_group::2 MMA per CTA pair). Integer ALU: every thread of 8 resident
// warps per SM scheduler ORs 64-bit words held in registers, the operation
// the bit-row kernels are built from.
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

// The 2-SM form: CTA pairs (2-CTA clusters); the even CTA issues M256 N256 K64
// kind::mxf4 MMAs over both CTAs' tiles and TMEM. With N1 = 224, each K step
// also issues an M256 N224 K64 MMA into columns 256..479 (the squaring
// kernel's 480-column pair tile; scale factors in columns 480..511).
template <int N1>
__global__ void __launch_bounds__(128, 1) __cluster_dims__(2, 1, 1) mma_rate_2sm_kernel(int iters, int* err) {
    extern __shared__ uint8_t raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    __shared__ int abort_flag;
    for (int i = threadIdx.x; i < 48 * 1024 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    const int warp = threadIdx.x >> 5;
    const bool leader = cluster_ctarank() == 0;
    if (warp == 0) {
        tmem_alloc_2sm(&slot, 512);
        tmem_relinquish_2sm();
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t base = slot;
    {
        const uint32_t lanes = static_cast<uint32_t>(warp * 32) << 16;
        const uint32_t ones[8] = {0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu,
                                  0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu};
        if (N1) {
#pragma unroll
            for (int c = 480; c < 512; c += 8) tmem_st_32x32b_x8(base + lanes + c, ones);
        } else {
            tmem_st_32x32b_x8(base + lanes + 256, ones);
            tmem_st_32x32b_x8(base + lanes + 384, ones);
        }
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' tiles, scale factors and barriers are in place
    tc_fence_after();
    if (leader && threadIdx.x == 0) {
        const uint32_t a0 = smem_u32(sm), b0 = smem_u32(sm + 16384), b1 = smem_u32(sm + 32768);
        const uint32_t sfa = base + (N1 ? 480 : 256), sfb = base + (N1 ? 480 : 384);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t da = smem_desc_kmajor_sw128(a0 + k * 32);
                tc_mma_mxf4_2sm(base, da, smem_desc_kmajor_sw128(b0 + k * 32), idesc_mxf4_ue8m0(256, 256), sfa, sfb,
                                1);
                if (N1)
                    tc_mma_mxf4_2sm(base + 256, da, smem_desc_kmajor_sw128(b1 + k * 32), idesc_mxf4_ue8m0(256, N1),
                                    sfa, sfb, 1);
            }
        }
        tc_commit_2sm_mcast(&bar, 0x1);
        if (!mbar_wait_bounded(&bar, 0, &abort_flag, 8000000000LL)) atomicAdd(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // the even CTA's MMAs into this CTA's TMEM have completed
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_2sm(base, 512);
    }
}

// 64-bit word ORs from registers: 8 independent accumulators per thread, each
// OR a dependent step of its chain; `seed` is unknown to the compiler and the
// result is stored, so nothing is folded away.
__global__ void __launch_bounds__(256) or_rate_kernel(int iters, uint64_t seed, uint64_t* sink) {
    uint64_t acc[8], v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        acc[j] = seed * (threadIdx.x + 1 + j);
        v[j] = seed ^ (static_cast<uint64_t>(j) << 32 | blockIdx.x);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int j = 0; j < 8; ++j) asm volatile("or.b64 %0, %0, %1;" : "+l"(acc[j]) : "l"(v[(j + r) & 7]));
        }
    }
    uint64_t x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x ^= acc[j];
    if (x == 0x9E3779B97F4A7C15ull) sink[0] = x;  // practically never true; keeps the chains alive
}

bmlp_status run_probe(bmlp_ctx* ctx, int kind, int iters, double* rate) {
    void* e = nullptr;
    const bmlp_status ws = ws_get(ctx, 26, 16, &e);  // workspace slot of the probe's error word and sink
    if (ws != BMLP_OK) return ws;
    int* err = static_cast<int*>(e);
    cudaError_t ce = cudaSuccess;
    if (kind == 0) ce = cudaFuncSetAttribute(mma_rate_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (kind == 1) ce = cudaFuncSetAttribute(mma_rate_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (kind == 2)
        ce = cudaFuncSetAttribute(mma_rate_2sm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (kind == 4)
        ce = cudaFuncSetAttribute(mma_rate_2sm_kernel<224>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (ce != cudaSuccess) return cuda_err(ctx, ce, "probe attribute");
    const int pairs = ctx->sm_count / 2;
    auto launch = [&](int it) {
        if (kind == 0) mma_rate_kernel<0><<<ctx->sm_count, 128, PROBE_SMEM>>>(it, err);
        if (kind == 1) mma_rate_kernel<1><<<ctx->sm_count, 128, PROBE_SMEM>>>(it, err);
        if (kind == 2) mma_rate_2sm_kernel<0><<<2 * pairs, 128, PROBE_SMEM>>>(it, err);
        if (kind == 4) mma_rate_2sm_kernel<224><<<2 * pairs, 128, PROBE_SMEM>>>(it, err);
        if (kind == 3) or_rate_kernel<<<4 * ctx->sm_count, 256>>>(it, 0x243F6A8885A308D3ull,
                                                                   reinterpret_cast<uint64_t*>(err + 2));
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemset(err, 0, sizeof(int));
    launch(50);  // warm-up
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    int herr = 0;
    if (ce == cudaSuccess) ce = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return cuda_err(ctx, ce, "probe launch");
    if (herr) return set_err(ctx, BMLP_ERR_TIMEOUT, "probe wait timed out");
    double work = 0.0;  // FLOP (tensor kinds) or 64-bit word ORs (kind 3)
    if (kind == 0) work = static_cast<double>(ctx->sm_count) * iters * 4.0 * 2.0 * 128.0 * 256.0 * 32.0;
    if (kind == 1) work = static_cast<double>(ctx->sm_count) * iters * 4.0 * 2.0 * 128.0 * 256.0 * 64.0;
    if (kind == 2) work = static_cast<double>(pairs) * iters * 4.0 * 2.0 * 256.0 * 256.0 * 64.0;
    if (kind == 3) work = 4.0 * ctx->sm_count * 256.0 * static_cast<double>(iters) * 16.0 * 8.0;
    if (kind == 4) work = static_cast<double>(pairs) * iters * 4.0 * 2.0 * 256.0 * 480.0 * 64.0;
    *rate = work / (static_cast<double>(ms) * 1e-3) / 1e12;
    return BMLP_OK;
}

}  // namespace
}  // namespace bmlp

extern "C" bmlp_status bmlp_mma_issue_rate(bmlp_ctx* ctx, int32_t kind, int32_t iters, double* tflops) {
    if (!ctx || !tflops || iters <= 0 || kind < 0 || kind > 4) return BMLP_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const bmlp_status st = bmlp::run_probe(ctx, kind, iters, tflops);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return st;
}
