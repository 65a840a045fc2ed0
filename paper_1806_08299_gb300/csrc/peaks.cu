// peaks.cu -- microbenchmarks for the ALU and shared-memory roofs
// (include/wave_peaks.h).
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "wave.h"
#include "wave_peaks.h"

namespace {

__device__ float g_peak_sink[16];  // written only for impossible values: keeps results live

constexpr int kThreads = 256;
constexpr int kChains = 8;

// Independent paired-FP32 FMA chains: every thread runs kChains chains of
// `iters` FMAs on two lanes each.
__global__ void __launch_bounds__(kThreads) fma2_kernel(int iters, float2 a, float2 b)
{
    float2 acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = make_float2(1e-7f * threadIdx.x + i, 1e-7f * i);
    for (int n = 0; n < iters; ++n) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc[i] = __ffma2_rn(acc[i], a, b);
    }
    float2 s = acc[0];
#pragma unroll
    for (int i = 1; i < kChains; ++i) s = __fadd2_rn(s, acc[i]);
    if (s.x == 12345.f && s.y == -12345.f) g_peak_sink[0] = s.x;
}

// Conflict-free 16-byte shared loads: in iteration n, load k of thread t
// reads float4 t + 256 ((4n + k) mod 8).  The address changes with n, so the
// compiler cannot keep a loaded value across iterations (with a fixed address
// every load is loop-invariant and may be hoisted, which would time the adds
// instead of the loads).
__global__ void __launch_bounds__(kThreads) lds_kernel(int iters)
{
    __shared__ float4 buf[8 * kThreads];
    for (int k = 0; k < 8; ++k)
        buf[threadIdx.x + kThreads * k] = make_float4(threadIdx.x, k, 1.f, 2.f);
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf + threadIdx.x);
    float2 lo = make_float2(0.f, 0.f), hi = lo;
    for (int n = 0; n < iters; ++n) {
        const uint32_t half = (uint32_t)(n & 1) * (16u * kThreads * 4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 v;
            asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "r"(base + half + 16u * kThreads * k)
                         : "memory");
            lo = __fadd2_rn(lo, make_float2(v.x, v.y));
            hi = __fadd2_rn(hi, make_float2(v.z, v.w));
        }
    }
    if (lo.x == 12345.f && hi.y == -12345.f) g_peak_sink[1] = lo.y + hi.x;
}

}  // namespace

extern "C" int32_t wave_measure_peaks(double *fp32_tflops, double *smem_tbs, void *stream_)
{
    if (fp32_tflops == nullptr || smem_tbs == nullptr) return WAVE_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return WAVE_ECUDA;
    const int blocks = sms * 8;  // 2048 threads per SM
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return WAVE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return WAVE_ECUDA;
    }
    int32_t rc = WAVE_OK;
    float best_fma = 1e30f, best_lds = 1e30f;
    const int fma_iters = 1 << 15, lds_iters = 1 << 13;
    for (int rep = 0; rep < 4 && rc == WAVE_OK; ++rep) {  // rep 0 warms up
        float ms = 0.f;
        cudaEventRecord(e0, stream);
        fma2_kernel<<<blocks, kThreads, 0, stream>>>(fma_iters, make_float2(0.9999999f, 0.9999999f),
                                                     make_float2(1e-7f, 1e-7f));
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = WAVE_ECUDA;
        if (rep > 0) best_fma = std::min(best_fma, ms);
        cudaEventRecord(e0, stream);
        lds_kernel<<<blocks, kThreads, 0, stream>>>(lds_iters);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = WAVE_ECUDA;
        if (rep > 0) best_lds = std::min(best_lds, ms);
    }
    if (cudaGetLastError() != cudaSuccess) rc = WAVE_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != WAVE_OK) return rc;
    const double threads = (double)blocks * kThreads;
    *fp32_tflops = threads * fma_iters * kChains * 2.0 /* lanes */ * 2.0 /* flops */ / (best_fma * 1e-3) / 1e12;
    *smem_tbs = threads * lds_iters * 4.0 * 16.0 / (best_lds * 1e-3) / 1e12;
    return WAVE_OK;
}
