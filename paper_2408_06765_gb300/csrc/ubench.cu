// ubench.cu -- throughput probes of the FP32 pipe and of the multi-function
// unit (MUFU), the two units that bound the FP32C source x target kernels,
// and of the FP64 pipe, which bounds the FP64 stage kernel.  Each thread runs
// 8 independent dependency chains so that issue, not latency, limits the
// rate.
#include "rsi_internal.cuh"

namespace {

template <int KIND>
__global__ void __launch_bounds__(256) ubench_kernel(int iters, float* sink) {
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = 1.0f + 1e-3f * float(threadIdx.x + 32 * c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (KIND == RSI_UB_FFMA) {
                v[c] = fmaf(v[c], 0.999999f, 1e-7f);
            } else if (KIND == RSI_UB_RSQRT) {
                asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
            } else {
                asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += v[c];
    sink[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ubench_dfma_kernel(int iters, float* sink) {
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = 1.0 + 1e-3 * double(threadIdx.x + 32 * c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = fma(v[c], 0.999999999, 1e-9);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += v[c];
    sink[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = float(s);
}

}  // namespace

extern "C" int rsi_ubench(int32_t kind, int32_t blocks, int32_t iters, float* sink, void* stream) {
    if (!sink || blocks < 1 || iters < 1) return rsi_fail(RSI_E_INVAL, "rsi_ubench: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case RSI_UB_FFMA: ubench_kernel<RSI_UB_FFMA><<<blocks, 256, 0, s>>>(iters, sink); break;
        case RSI_UB_RSQRT: ubench_kernel<RSI_UB_RSQRT><<<blocks, 256, 0, s>>>(iters, sink); break;
        case RSI_UB_SIN: ubench_kernel<RSI_UB_SIN><<<blocks, 256, 0, s>>>(iters, sink); break;
        case RSI_UB_DFMA: ubench_dfma_kernel<<<blocks, 256, 0, s>>>(iters, sink); break;
        default: return rsi_fail(RSI_E_INVAL, "rsi_ubench: unknown kind %d", kind);
    }
    RSI_CHECK_LAUNCH("ubench_kernel");
    return RSI_OK;
}
