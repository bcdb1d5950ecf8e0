// fpt_pipe_rates: measured throughput of the execution pipes the stepper
// kernels are bound by, on the current device (no paper counterpart; the
// denominators of the kernels' rooflines).
//
// One kernel per pipe, each a loop of one instruction kind over eight
// independent dependency chains per thread, 32 warps per SM on every SM, timed
// with CUDA events after a warm-up launch:
//   - binary64 fused multiply-add (the FP64 pipe: the binary64 stepper),
//   - lg2.approx.f32 (the XU / MUFU pipe: Box–Muller, reciprocal, tanh),
//   - mul.wide.u32, the 32 x 32 -> 64-bit multiply of each Philox round (the
//     fma-heavy pipe),
//   - binary32 fused multiply-add (the FMA pipes).
// Each chain's recurrence keeps its value bounded and data-dependent so the
// loop cannot be folded; the results feed a store that never happens (the
// kernel writes only when a chain reaches a value it cannot reach).
#include <cuda_runtime.h>

#include <cstdint>

#include "abi_internal.h"
#include "fpt.h"

namespace fpt {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

enum PipeOp { kOpDfma = 0, kOpLg2 = 1, kOpWideMul = 2, kOpFfma = 3 };

// target of the store that keeps the loops' results alive (never taken)
__device__ unsigned long long g_pipe_sink;

__device__ __forceinline__ float lg2_approx_f32(float x) {
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long mul_wide_u32(uint32_t a, uint32_t b) {
    unsigned long long p;
    asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    return p;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) pipe_loop(int iters) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (OP == kOpDfma) {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-9 * (double)(t + k);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], 0.9999999999, 1e-10);
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == -1.0) g_pipe_sink = t;
    } else if constexpr (OP == kOpLg2) {
        // x in [1, 2): lg2(x) + 1 stays in [1, 2)
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-6f * (float)((t + k) & 1023);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = lg2_approx_f32(a[k]) + 1.0f;
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == -1.0f) g_pipe_sink = t;
    } else if constexpr (OP == kOpWideMul) {
        uint32_t a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = t * 2654435761u + (uint32_t)k;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                const unsigned long long p = mul_wide_u32(a[k], 0xD2511F53u);
                a[k] = (uint32_t)(p >> 32) ^ (uint32_t)p;
            }
        }
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s ^= a[k];
        if (s == 0x12345678u && t == 0xffffffffu) g_pipe_sink = s;
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-6f * (float)((t + k) & 1023);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], 0.99999f, 1e-5f);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        if (s == -1.0f) g_pipe_sink = t;
    }
}

// operations per second of one loop kernel: warm-up launch, then a timed one
template <int OP>
int time_loop(int grid, int iters, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, double* rate) {
    pipe_loop<OP><<<grid, kThreads, 0, st>>>(iters / 8);
    cudaEventRecord(a, st);
    pipe_loop<OP><<<grid, kThreads, 0, st>>>(iters);
    cudaEventRecord(b, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) return cuda_fail(e, "pipe-rate kernel");
    *rate = (double)grid * kThreads * (double)iters * kChains / (ms * 1e-3);
    return FPT_OK;
}

}  // namespace
}  // namespace fpt

using namespace fpt;

extern "C" int fpt_pipe_rates(fpt_pipe_rates_out* out, void* stream) {
    if (!out) return fail(FPT_EINVAL, "out is NULL");
    int n_sm = 0;
    int rc = device_sm_count(&n_sm);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int grid = n_sm * kBlocksPerSm;
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return cuda_fail(e, "event");
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_fail(e, "event");
    }
    // iteration counts sized for a few tens of milliseconds per kernel on GB300
    rc = time_loop<kOpDfma>(grid, 1 << 13, st, a, b, &out->fp64_fma_per_s);
    if (!rc) rc = time_loop<kOpLg2>(grid, 1 << 16, st, a, b, &out->xu_lg2_per_s);
    if (!rc) rc = time_loop<kOpWideMul>(grid, 1 << 17, st, a, b, &out->wide_mul_per_s);
    if (!rc) rc = time_loop<kOpFfma>(grid, 1 << 18, st, a, b, &out->fp32_fma_per_s);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}
