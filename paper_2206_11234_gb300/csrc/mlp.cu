// Batched forward and backward of the learned-bias MLP on the tensor cores.
//
// Backward of sum_i g_i b(x_i) for a tile of 128 rows (arXiv:2206.11234 has no
// learned bias; the objective it serves is described with the training step):
//   h1 = tanh(W1 x + b1), z2 = W2 h1 + b2, h2 = tanh(z2), b = w3 . h2 + b3
//   d2 = g w3 (1 - h2^2)          dw3 += g h2,  db3 += g,  db2 += d2
//   dh1 = W2^T d2  (tensor cores)  d1 = dh1 (1 - h1^2)
//   dW2 += d2^T h1 (tensor cores, K = the 128 rows, accumulated in TMEM over tiles)
//   dW1 += d1 x^T, db1 += d1
#include <cuda_runtime.h>

#include <cstdint>

#include "abi_internal.h"
#include "fpt.h"
#include "mlp.cuh"

namespace fpt {
namespace {

constexpr int kFwdTmemCols = 64;
constexpr int kBwdTmemCols = 128;
// Forward CTAs use 64 TMEM columns each: at most 7 can be resident per SM
// (7 x 64 <= 512) because each requests at least this much shared memory.
constexpr size_t kFwdMinSmem = 30 * 1024;

__global__ void __launch_bounds__(128) mlp_forward_kernel(const fpt_mlp_params* __restrict__ P,
                                                          const float* __restrict__ phi,
                                                          const float* __restrict__ N, long long n,
                                                          float* __restrict__ out_b, unsigned* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char s_raw[];
    MlpTile& S = *reinterpret_cast<MlpTile*>(s_raw);
    if ((threadIdx.x >> 5) == 0) {
        tc::tmem_alloc(&S.tmem, kFwdTmemCols);
        tc::tmem_relinquish();
        tc::fence_before_sync();
    }
    mlp_tile_load(S, P);  // ends with __syncthreads (also publishes S.tmem)
    tc::fence_after_sync();
    uint32_t phase = 0;
    const long long tiles = (n + 127) / 128;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long i = t * 128 + threadIdx.x;
        const float p = i < n ? phi[i] : 0.f;
        const float x = i < n ? N[i] : 0.f;
        const float b = mlp_tile_forward(S, p, x, phase);
        if (i < n) out_b[i] = b;
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0 && S.status) atomicOr(status, S.status);
    if ((threadIdx.x >> 5) == 0) {
        if (S.status) tc::mbar_wait(&S.mbar, phase ^ 1u);  // a commit left pending by an expired wait
        tc::tmem_dealloc(S.tmem, kFwdTmemCols);
    }
}

struct MlpBwdSmem {
    MlpTile f;                                      // A = h1 (rows r, K = k), W2 (rows n, K = k)
    alignas(128) unsigned char W2T[64 * 64 * 2];    // rows k, K = n
    alignas(128) unsigned char D2[kTileBytes64];    // delta2: rows r, K = n
    alignas(128) unsigned char D2T[128 * 128 * 2];  // delta2^T: rows n (64..127 zero), K = r
    alignas(128) unsigned char H1T[64 * 128 * 2];   // h1^T: rows k, K = r
    float gw1[kHid][2];
    float gb1[kHid];
    float gb2[kHid];
    float gw3[kHid];
    float gb3;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of v[0..15] over the 32 lanes of the warp, 16 at once: at each step a
// lane keeps one half of its values (the upper half when its lane bit is set)
// and adds its partner's copy of that half, so the values carried halve while
// the lanes summed double.  Returns in lane L the sum of index L >> 1 (lanes
// 2u and 2u + 1 both hold index u).  16 shuffles for 16 sums instead of 80.
// v is overwritten.
__device__ __forceinline__ float warp_sum16(float v[16]) {
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int step = 0; step < 4; ++step) {
        const int o = 16 >> step, h = 8 >> step;
        const bool up = (lane & (unsigned)o) != 0u;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ void store_bf16(unsigned char* base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(128) mlp_backward_kernel(const fpt_mlp_params* __restrict__ P,
                                                           const float* __restrict__ phi,
                                                           const float* __restrict__ N,
                                                           const float* __restrict__ g, long long n,
                                                           float* __restrict__ grad,
                                                           unsigned* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char s_raw[];
    MlpBwdSmem& B = *reinterpret_cast<MlpBwdSmem*>(s_raw);
    MlpTile& S = B.f;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(&S.tmem, kBwdTmemCols);
        tc::tmem_relinquish();
        tc::fence_before_sync();
    }
    // W2^T in its tile, zero padding rows of delta2^T, clear the partial sums
    for (int e = tid; e < 64 * 64; e += blockDim.x) {
        const int nn = e >> 6, k = e & 63;
        *reinterpret_cast<uint16_t*>(B.W2T + tc::kmajor_offset(k, nn, 64)) = P->w[kW2 + nn * kHid + k];
    }
    for (int e = tid; e < 64 * 128 * 2 / 16; e += blockDim.x)
        reinterpret_cast<uint4*>(B.D2T + 64 * 128 * 2)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int j = tid; j < kHid; j += blockDim.x) {
        B.gw1[j][0] = B.gw1[j][1] = 0.f;
        B.gb1[j] = B.gb2[j] = B.gw3[j] = 0.f;
    }
    if (tid == 0) B.gb3 = 0.f;
    mlp_tile_load(S, P);  // fences the generic writes above and synchronises
    tc::fence_after_sync();
    uint32_t phase = 0;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const long long tiles = (n + 127) / 128;
    int done = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++done) {
        const long long i = t * 128 + tid;
        const bool valid = i < n;
        const float gi = valid ? g[i] : 0.f;
        const float x0 = ((valid ? phi[i] : 0.f) - S.norm[0]) * S.norm[1];
        const float x1 = ((valid ? N[i] : 0.f) - S.norm[2]) * S.norm[3];
        // layer 1 into A (rows) and H1T (columns)
        mlp_layer1_to_tile(S, S.A, tid, x0, x1);
#pragma unroll 8
        for (int k = 0; k < kHid; ++k) {
            const uint16_t h = *reinterpret_cast<const uint16_t*>(S.A + tc::kmajor_offset(tid, k, 64));
            *reinterpret_cast<uint16_t*>(B.H1T + tc::kmajor_offset(k, tid, 128)) = h;
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) mlp_issue_z2(S);
        if (S.status != 0u || !tc::mbar_wait(&S.mbar, phase)) S.status = 1u;  // one expiry, not one per tile
        phase ^= 1u;
        tc::fence_after_sync();
        // output layer and delta2
        for (int c = 0; c < 4; ++c) {
            float z[16];
            tc::tmem_ld16(S.tmem + lane_base + 16 * c, z);
            tc::tmem_wait_ld();
            uint32_t q[8];
            float dd[16], gh[16];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const int n0 = 16 * c + e;
                const uint32_t hh = tc::tanh_bf16x2(tc::pack_bf16(z[e] + S.b2[n0], z[e + 1] + S.b2[n0 + 1]));
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int nn = n0 + u;
                    const float h2 = u == 0 ? tc::bf16_lo(hh) : tc::bf16_hi(hh);
                    dd[e + u] = gi * S.w3[nn] * (1.f - h2 * h2);
                    gh[e + u] = gi * h2;
                    store_bf16(B.D2T, tc::kmajor_offset(nn, tid, 128), dd[e + u]);
                }
                q[e / 2] = tc::pack_bf16(dd[e], dd[e + 1]);
            }
            *reinterpret_cast<uint4*>(B.D2 + tc::kmajor_offset(tid, 16 * c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4*>(B.D2 + tc::kmajor_offset(tid, 16 * c + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
            // dw3 += g h2, db2 += delta2, summed over the warp's rows
            const float sw3 = warp_sum16(gh);
            const float sb2 = warp_sum16(dd);
            if ((lane & 1u) == 0u) {
                atomicAdd(&B.gw3[16 * c + (lane >> 1)], sw3);
                atomicAdd(&B.gb2[16 * c + (lane >> 1)], sb2);
            }
        }
        const float sg = warp_sum(gi);
        if (lane == 0) atomicAdd(&B.gb3, sg);
        tc::fence_before_sync();
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t d2 = tc::smem_u32(B.D2), w2t = tc::smem_u32(B.W2T);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // dh1 = delta2 W2 -> columns 0..63
                tc::mma_bf16(S.tmem, tc::smem_desc(d2 + 256 * kk, 128, 1024),
                             tc::smem_desc(w2t + 256 * kk, 128, 1024), kIdescZ2, kk > 0 ? 1u : 0u);
            const uint32_t d2t = tc::smem_u32(B.D2T), h1t = tc::smem_u32(B.H1T);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)  // dW2 += delta2^T h1 -> columns 64..127
                tc::mma_bf16(S.tmem + 64, tc::smem_desc(d2t + 256 * kk, 128, 2048),
                             tc::smem_desc(h1t + 256 * kk, 128, 2048), kIdescZ2,
                             (done > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(&S.mbar);
        }
        if (S.status != 0u || !tc::mbar_wait(&S.mbar, phase)) S.status = 1u;  // one expiry, not one per tile
        phase ^= 1u;
        tc::fence_after_sync();
        // delta1 and the first-layer gradients
        for (int c = 0; c < 4; ++c) {
            float dh[16];
            tc::tmem_ld16(S.tmem + lane_base + 16 * c, dh);
            tc::tmem_wait_ld();
            float d0[16], d1x0[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int k = 16 * c + e;
                const uint16_t hb = *reinterpret_cast<const uint16_t*>(S.A + tc::kmajor_offset(tid, k, 64));
                const float h1 = __uint_as_float((uint32_t)hb << 16);
                const float d1 = dh[e] * (1.f - h1 * h1);
                d0[e] = d1;
                d1x0[e] = d1 * x0;
                dh[e] = d1 * x1;  // dh is dead after this element: reuse it for d1 x1
            }
            // db1 += delta1, dW1 += delta1 x^T, summed over the warp's rows
            const float s0 = warp_sum16(d0), s1 = warp_sum16(d1x0), s2 = warp_sum16(dh);
            if ((lane & 1u) == 0u) {
                const int k = 16 * c + (int)(lane >> 1);
                atomicAdd(&B.gb1[k], s0);
                atomicAdd(&B.gw1[k][0], s1);
                atomicAdd(&B.gw1[k][1], s2);
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_after_sync();
    // dW2 from TMEM rows 0..63 (warps 0 and 1), the vector sums from shared memory
    if (done > 0 && warp < 2) {
        const int nn = 32 * warp + lane;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tc::tmem_ld16(S.tmem + lane_base + 64 + 16 * c, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e) atomicAdd(&grad[kW2 + nn * kHid + 16 * c + e], v[e]);
        }
    }
    if (done > 0) {
        for (int j = tid; j < kHid; j += blockDim.x) {
            atomicAdd(&grad[kW1 + 2 * j], B.gw1[j][0]);
            atomicAdd(&grad[kW1 + 2 * j + 1], B.gw1[j][1]);
            atomicAdd(&grad[kB1 + j], B.gb1[j]);
            atomicAdd(&grad[kB2 + j], B.gb2[j]);
            atomicAdd(&grad[kW3 + j], B.gw3[j]);
        }
        if (tid == 0) atomicAdd(&grad[kB3], B.gb3);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && S.status) atomicOr(status, S.status);
    if (warp == 0) {
        if (S.status) tc::mbar_wait(&S.mbar, phase ^ 1u);  // a commit left pending by an expired wait
        tc::tmem_dealloc(S.tmem, kBwdTmemCols);
    }
}

// Grid for a persistent MLP kernel and a check that its resident CTAs cannot
// ask for more TMEM columns than an SM has (an allocation would then wait for
// a CTA that never exits).
int mlp_grid(const void* func, size_t smem, int tmem_cols, long long tiles, int* grid) {
    int n_sm = 0;
    int rc = device_sm_count(&n_sm);
    if (rc) return rc;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "MLP kernel shared memory");
    int per_sm = 0;
    rc = resident_ctas(func, 128, smem, tmem_cols, &per_sm);
    if (rc) return rc;
    if (per_sm < 1) return fail(FPT_EUNSUPPORTED, "MLP kernel does not fit on an SM");
    const long long full = (long long)per_sm * n_sm;
    *grid = (int)(tiles < full ? (tiles < 1 ? 1 : tiles) : full);
    return FPT_OK;
}

int run_status(unsigned* d_status, cudaStream_t st) {
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaError_t ef = cudaFreeAsync(d_status, st);
    if (e != cudaSuccess) return cuda_fail(e, "MLP status readback");
    if (ef != cudaSuccess) return cuda_fail(ef, "MLP status free");
    if (h) return fail(FPT_EDEVICE_STATUS, "MLP kernel: a tensor-core wait expired (status 0x%x)", h);
    return FPT_OK;
}

}  // namespace

size_t mlp_fwd_smem_bytes() {
    return sizeof(MlpTile) > kFwdMinSmem ? sizeof(MlpTile) : kFwdMinSmem;
}

}  // namespace fpt

using namespace fpt;

namespace fpt {
namespace {
// One warp waits, with the library's bounded wait, on an mbarrier that nobody
// arrives at; it records the expiry and then completes the phase itself, so the
// barrier ends in a clean state.
__global__ void wait_selftest_kernel(unsigned* __restrict__ expired) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
    __syncthreads();
    const bool ok = tc::mbar_wait(&mbar, 0u);
    if (!ok) atomicOr(expired, 1u);
    __syncwarp();
    if (threadIdx.x == 0) tc::mbar_arrive(&mbar);
}
}  // namespace
}  // namespace fpt

extern "C" int fpt_wait_selftest(int32_t* expired_out, double* seconds_out, void* stream) {
    if (!expired_out) return fail(FPT_EINVAL, "expired_out is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned* d = nullptr;
    cudaError_t e = lib_malloc_async(reinterpret_cast<void**>(&d), sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "self-test flag");
    cudaMemsetAsync(d, 0, sizeof(unsigned), st);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    wait_selftest_kernel<<<1, 32, 0, st>>>(d);
    e = cudaGetLastError();
    cudaEventRecord(b, st);
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(d, st);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    *expired_out = (int32_t)h;
    if (seconds_out) *seconds_out = ms / 1e3;
    return FPT_OK;
}

extern "C" int fpt_mlp_forward(const fpt_mlp_params* w, const float* phi, const float* N, int64_t n, float* out_b,
                               void* stream) {
    NvtxRange nvtx_range("fpt_mlp_forward");
    if (n < 0) return fail(FPT_EINVAL, "n %lld < 0", (long long)n);
    if (!w || (n > 0 && (!phi || !N || !out_b))) return fail(FPT_EINVAL, "pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(w) & 15u) != 0) return fail(FPT_EINVAL, "parameters must be 16-byte aligned");
    if (n == 0) return FPT_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = mlp_fwd_smem_bytes();
    int grid = 0;
    int rc = mlp_grid((const void*)mlp_forward_kernel, smem, kFwdTmemCols, (n + 127) / 128, &grid);
    if (rc) return rc;
    unsigned* d_status = nullptr;
    cudaError_t e = lib_malloc_async(reinterpret_cast<void**>(&d_status), sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "MLP status");
    cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
    mlp_forward_kernel<<<grid, 128, smem, st>>>(w, phi, N, (long long)n, out_b, d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(d_status, st);
        return cuda_fail(e, "MLP forward launch");
    }
    return run_status(d_status, st);
}

extern "C" int fpt_mlp_backward(const fpt_mlp_params* w, const float* phi, const float* N, const float* g,
                                int64_t n, float* grad, void* stream) {
    NvtxRange nvtx_range("fpt_mlp_backward");
    if (n < 0) return fail(FPT_EINVAL, "n %lld < 0", (long long)n);
    if (!w || !grad || (n > 0 && (!phi || !N || !g))) return fail(FPT_EINVAL, "pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(w) & 15u) != 0) return fail(FPT_EINVAL, "parameters must be 16-byte aligned");
    if (n == 0) return FPT_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = sizeof(MlpBwdSmem) + 1024;
    int grid = 0;
    int rc = mlp_grid((const void*)mlp_backward_kernel, smem, kBwdTmemCols, (n + 127) / 128, &grid);
    if (rc) return rc;
    unsigned* d_status = nullptr;
    cudaError_t e = lib_malloc_async(reinterpret_cast<void**>(&d_status), sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "MLP status");
    cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
    mlp_backward_kernel<<<grid, 128, smem, st>>>(w, phi, N, g, (long long)n, grad, d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(d_status, st);
        return cuda_fail(e, "MLP backward launch");
    }
    return run_status(d_status, st);
}
