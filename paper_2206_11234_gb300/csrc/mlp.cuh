// Learned bias b(phi, N) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3 with
// x = ((phi - c_phi) s_phi, (N - c_N) s_N): 2 -> 64 -> 64 -> 1, BF16 parameters,
// FP32 accumulation.  This replaces the hand-picked constant amplitude of the
// bias B = b S (arXiv:2206.11234 §2.3 Eq. (18)) by a function of the state,
// which the paper names as the open problem of its bias optimisation (§3.4, §4).
//
// One tile form, one row per thread of a 128-thread CTA, shared by the
// learned-bias stepper, fpt_mlp_forward and the backward's forward
// recomputation: the 2-wide input layer on the CUDA cores (FP32 FMAs, tanh to
// BF16 straight into the A tile), z2 = W2 h1 on the tensor cores (tcgen05.mma,
// accumulator in TMEM), and tanh(z2 + b2) with the output layer w3 . h2 + b3
// back on the CUDA cores.  One matrix operation per evaluation: the CTA meets
// at one barrier and one mbarrier wait, and every path computes b the same way.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

#include "fpt.h"
#include "tc.cuh"

namespace fpt {

constexpr int kHid = FPT_MLP_HIDDEN;  // 64
// offsets in the packed parameter vector (same order as fpt_mlp_params.w)
constexpr int kW1 = 0, kB1 = kW1 + 2 * kHid, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
              kB3 = kW3 + kHid;
static_assert(kB3 + 1 == FPT_MLP_NPARAM, "parameter layout");

constexpr uint32_t kIdescZ2 = tc::idesc_bf16(128, 64);  // M = 128 rows, N = 64 outputs
constexpr int kTileBytes64 = 128 * 64 * 2;              // 128 rows x K 64, bf16

// Shared-memory state of the tile (per 128-thread CTA): W2 in the tensor-core
// layout, the other parameters as FP32.
struct MlpTile {
    alignas(128) unsigned char A[kTileBytes64];   // h1, rows = threads, K = 64 hidden
    alignas(128) unsigned char W2[64 * 64 * 2];   // rows = output n, K = input k
    float w1[kHid][2];
    float b1[kHid];
    float b2[kHid];
    float w3[kHid];
    float b3;
    float norm[4];
    uint64_t mbar;
    uint32_t tmem;    // TMEM base address (64 columns)
    uint32_t status;  // nonzero: a bounded wait expired
};

__device__ __forceinline__ float bf16_at(const uint16_t* w, int i) {
    return __uint_as_float((uint32_t)w[i] << 16);
}

// Load the parameters into shared memory (W2 in the tensor-core layout);
// all threads of the CTA; ends with a barrier.
__device__ __forceinline__ void mlp_tile_load(MlpTile& S, const fpt_mlp_params* P) {
    const int tid = threadIdx.x;
    for (int i = tid; i < 64 * 8; i += blockDim.x) {  // 16-byte chunks of W2 rows
        const int n = i >> 3, c = i & 7;
        const uint4 v = *reinterpret_cast<const uint4*>(P->w + kW2 + n * kHid + 8 * c);
        *reinterpret_cast<uint4*>(S.W2 + tc::kmajor_offset(n, 8 * c, 64)) = v;
    }
    for (int j = tid; j < kHid; j += blockDim.x) {
        S.w1[j][0] = bf16_at(P->w, kW1 + 2 * j);
        S.w1[j][1] = bf16_at(P->w, kW1 + 2 * j + 1);
        S.b1[j] = bf16_at(P->w, kB1 + j);
        S.b2[j] = bf16_at(P->w, kB2 + j);
        S.w3[j] = bf16_at(P->w, kW3 + j);
    }
    if (tid == 0) {
        S.b3 = bf16_at(P->w, kB3);
        for (int i = 0; i < 4; ++i) S.norm[i] = P->norm[i];
        S.status = 0u;
        tc::mbar_init(&S.mbar, 1);
        tc::mbar_init_fence();
    }
    tc::fence_proxy_async();
    __syncthreads();
}

// First layer of row `row` (this thread) into the A tile: h1 = tanh(W1 x + b1),
// two units per MUFU operation (bf16x2 tanh; the tile holds bf16 anyway).
__device__ __forceinline__ void mlp_layer1_to_tile(const MlpTile& S, unsigned char* A, int row, float x0,
                                                   float x1) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t q[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int j = 8 * c + 2 * p;
            const float a0 = fmaf(S.w1[j][0], x0, fmaf(S.w1[j][1], x1, S.b1[j]));
            const float a1 = fmaf(S.w1[j + 1][0], x0, fmaf(S.w1[j + 1][1], x1, S.b1[j + 1]));
            q[p] = tc::tanh_bf16x2(tc::pack_bf16(a0, a1));
        }
        *reinterpret_cast<uint4*>(A + tc::kmajor_offset(row, 8 * c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
}

// Issue z2 = h1 W2^T for the tile (one thread) and commit to the mbarrier.
__device__ __forceinline__ void mlp_issue_z2(MlpTile& S) {
    tc::fence_after_sync();
    const uint32_t a = tc::smem_u32(S.A), b = tc::smem_u32(S.W2);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)  // K = 64 in steps of 16 (two core matrices = 256 bytes)
        tc::mma_bf16(S.tmem, tc::smem_desc(a + 256 * kk, 128, 1024), tc::smem_desc(b + 256 * kk, 128, 1024),
                     kIdescZ2, kk > 0 ? 1u : 0u);
    tc::mma_commit(&S.mbar);
}

// All threads: publish this thread's operand writes, let thread 0 issue the
// MMAs of `issue` and commit them, wait for the commit (bounded).
template <class Issue>
__device__ __forceinline__ void mlp_tile_mma(MlpTile& S, uint32_t& phase, Issue issue) {
    tc::fence_before_sync();
    tc::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        issue();
        tc::mma_commit(&S.mbar);
    }
    if (S.status != 0u || !tc::mbar_wait(&S.mbar, phase)) S.status = 1u;  // one expiry, not one per tile
    phase ^= 1u;
    tc::fence_after_sync();
}

// b(phi, N) for every row of the tile: one call per thread of the 128-thread
// CTA, all threads together.  `phase` is the mbarrier parity to wait for (all
// threads keep the same value).  The A tile is free again when this returns.
__device__ __forceinline__ float mlp_tile_forward(MlpTile& S, float phi, float N, uint32_t& phase) {
    const int tid = threadIdx.x;
    const float x0 = (phi - S.norm[0]) * S.norm[1];
    const float x1 = (N - S.norm[2]) * S.norm[3];
    mlp_layer1_to_tile(S, S.A, tid, x0, x1);
    // z2 = W2 h1 (b2 is added below)
    mlp_tile_mma(S, phase, [&] {
        const uint32_t a = tc::smem_u32(S.A), w2 = tc::smem_u32(S.W2);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)  // K = 64 in steps of 16 (two core matrices = 256 bytes)
            tc::mma_bf16(S.tmem, tc::smem_desc(a + 256 * kk, 128, 1024), tc::smem_desc(w2 + 256 * kk, 128, 1024),
                         kIdescZ2, kk > 0 ? 1u : 0u);
    });
    // h2 = tanh(z2 + b2) in BF16 (two units per MUFU operation), b = w3 . h2 + b3
    const uint32_t taddr = S.tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16);
    float b = S.b3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float z[16];
        tc::tmem_ld16(taddr + 16 * c, z);
        tc::tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
            const int n0 = 16 * c + e;
            const uint32_t hh = tc::tanh_bf16x2(tc::pack_bf16(z[e] + S.b2[n0], z[e + 1] + S.b2[n0 + 1]));
            b = fmaf(S.w3[n0], tc::bf16_lo(hh), b);
            b = fmaf(S.w3[n0 + 1], tc::bf16_hi(hh), b);
        }
    }
    tc::fence_before_sync();
    return b;
}

}  // namespace fpt
