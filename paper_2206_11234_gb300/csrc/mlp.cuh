// Learned bias b(phi, N) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3 with
// x = ((phi - c_phi) s_phi, (N - c_N) s_N): 2 -> 64 -> 64 -> 1, BF16 parameters,
// FP32 accumulation.  This replaces the hand-picked constant amplitude of the
// bias B = b S (arXiv:2206.11234 §2.3 Eq. (18)) by a function of the state,
// which the paper names as the open problem of its bias optimisation (§3.4, §4).
//
// Two tile forms, one row per thread of a 128-thread CTA:
//  * MlpTile (inference: the learned-bias stepper and fpt_mlp_forward): all
//    three layers run on the tensor cores (tcgen05.mma, accumulator in TMEM).
//    The 2-wide input goes in as a K = 16 tile [x0_hi, x0_lo, x1_hi, x1_lo, 1,
//    0, ...] (x = hi + lo in two BF16 parts, ~17 significant bits) against
//    W1 rows [w_n0, w_n0, w_n1, w_n1, b1_n, 0, ...]; the same tile supplies the
//    constant 1 that adds b2 and b3 to the second and third layers.  Per row
//    the CUDA cores only convert the accumulators to BF16 and apply tanh.
//  * MlpFwdSmem (the backward kernel's forward recomputation): the 2-wide
//    input layer and the output layer on the CUDA cores, W2 on the tensor cores.
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

// Shared-memory state of the backward kernel's forward recomputation (per
// 128-thread CTA): W2 on the tensor cores, layers 1 and 3 on the CUDA cores.
struct MlpFwdSmem {
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
__device__ __forceinline__ void mlp_fwd_load(MlpFwdSmem& S, const fpt_mlp_params* P) {
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
__device__ __forceinline__ void mlp_layer1_to_tile(const MlpFwdSmem& S, unsigned char* A, int row, float x0,
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
__device__ __forceinline__ void mlp_issue_z2(MlpFwdSmem& S) {
    tc::fence_after_sync();
    const uint32_t a = tc::smem_u32(S.A), b = tc::smem_u32(S.W2);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)  // K = 64 in steps of 16 (two core matrices = 256 bytes)
        tc::mma_bf16(S.tmem, tc::smem_desc(a + 256 * kk, 128, 1024), tc::smem_desc(b + 256 * kk, 128, 1024),
                     kIdescZ2, kk > 0 ? 1u : 0u);
    tc::mma_commit(&S.mbar);
}

constexpr uint32_t kIdescN16 = tc::idesc_bf16(128, 16);  // M = 128 rows, N = 16 (output layer, column 0 used)
constexpr int kTileBytes16 = 128 * 16 * 2;                // 128 rows x K 16, bf16

// Shared-memory state of the tensor-core forward tile (per 128-thread CTA).
// Every operand is K-major without swizzle (tc.cuh); K = 16 tiles have
// SBO = 256, K = 64 tiles SBO = 1024.
struct MlpTile {
    alignas(128) unsigned char A[kTileBytes64];    // h1, then h2: rows = threads, K = 64 hidden units
    alignas(128) unsigned char X[kTileBytes16];    // rows = threads: x0_hi, x0_lo, x1_hi, x1_lo, 1, 0 ...
    alignas(128) unsigned char W1[64 * 16 * 2];    // rows = units n: w_n0, w_n0, w_n1, w_n1, b1_n, 0 ...
    alignas(128) unsigned char W2[64 * 64 * 2];    // rows = units n, K = input unit k
    alignas(128) unsigned char W2b[64 * 16 * 2];   // rows = units n: b2_n in column 4
    alignas(128) unsigned char W3[16 * 64 * 2];    // row 0 = w3, rows 1..15 zero
    alignas(128) unsigned char W3b[16 * 16 * 2];   // row 0: b3 in column 4
    float norm[4];
    uint64_t mbar;
    uint32_t tmem;    // TMEM base address (64 columns)
    uint32_t status;  // nonzero: a bounded wait expired
};

__device__ __forceinline__ uint32_t bf16_pair(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Write the constant operand tiles (all threads of the CTA; ends with a barrier).
__device__ __forceinline__ void mlp_tile_load(MlpTile& S, const fpt_mlp_params* P) {
    const int tid = threadIdx.x;
    const uint16_t* w = P->w;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < 64 * 8; i += blockDim.x) {  // W2 and W3 (row 0), 16-byte chunks of 8 bf16
        const int n = i >> 3, c = i & 7;
        *reinterpret_cast<uint4*>(S.W2 + tc::kmajor_offset(n, 8 * c, 64)) =
            *reinterpret_cast<const uint4*>(w + kW2 + n * kHid + 8 * c);
        if (n < 16)
            *reinterpret_cast<uint4*>(S.W3 + tc::kmajor_offset(n, 8 * c, 64)) =
                n == 0 ? *reinterpret_cast<const uint4*>(w + kW3 + 8 * c) : z;
    }
    for (int n = tid; n < 64; n += blockDim.x) {  // W1 with b1, W2b, W3b: one row each
        *reinterpret_cast<uint4*>(S.W1 + tc::kmajor_offset(n, 0, 16)) =
            make_uint4(bf16_pair(w[kW1 + 2 * n], w[kW1 + 2 * n]), bf16_pair(w[kW1 + 2 * n + 1], w[kW1 + 2 * n + 1]),
                       bf16_pair(w[kB1 + n], 0), 0u);
        *reinterpret_cast<uint4*>(S.W1 + tc::kmajor_offset(n, 8, 16)) = z;
        *reinterpret_cast<uint4*>(S.W2b + tc::kmajor_offset(n, 0, 16)) = make_uint4(0u, 0u, bf16_pair(w[kB2 + n], 0), 0u);
        *reinterpret_cast<uint4*>(S.W2b + tc::kmajor_offset(n, 8, 16)) = z;
        if (n < 16) {
            *reinterpret_cast<uint4*>(S.W3b + tc::kmajor_offset(n, 0, 16)) =
                n == 0 ? make_uint4(0u, 0u, bf16_pair(w[kB3], 0), 0u) : z;
            *reinterpret_cast<uint4*>(S.W3b + tc::kmajor_offset(n, 8, 16)) = z;
        }
    }
    for (int r = tid; r < 128; r += blockDim.x)  // X columns 8..15 stay zero
        *reinterpret_cast<uint4*>(S.X + tc::kmajor_offset(r, 8, 16)) = z;
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) S.norm[i] = P->norm[i];
        S.status = 0u;
        tc::mbar_init(&S.mbar, 1);
        tc::mbar_init_fence();
    }
    tc::fence_proxy_async();
    __syncthreads();
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

// tanh of the 64 accumulator columns of this thread's row into row `row` of
// the A tile, two units per conversion and per MUFU operation (bf16x2).
__device__ __forceinline__ void mlp_tile_tanh_to_A(MlpTile& S, uint32_t taddr, int row) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float z[16];
        tc::tmem_ld16(taddr + 16 * c, z);
        tc::tmem_wait_ld();
        uint32_t q[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) q[i] = tc::tanh_bf16x2(tc::pack_bf16(z[2 * i], z[2 * i + 1]));
        *reinterpret_cast<uint4*>(S.A + tc::kmajor_offset(row, 16 * c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
        *reinterpret_cast<uint4*>(S.A + tc::kmajor_offset(row, 16 * c + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
    }
}

// b(phi, N) for every row of the tile: one call per thread of the 128-thread
// CTA, all threads together.  `phase` is the mbarrier parity to wait for (all
// threads keep the same value).  The A tile is free again when this returns.
__device__ __forceinline__ float mlp_tile_forward(MlpTile& S, float phi, float N, uint32_t& phase) {
    const int tid = threadIdx.x;
    const float x0 = (phi - S.norm[0]) * S.norm[1];
    const float x1 = (N - S.norm[2]) * S.norm[3];
    const uint32_t hi = tc::pack_bf16(x0, x1);
    const uint32_t lo = tc::pack_bf16(x0 - tc::bf16_lo(hi), x1 - tc::bf16_hi(hi));  // exact differences
    *reinterpret_cast<uint4*>(S.X + tc::kmajor_offset(tid, 0, 16)) =
        make_uint4(__byte_perm(hi, lo, 0x5410), __byte_perm(hi, lo, 0x7632), 0x3f80u /* 1.0, 0 */, 0u);
    const uint32_t x = tc::smem_u32(S.X), a = tc::smem_u32(S.A);
    const uint32_t taddr = S.tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16);
    // z1 = W1 x + b1
    mlp_tile_mma(S, phase, [&] {
        tc::mma_bf16(S.tmem, tc::smem_desc(x, 128, 256), tc::smem_desc(tc::smem_u32(S.W1), 128, 256), kIdescZ2, 0u);
    });
    mlp_tile_tanh_to_A(S, taddr, tid);
    // z2 = W2 h1 + b2
    mlp_tile_mma(S, phase, [&] {
        const uint32_t w2 = tc::smem_u32(S.W2);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_bf16(S.tmem, tc::smem_desc(a + 256 * kk, 128, 1024), tc::smem_desc(w2 + 256 * kk, 128, 1024),
                         kIdescZ2, kk > 0 ? 1u : 0u);
        tc::mma_bf16(S.tmem, tc::smem_desc(x, 128, 256), tc::smem_desc(tc::smem_u32(S.W2b), 128, 256), kIdescZ2, 1u);
    });
    mlp_tile_tanh_to_A(S, taddr, tid);
    // b = w3 . h2 + b3 (column 0 of an N = 16 accumulator)
    mlp_tile_mma(S, phase, [&] {
        const uint32_t w3 = tc::smem_u32(S.W3);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_bf16(S.tmem, tc::smem_desc(a + 256 * kk, 128, 1024), tc::smem_desc(w3 + 256 * kk, 128, 1024),
                         kIdescN16, kk > 0 ? 1u : 0u);
        tc::mma_bf16(S.tmem, tc::smem_desc(x, 128, 256), tc::smem_desc(tc::smem_u32(S.W3b), 128, 256), kIdescN16, 1u);
    });
    const float b = tc::tmem_ld1(taddr);
    tc::tmem_wait_ld();
    tc::fence_before_sync();
    return b;
}

}  // namespace fpt
