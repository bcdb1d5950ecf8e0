// Counter-based normal generator for the Euler–Maruyama noise xi_m
// (arXiv:2206.11234 §2.1, below Eq. (8): each xi_m is a unit normal; the
// paper does not name a generator).
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter
// (k, id_lo, id_hi, set_id), key (seed_lo, seed_hi); one block gives the
// normals of steps 4k..4k+3 of trajectory `id` by Box–Muller.  Each
// trajectory's noise is therefore a pure function of (seed, set_id, id, m).
#pragma once
#include <cstdint>

namespace fpt {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Round keys of Philox4x32-10 for one seed: key r = (seed_lo + r W0, seed_hi + r W1).
// Computed once on the host and passed by value as a kernel parameter, so each
// round XORs a constant-bank operand instead of recomputing its key.
struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys k;
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = (uint32_t)seed + (uint32_t)r * kPhiloxW0;
        k.k1[r] = (uint32_t)(seed >> 32) + (uint32_t)r * kPhiloxW1;
    }
    return k;
}

// Per-trajectory part of Philox round 1.  Round 1 multiplies counter word 2
// (id_hi) and XORs word 1 (id_lo) and word 3 (set_id): those do not change
// along a trajectory, so they are folded once at refill.
struct PhiloxLane {
    uint32_t r1_x0;  // hi(M1 * id_hi) ^ id_lo ^ key0
    uint32_t r1_x1;  // lo(M1 * id_hi)
    uint32_t r1_set; // set_id ^ key1
};

__device__ __forceinline__ PhiloxLane philox_lane(uint64_t id, uint32_t set_id, const PhiloxKeys& K) {
    const uint64_t p = (uint64_t)kPhiloxM1 * (uint32_t)(id >> 32);
    PhiloxLane l;
    l.r1_x0 = (uint32_t)(p >> 32) ^ (uint32_t)id ^ K.k0[0];
    l.r1_x1 = (uint32_t)p;
    l.r1_set = set_id ^ K.k1[0];
    return l;
}

__device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                             uint32_t k0, uint32_t k1) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * x0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * x2;
    const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    x1 = (uint32_t)p1;
    x3 = (uint32_t)p0;
    x0 = y0;
    x2 = y2;
}

// Philox4x32-10 of counter (k, id_lo, id_hi, set_id): round 1 from the lane's
// folded words, rounds 2..10 with the precomputed keys.
__device__ __forceinline__ void philox_block(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K,
                                             uint32_t w[4]) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * k;
    uint32_t x0 = l.r1_x0;
    uint32_t x1 = l.r1_x1;
    uint32_t x2 = (uint32_t)(p0 >> 32) ^ l.r1_set;
    uint32_t x3 = (uint32_t)p0;
#pragma unroll
    for (int r = 1; r < 10; ++r) philox_round(x0, x1, x2, x3, K.k0[r], K.k1[r]);
    w[0] = x0;
    w[1] = x1;
    w[2] = x2;
    w[3] = x3;
}

// Plain (unfolded) Philox4x32-10 of an arbitrary counter; used by the RNG
// self-test entry of the library.
__device__ __forceinline__ void philox4x32_10(const uint32_t c[4], uint32_t key0, uint32_t key1,
                                              uint32_t w[4]) {
    uint32_t x0 = c[0], x1 = c[1], x2 = c[2], x3 = c[3];
#pragma unroll
    for (int r = 0; r < 10; ++r)
        philox_round(x0, x1, x2, x3, key0 + (uint32_t)r * kPhiloxW0, key1 + (uint32_t)r * kPhiloxW1);
    w[0] = x0;
    w[1] = x1;
    w[2] = x2;
    w[3] = x3;
}

// ---- Box–Muller, binary64: u = (w + 1/2) 2^-32 (exact), r = sqrt(-2 ln u0),
// (r cos 2 pi u1, r sin 2 pi u1) with CUDA's log, sqrt and sincos. ----
__device__ __forceinline__ void box_muller_f64(uint32_t w0, uint32_t w1, double& z0, double& z1) {
    const double u0 = ((double)w0 + 0.5) * 0x1p-32;
    const double u1 = ((double)w1 + 0.5) * 0x1p-32;
    const double r = sqrt(-2.0 * log(u0));
    const double angle = 6.283185307179586 * u1;
    double s, c;
    sincos(angle, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

__device__ __forceinline__ void normals4_f64(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K,
                                             double xi[4]) {
    uint32_t w[4];
    philox_block(l, k, K, w);
    box_muller_f64(w[0], w[1], xi[0], xi[1]);
    box_muller_f64(w[2], w[3], xi[2], xi[3]);
}

// ---- Box–Muller, binary32 (hardware approximations) ----
// u = ((w >> 9) + 1/2) 2^-23 is exact in binary32: put the top 23 bits into
// the mantissa of 1.0 (a shift-add, the bits do not overlap) and subtract
// 1 - 2^-24 (exact by Sterbenz).  The radius is r = sqrt(-2 ln u0) =
// sqrt(2 ln 2) * rho with rho = sqrt(-log2 u0); the angle is taken as
// 2 pi u1 - pi in [-pi, pi), where the fast sine/cosine are accurate, and
// sin(2 pi u1 - pi) = -sin(2 pi u1), likewise for cos.  A pair of normals is
// therefore  xi0 = -sqrt(2 ln 2) rho c,  xi1 = -sqrt(2 ln 2) rho s  with
// (c, s) = (cos, sin)(2 pi u1 - pi).  The stepper works with (rho, c, s) and
// folds the constant -sqrt(2 ln 2) into its own per-run constants, so it never
// forms xi; the values track the binary64 normals to ~1e-6.
constexpr float kSqrt2Ln2 = 1.1774100225154747f;

__device__ __forceinline__ float uniform_f32(uint32_t w) {
    return __int_as_float((w >> 9) + 0x3f800000u) - (1.0f - 0x1p-24f);
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct NormalPair {
    float rho;  // sqrt(-log2 u0)
    float c;    // cos(2 pi u1 - pi)
    float s;    // sin(2 pi u1 - pi)
};

__device__ __forceinline__ NormalPair normal_pair_f32(uint32_t w0, uint32_t w1) {
    NormalPair p;
    p.rho = sqrt_approx(-__log2f(uniform_f32(w0)));
    // 2 pi u1 - pi = 2 pi f - (pi + 2 pi (1 - 2^-24)) with f = 1 + (w1 >> 9) 2^-23: one rounding
    const float f = __int_as_float((w1 >> 9) + 0x3f800000u);
    const float angle = __fmaf_rn(6.283185307179586f, f, -9.424777586f);
    __sincosf(angle, &p.s, &p.c);
    return p;
}

// The four normals of one Philox block as values (probe / tests only).
__device__ __forceinline__ void normals4_f32(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K,
                                             float xi[4]) {
    uint32_t w[4];
    philox_block(l, k, K, w);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const NormalPair q = normal_pair_f32(w[2 * p], w[2 * p + 1]);
        const float r = -kSqrt2Ln2 * q.rho;
        xi[2 * p] = r * q.c;
        xi[2 * p + 1] = r * q.s;
    }
}

}  // namespace fpt
