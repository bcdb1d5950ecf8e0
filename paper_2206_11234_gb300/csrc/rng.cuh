// Counter-based normal generator for the Euler–Maruyama noise xi_m
// (arXiv:2206.11234 §2.1, below Eq. (8): each xi_m is a unit normal; the
// paper does not name a generator).
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter
// (c, id_lo, id_hi, set_id), key (seed_lo, seed_hi).  Steps come in groups of
// sixteen: group G uses the twelve words of the counters 3G, 3G + 1, 3G + 2
// (in that order).  Block j (steps 16G + 4j .. 16G + 4j + 3) takes words 3j,
// 3j + 1, 3j + 2 of the twelve: the radius words of its two Box–Muller pairs
// and a word holding their angles (first pair: high 16 bits, second pair: low
// 16 bits), 48 bits per pair.  Each trajectory's noise is a pure function of
// (seed, set_id, id, m).
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

// The twelve words of 16-step group G: counters 3G, 3G + 1, 3G + 2.
__device__ __forceinline__ void philox_group(const PhiloxLane& l, uint32_t G, const PhiloxKeys& K,
                                             uint32_t V[12]) {
    philox_block(l, 3u * G, K, V);
    philox_block(l, 3u * G + 1u, K, V + 4);
    philox_block(l, 3u * G + 2u, K, V + 8);
}

// The three words of 4-step block k (group k >> 2, j = k & 3) for kernels that
// step four at a time: words 3j .. 3j + 2 of the group lie in one counter
// (j = 0, 3) or two adjacent ones (j = 1, 2).  Both counters are always
// evaluated and the words picked by selects, so lanes at different j do not
// diverge.
struct BlockWords {
    uint32_t rad0, rad1, ang;
};
__device__ __forceinline__ BlockWords block_words(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K) {
    const uint32_t first = 3u * (k & 3u);      // index of the block's first word among the twelve
    const uint32_t c0 = 3u * (k >> 2) + (first >> 2);
    uint32_t a[4], b[4];
    philox_block(l, c0, K, a);
    philox_block(l, c0 + 1u, K, b);
    const uint32_t o = first & 3u;             // 0, 3, 2, 1 for j = 0..3
    const uint32_t w0 = o == 0u ? a[0] : o == 1u ? a[1] : o == 2u ? a[2] : a[3];
    const uint32_t w1 = o == 0u ? a[1] : o == 1u ? a[2] : o == 2u ? a[3] : b[0];
    const uint32_t w2 = o == 0u ? a[2] : o == 1u ? a[3] : o == 2u ? b[0] : b[1];
    return BlockWords{w0, w1, w2};
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

// ---- Box–Muller, binary64: u0 = (w + 1/2) 2^-32 from a radius word, u1 =
// (h + 1/2) 2^-16 from a 16-bit angle field (both exact), r = sqrt(-2 ln u0),
// (r cos 2 pi u1, r sin 2 pi u1) with CUDA's log, sqrt and sincos. ----
__device__ __forceinline__ void box_muller_f64(uint32_t rad, uint32_t ang16, double& z0, double& z1) {
    const double u0 = ((double)rad + 0.5) * 0x1p-32;
    const double u1 = ((double)ang16 + 0.5) * 0x1p-16;
    const double r = sqrt(-2.0 * log(u0));
    const double angle = 6.283185307179586 * u1;
    double s, c;
    sincos(angle, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

__device__ __forceinline__ void normals4_f64(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K,
                                             double xi[4]) {
    const BlockWords w = block_words(l, k, K);
    box_muller_f64(w.rad0, w.ang >> 16, xi[0], xi[1]);
    box_muller_f64(w.rad1, w.ang & 0xffffu, xi[2], xi[3]);
}

// ---- Box–Muller, binary32 (hardware approximations) ----
// u0 = ((w >> 9) + 1/2) 2^-23 is exact in binary32: put the top 23 bits of the
// radius word into the mantissa of 1.0 (a shift-add, the bits do not overlap)
// and subtract 1 - 2^-24 (exact by Sterbenz).  The radius is r = sqrt(-2 ln u0)
// = sqrt(2 ln 2) * rho with rho = sqrt(-log2 u0).  The 16-bit angle field h
// sits in the top 16 bits of an angle word (zeros below), so f = 1 + h 2^-16
// is exact, and the angle is taken as 2 pi u1 - pi = 2 pi f - (3 pi - 2 pi
// 2^-17) in [-pi, pi), where the fast sine/cosine are accurate; sin(2 pi u1 -
// pi) = -sin(2 pi u1), likewise for cos.  A pair of normals is therefore
// xi0 = -sqrt(2 ln 2) rho c,  xi1 = -sqrt(2 ln 2) rho s  with
// (c, s) = (cos, sin)(2 pi u1 - pi).  The stepper works with (rho, c, s) and
// folds the constant -sqrt(2 ln 2) into its own per-run constants, so it never
// forms xi; the values track the binary64 normals to ~1e-6.
constexpr float kSqrt2Ln2 = 1.1774100225154747f;
constexpr float kAngleOffset = (float)(3.0 * 3.141592653589793 - 6.283185307179586 * 0x1p-17);

__device__ __forceinline__ float uniform_f32(uint32_t w) {
    return __int_as_float((w >> 9) + 0x3f800000u) - (1.0f - 0x1p-24f);
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// angle words of a block's two pairs: the high and the low 16 bits of its
// angle word, each moved to the top (zeros below)
__device__ __forceinline__ uint32_t angle_word_first(uint32_t ang) { return ang & 0xffff0000u; }
__device__ __forceinline__ uint32_t angle_word_second(uint32_t ang) { return __byte_perm(ang, 0u, 0x1044); }

struct NormalPair {
    float rho;  // sqrt(-log2 u0)
    float c;    // cos(2 pi u1 - pi)
    float s;    // sin(2 pi u1 - pi)
};

__device__ __forceinline__ NormalPair normal_pair_f32(uint32_t rad, uint32_t angle_word) {
    NormalPair p;
    p.rho = sqrt_approx(-__log2f(uniform_f32(rad)));
    const float f = __int_as_float((angle_word >> 9) + 0x3f800000u);
    const float angle = __fmaf_rn(6.283185307179586f, f, -kAngleOffset);
    __sincosf(angle, &p.s, &p.c);
    return p;
}

// The two pairs of block j of a 16-step group's words.
__device__ __forceinline__ NormalPair group_pair_f32(const uint32_t V[12], int j, int p) {
    const uint32_t ang = V[3 * j + 2];
    return normal_pair_f32(V[3 * j + p], p == 0 ? angle_word_first(ang) : angle_word_second(ang));
}

// The four normals of 4-step block k as values (probe / tests only).
__device__ __forceinline__ void normals4_f32(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K,
                                             float xi[4]) {
    const BlockWords w = block_words(l, k, K);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const NormalPair q = normal_pair_f32(p == 0 ? w.rad0 : w.rad1,
                                             p == 0 ? angle_word_first(w.ang) : angle_word_second(w.ang));
        const float r = -kSqrt2Ln2 * q.rho;
        xi[2 * p] = r * q.c;
        xi[2 * p + 1] = r * q.s;
    }
}

}  // namespace fpt
