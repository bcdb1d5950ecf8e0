// Persistent Euler–Maruyama first-passage stepper (arXiv:2206.11234 §2.2).
//
// One lane = one run.  A run's state (phi, step count, the running sum of its
// normals) lives in registers.  Lanes advance in scheduling blocks of KS
// steps with no per-step control flow: each step is the biased EM update of
// §2.2 Eq. (11) followed by the reflecting wall, and the lane keeps the
// minimum phi of the block.  At the block end a lane whose minimum reached
// phi_end (first passage, §2.1 below Eq. (8)) or whose step count reached the
// censoring cap has finished somewhere inside the block: it pushes its
// block-start state onto its warp's replay queue in shared memory and refills
// at once from a global ticket counter (one atomicAdd per warp), so a warp
// keeps 32 live runs whatever their lengths (persistent scheduler).  When 32
// finished runs are queued, the warp replays their blocks together, step by
// step with a test after each step — bit-identical arithmetic, the same
// Philox counters — to find the exact step, interpolates the crossing time in
// binary64 and writes the records.  Replays thus run with all 32 lanes busy
// instead of stalling a warp once per finished run.
//
// Log-weight (§2.2 Eqs. (12)-(14), sign as derived from Eqs. (13)-(14)):
// with B = b S the step term is -(b xi sqrt(dN) + b^2 dN / 2), so a run of M
// steps has ln w = -b sqrt(dN) W - b^2 M dN / 2 with W = sum xi.  W is summed
// per block in the state precision and folded into a running sum that is
// either compensated binary32 (Kahan) or binary64.  With the power-law bias
// B = A_p phi^p (§3.4 Eq. (26)) the amplitude B/S changes every step, so the
// power models sum the step log-weights themselves instead of the normals.
#pragma once
#include <cstdint>

#include "rng.cuh"
#include "stepper_types.h"

namespace fpt {

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// minimum of three binary32 values in one instruction (sm_100 and later)
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float y;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
    return y;
}


// ---------------------------------------------------------------------------
// Model steps.  phi' = phi + (D + b S) dN + S xi sqrt(dN)   (§2.2 Eq. (11))
// ---------------------------------------------------------------------------
template <typename Real, int MODEL>
struct ModelStep;

// Quadratic potential, binary32.  The increment is formed on its own and then
// added: dphi = phi t - 2 dN / phi with t = b c m dN + c m sqrt(dN) xi.
// (Folding the bias into a factor 1 + b c m dN would round b c m dN ~ 1e-6 on
// the 2^-23 grid of numbers near 1, i.e. change b by ~1%, which the weights
// would not know about.)  t is formed from a Box–Muller pair as
// fma(kq rho, c, tc) with kq = -sqrt(2 ln 2) c m sqrt(dN) (rng.cuh), so xi is
// never formed.  Explicit intrinsics fix the rounding so the replay of a block
// reproduces it bit for bit.
template <>
struct ModelStep<float, FPT_MODEL_QUADRATIC> {
    float tc, kq, m2dN;  // tc = b c m dN (the bias part of t), kq, m2dN = -2 dN
    __device__ __forceinline__ void load(const SetConst& s) {
        tc = s.f_c1;
        kq = s.f_c2;
        m2dN = s.f_c3;
    }
    __device__ __forceinline__ float step(float phi, float t) const {
        const float inv = rcp_approx(phi);
        const float v = __fmul_rn(m2dN, inv);
        return __fadd_rn(phi, __fmaf_rn(phi, t, v));
    }
};

// The same step in the scaled variable psi = phi / sqrt(2 dN), used by the
// constant-bias stepper: multiplying phi' = phi + phi t - 2 dN / phi by
// 1/sqrt(2 dN) gives psi' = psi + (psi t - 1/psi), so the drift needs no
// multiply.  The increment is still formed on its own (one rounding) and then
// added.  Crossing and wall tests compare psi with the scaled phi_end and
// 2 phi_uv of the set table; the crossing fraction is scale-free.
struct QuadPsiStep {
    float tc, kq;  // as in ModelStep<float, FPT_MODEL_QUADRATIC>
    __device__ __forceinline__ void load(const SetConst& s) {
        tc = s.f_c1;
        kq = s.f_c2;
    }
    __device__ __forceinline__ float step(float psi, float t) const {
        return __fadd_rn(psi, __fmaf_rn(psi, t, -rcp_approx(psi)));
    }
};

// Constant drift a0 and noise s0, binary32: dphi = t = (a0 + b s0) dN + s0 sqrt(dN) xi.
template <>
struct ModelStep<float, FPT_MODEL_CONSTANT> {
    float tc, kq;  // tc = (a0 + b s0) dN, kq = -sqrt(2 ln 2) s0 sqrt(dN)
    __device__ __forceinline__ void load(const SetConst& s) {
        tc = s.f_c1;
        kq = s.f_c2;
    }
    __device__ __forceinline__ float step(float phi, float t) const { return __fadd_rn(phi, t); }
};

// Polynomial potential V = sum_k c_k phi^k (§2.3 Eq. (17), M_Pl = 1), binary32:
// D = -V'/V and S = sqrt(V) / (2 pi sqrt 3), and the step is
// dphi = S t + D dN with t = b dN + sqrt(dN) xi (so the bias is B = b S).  The
// coefficients are read from the set table in shared memory.
template <>
struct ModelStep<float, FPT_MODEL_POLYNOMIAL> {
    float tc, kq, dN;   // tc = b dN, kq = -sqrt(2 ln 2) sqrt(dN), dN
    const float* c;     // V
    const float* dc;    // V'
    __device__ __forceinline__ void load(const SetConst& s) {
        tc = s.f_c1;
        kq = s.f_c2;
        dN = s.f_c3;
        c = s.f_poly;
        dc = s.f_dpoly;
    }
    __device__ __forceinline__ float step(float phi, float t) const {
        constexpr float kS = 0.091888149f;  // 1 / (2 pi sqrt 3)
        float v = c[FPT_POLY_TERMS - 1], dv = dc[FPT_POLY_TERMS - 1];
#pragma unroll
        for (int k = FPT_POLY_TERMS - 2; k >= 0; --k) {
            v = __fmaf_rn(v, phi, c[k]);
            dv = __fmaf_rn(dv, phi, dc[k]);
        }
        const float S = __fmul_rn(kS, sqrt_approx(v));
        const float D = -__fmul_rn(dv, rcp_approx(v));
        return __fadd_rn(phi, __fmaf_rn(S, t, __fmul_rn(D, dN)));
    }
};

// Quadratic potential with B = A_p phi^p, binary32.  With u = phi^(p-1):
// dphi = phi t - 2 dN / phi, t = A_p dN u + c m sqrt(dN) xi, and the step's
// log-weight -beta sqrt(dN) xi - beta^2 dN / 2 with beta = B/S = (A_p / c m) u,
// i.e. u (a1 g + a2 u) with g = c m sqrt(dN) xi, a1 = -A_p/(c m)^2 and
// a2 = -A_p^2 dN / (2 (c m)^2).  g is formed from a Box–Muller pair as
// (kq rho) trig, like the constant-bias step.
template <int MODEL>
struct ModelStep<float, MODEL> {
    static_assert(is_pow_model(MODEL), "binary32 model tag");
    float tc, kq, m2dN, a1, a2, pm1;
    __device__ __forceinline__ void load(const SetConst& s) {
        tc = s.f_c1;
        kq = s.f_c2;
        m2dN = s.f_c3;
        a1 = s.f_pw1;
        a2 = s.f_pw2;
        pm1 = s.f_pm1;
    }
    __device__ __forceinline__ float u_of(float phi, float inv) const {
        constexpr int p = MODEL - kModelPow;
        if constexpr (p == 0) return inv;
        else if constexpr (p == 1) return 1.0f;
        else if constexpr (p == 2) return phi;
        else if constexpr (p == 3) return __fmul_rn(phi, phi);
        else if constexpr (p == 4) return __fmul_rn(__fmul_rn(phi, phi), phi);
        else return ex2_approx(__fmul_rn(pm1, lg2_approx(phi)));
    }
    // one step from phi with noise factor q trig; adds the step's log-weight to acc
    __device__ __forceinline__ float advance(float phi, float q, float trig, float& acc) const {
        const float inv = rcp_approx(phi);
        const float u = u_of(phi, inv);
        const float g = __fmul_rn(q, trig);
        const float t = __fmaf_rn(tc, u, g);
        acc = __fmaf_rn(u, __fmaf_rn(a2, u, __fmul_rn(a1, g)), acc);
        return __fadd_rn(phi, __fmaf_rn(phi, t, __fmul_rn(m2dN, inv)));
    }
};

// The step a stepper kernel runs: the scaled quadratic step for the binary32
// constant-bias quadratic model, the model's own step otherwise.
template <typename Real, int MODEL>
struct StepOf { using type = ModelStep<Real, MODEL>; };
template <>
struct StepOf<float, FPT_MODEL_QUADRATIC> { using type = QuadPsiStep; };

// Sixteen binary32 EM steps of a power model from one Philox group: as
// Block j (four steps, two Box–Muller pairs) of a 16-step group for the
// power-law models: as quad_block_f32, with the log-weight summed step by step
// into acc.
template <int MODEL, bool WALL>
__device__ __forceinline__ void pow_block_f32(const ModelStep<float, MODEL>& model, const uint32_t V[12], int j,
                                              float twouv, float& phi, float& mn, float& acc) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const NormalPair np = group_pair_f32(V, j, p);
        const float q = __fmul_rn(model.kq, np.rho);
        phi = model.advance(phi, q, np.c, acc);
        if constexpr (WALL) phi = fminf(phi, twouv - phi);
        const float first = phi;
        phi = model.advance(phi, q, np.s, acc);
        if constexpr (WALL) phi = fminf(phi, twouv - phi);
        mn = min3f(mn, first, phi);
    }
}

// One binary32 EM step and the wall.
template <bool WALL, typename Step>
__device__ __forceinline__ float step1_f32(const Step& model, float phi, float t, float twouv) {
    phi = model.step(phi, t);
    if constexpr (WALL) phi = fminf(phi, twouv - phi);
    return phi;
}

// Block j (four steps, two Box–Muller pairs) of a 16-step group's words V:
// the state update, the wall, the block minimum (one three-way minimum per
// pair) and the running sum of rho (c + s) = -(xi0 + xi1) / sqrt(2 ln 2).
template <bool WALL, typename Step>
__device__ __forceinline__ void quad_block_f32(const Step& model, const uint32_t V[12], int j, float twouv,
                                               float& phi, float& mn, float& srho) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const NormalPair np = group_pair_f32(V, j, p);
        const float q = __fmul_rn(model.kq, np.rho);
        phi = step1_f32<WALL>(model, phi, __fmaf_rn(q, np.c, model.tc), twouv);
        const float first = phi;
        phi = step1_f32<WALL>(model, phi, __fmaf_rn(q, np.s, model.tc), twouv);
        mn = min3f(mn, first, phi);
        srho = __fmaf_rn(np.rho, np.c + np.s, srho);
    }
}

// KS binary32 steps: Philox groups G0 .. G0 + KS/16 - 1, each three Philox
// blocks and four Box–Muller blocks block(V, j), j = 0..3.  Software-pipelined:
// the Philox blocks of group g + 1 are computed between the Box–Muller blocks
// of group g, so that a warp's instruction stream interleaves the integer
// multiplies with the XU work instead of alternating between the two phases.
// The words, and so the results, are those of computing each group in turn.
template <int KS, typename Block>
__device__ __forceinline__ void pipelined_groups(const PhiloxLane& pl, uint32_t G0, const PhiloxKeys& keys,
                                                 Block&& block) {
    static_assert(KS % 16 == 0, "whole 16-step groups");
    uint32_t V[12];
    philox_group(pl, G0, keys, V);
#pragma unroll
    for (int g = 0; g < KS / 16; ++g) {
        uint32_t Vn[12];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (g + 1 < KS / 16 && j < 3)
                philox_block(pl, 3u * (G0 + (uint32_t)g + 1u) + (uint32_t)j, keys, Vn + 4 * j);
            block(V, j);
        }
        if (g + 1 < KS / 16) {
#pragma unroll
            for (int i = 0; i < 12; ++i) V[i] = Vn[i];
        }
    }
}

// The binary32 sums are kept in units of -1/sqrt(2 ln 2) of the sum of the normals.
constexpr double kXiPerRho = -1.1774100225154747;  // -sqrt(2 ln 2)

// Binary64 (reference) steps: the update exactly as written in Eq. (11).  This
// translation unit is compiled without FMA contraction, so each operation is
// rounded as written.
template <>
struct ModelStep<double, FPT_MODEL_QUADRATIC> {
    double cm, b, dN, sq;
    __device__ __forceinline__ void load(const SetConst& s) {
        cm = s.cm;
        b = s.b;
        dN = s.dN;
        sq = s.sq;
    }
    __device__ __forceinline__ double step(double phi, double xi) const {
        const double D = -2.0 / phi;
        const double S = cm * phi;
        const double B = b * S;
        return phi + (D + B) * dN + S * xi * sq;
    }
};

template <>
struct ModelStep<double, FPT_MODEL_CONSTANT> {
    double a0, s0, b, dN, sq;
    __device__ __forceinline__ void load(const SetConst& s) {
        a0 = s.a0;
        s0 = s.cm;
        b = s.b;
        dN = s.dN;
        sq = s.sq;
    }
    __device__ __forceinline__ double step(double phi, double xi) const {
        return phi + (a0 + b * s0) * dN + s0 * xi * sq;
    }
};

// Polynomial potential, binary64: V and V' by Horner's rule from the top term,
// D = -V'/(3 H^2) with H^2 = V/3 and S = sqrt(V/3) / (2 pi), as written in §2.3
// Eq. (17); the update of Eq. (11) with B = b S.
template <>
struct ModelStep<double, FPT_MODEL_POLYNOMIAL> {
    double b, dN, sq;
    const double* c;
    __device__ __forceinline__ void load(const SetConst& s) {
        b = s.b;
        dN = s.dN;
        sq = s.sq;
        c = s.poly;
    }
    __device__ __forceinline__ double step(double phi, double xi) const {
        double V = 0.0, dV = 0.0;
        for (int k = FPT_POLY_TERMS - 1; k >= 0; --k) V = V * phi + c[k];
        for (int k = FPT_POLY_TERMS - 1; k >= 1; --k) dV = dV * phi + (double)k * c[k];
        const double H2 = V / 3.0;
        const double D = -dV / (3.0 * H2);
        const double S = sqrt(V / 3.0) / (2.0 * 3.14159265358979323846);
        const double B = b * S;
        return phi + (D + B) * dN + S * xi * sq;
    }
};

// Quadratic potential with B = A_p phi^p (§3.4 Eq. (26)), binary64: the update
// of Eq. (11) and the step's log-weight -(B/S^2)(B dN/2 + S xi sqrt(dN)) of
// Eqs. (12)-(14), as written.
template <int MODEL>
struct ModelStep<double, MODEL> {
    static_assert(MODEL == kModelPowReal, "binary64 model tag");
    double cm, A, p, dN, sq;
    __device__ __forceinline__ void load(const SetConst& s) {
        cm = s.cm;
        A = s.b;
        p = s.pw;
        dN = s.dN;
        sq = s.sq;
    }
    __device__ __forceinline__ double advance(double phi, double xi, double& acc) const {
        const double D = -2.0 / phi;
        const double S = cm * phi;
        const double B = A * pow(phi, p);
        acc -= (B / (S * S)) * (0.5 * B * dN + S * xi * sq);
        return phi + (D + B) * dN + S * xi * sq;
    }
};

// ---------------------------------------------------------------------------
// Running sum of the normals (W)
// ---------------------------------------------------------------------------
template <int PREC>
struct WSum;

template <>
struct WSum<FPT_PREC_F32_KAHAN> {
    float s, c;  // Kahan sum and compensation
    __device__ __forceinline__ void reset() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double total(float tail) const {
        return ((double)s - (double)c) + (double)tail;
    }
};

template <>
struct WSum<FPT_PREC_F32_F64ACC> {
    double s;
    __device__ __forceinline__ void reset() { s = 0.0; }
    __device__ __forceinline__ void add(float x) { s += (double)x; }
    __device__ __forceinline__ double total(float tail) const { return s + (double)tail; }
};

template <>
struct WSum<FPT_PREC_F64> {
    double s;
    __device__ __forceinline__ void reset() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double total(double tail) const { return s + tail; }
};

template <typename Real>
__device__ __forceinline__ void normals4(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K, Real xi[4]);
template <>
__device__ __forceinline__ void normals4<double>(const PhiloxLane& l, uint32_t k, const PhiloxKeys& K,
                                                 double xi[4]) {
    normals4_f64(l, k, K, xi);
}

template <typename Real>
__device__ __forceinline__ Real real_min(Real a, Real b);
template <>
__device__ __forceinline__ float real_min<float>(float a, float b) { return fminf(a, b); }
template <>
__device__ __forceinline__ double real_min<double>(double a, double b) { return fmin(a, b); }

// phi_in, phi_end and 2 phi_uv in the stepper's state variable: binary64 phi,
// binary32 phi, or binary32 psi = phi / sqrt(2 dN) for the quadratic constant-bias step
template <typename Real, int MODEL>
__device__ __forceinline__ Real set_phi_in(const SetConst& S) {
    if constexpr (sizeof(Real) == 8) return (Real)S.phi_in;
    else if constexpr (MODEL == FPT_MODEL_QUADRATIC) return S.f_psi_in;
    else return S.f_phi_in;
}
template <typename Real, int MODEL>
__device__ __forceinline__ Real set_phi_end(const SetConst& S) {
    if constexpr (sizeof(Real) == 8) return (Real)S.phi_end;
    else if constexpr (MODEL == FPT_MODEL_QUADRATIC) return S.f_psi_end;
    else return S.f_phi_end;
}
template <typename Real, int MODEL>
__device__ __forceinline__ Real set_twouv(const SetConst& S) {
    if constexpr (sizeof(Real) == 8) return (Real)S.twouv;
    else if constexpr (MODEL == FPT_MODEL_QUADRATIC) return S.f_psi_twouv;
    else return S.f_twouv;
}

// A run that finished inside its last block, waiting for the replay.
template <typename Real, int PREC>
struct Pending {
    unsigned long long rec;  // record index
    int m0;                  // step count at the block start
    int set;                 // parameter set
    Real phi0;               // phi at the block start
    WSum<PREC> W;            // running sum of the normals before the block
};

constexpr int kQueueCap = 64;  // per warp: up to 31 waiting + 32 new
constexpr int kParkWords = 12;  // per thread: a run's live state during a batch replay

// Park / unpark 32-bit words through volatile shared memory, so the values are
// really dead in registers while the replay runs (no store-to-load forwarding).
// The slots are interleaved by thread: word j of a thread is at v[j * stride]
// (stride = threads per block), so a 64-bit value takes words i and i + stride.
__device__ __forceinline__ void park(volatile unsigned* v, int i, unsigned x) { v[i] = x; }
__device__ __forceinline__ unsigned unpark(volatile unsigned* v, int i) { return v[i]; }
__device__ __forceinline__ void park_f(volatile unsigned* v, int i, float x) { v[i] = __float_as_uint(x); }
__device__ __forceinline__ float unpark_f(volatile unsigned* v, int i) { return __uint_as_float(v[i]); }
__device__ __forceinline__ void park_d(volatile unsigned* v, int i, int stride, double x) {
    v[i] = (unsigned)__double2loint(x);
    v[i + stride] = (unsigned)__double2hiint(x);
}
__device__ __forceinline__ double unpark_d(volatile unsigned* v, int i, int stride) {
    return __hiloint2double((int)v[i + stride], (int)v[i]);
}
template <typename Real>
__device__ __forceinline__ void park_r(volatile unsigned* v, int i, int stride, Real x) {
    if constexpr (sizeof(Real) == 4) park_f(v, i, (float)x); else park_d(v, i, stride, (double)x);
}
template <typename Real>
__device__ __forceinline__ Real unpark_r(volatile unsigned* v, int i, int stride) {
    if constexpr (sizeof(Real) == 4) return (Real)unpark_f(v, i); else return (Real)unpark_d(v, i, stride);
}
template <int PREC>
__device__ __forceinline__ void park_w(volatile unsigned* v, int i, int stride, const WSum<PREC>& W) {
    if constexpr (PREC == FPT_PREC_F32_KAHAN) { park_f(v, i, W.s); park_f(v, i + stride, W.c); }
    else park_d(v, i, stride, W.s);
}
template <int PREC>
__device__ __forceinline__ void unpark_w(volatile unsigned* v, int i, int stride, WSum<PREC>& W) {
    if constexpr (PREC == FPT_PREC_F32_KAHAN) { W.s = unpark_f(v, i); W.c = unpark_f(v, i + stride); }
    else W.s = unpark_d(v, i, stride);
}
// dynamic shared memory per warp: the replay queue plus the parking slots
template <typename Real, int PREC>
constexpr int warp_smem_bytes() { return kQueueCap * (int)sizeof(Pending<Real, PREC>) + 32 * kParkWords * 4; }

// Replay the blocks of cnt queued runs (lane j takes entry j), find each run's
// first passage or cap step and write its record.  Called by a whole warp, once
// per 32 finished runs, while the lanes' own runs are parked in shared memory.
template <typename Real, int PREC, int MODEL, bool WALL, int KS>
__device__ __forceinline__ void replay_batch(const Pending<Real, PREC>* q, int cnt, const StepperParams& P,
                                             const SetConst* s_sets, unsigned lane,
                                             unsigned long long& my_steps) {
    const unsigned mask = cnt >= 32 ? 0xffffffffu : ((1u << cnt) - 1u);
    if ((int)lane >= cnt) return;
    const Pending<Real, PREC> e = q[lane];
    const SetConst& S = s_sets[e.set];
    typename StepOf<Real, MODEL>::type model;
    model.load(S);
    const Real phi_end = set_phi_end<Real, MODEL>(S);
    const Real twouv = set_twouv<Real, MODEL>(S);
    const PhiloxLane pl = philox_lane(S.traj_offset + (e.rec - (unsigned long long)S.first), S.set_id, P.keys);
    Real ph = e.phi0, prev = e.phi0, s2 = (Real)0;
    int M = 0;
    bool crossed = false;
    if constexpr (sizeof(Real) == 4) {
        // binary32: whole 16-step groups, as the stepping loop draws them
        for (int gg = 0; gg < KS / 16; ++gg) {
            uint32_t V[12];
            philox_group(pl, ((uint32_t)e.m0 >> 4) + (uint32_t)gg, P.keys, V);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const NormalPair np = group_pair_f32(V, j, p);
                    const float q = __fmul_rn(model.kq, np.rho);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (M == 0) {
                            const float trig = h == 0 ? np.c : np.s;
                            prev = ph;
                            if constexpr (is_pow_model(MODEL)) {
                                ph = model.advance(ph, q, trig, s2);
                                if constexpr (WALL) ph = fminf(ph, twouv - ph);
                            } else {
                                ph = step1_f32<WALL>(model, ph, __fmaf_rn(q, trig, model.tc), twouv);
                                s2 = __fmaf_rn(np.rho, trig, s2);
                            }
                            const int step_index = e.m0 + 16 * gg + 4 * j + 2 * p + h;
                            if (ph <= phi_end) {
                                crossed = true;
                                M = step_index + 1;
                            } else if (step_index + 1 >= S.m_max) {
                                M = step_index + 1;
                            }
                        }
                    }
                }
            }
            if (__all_sync(mask, M != 0)) break;
        }
    } else {
        const uint32_t k0 = (uint32_t)e.m0 >> 2;
        for (int g = 0; g < KS / 4; ++g) {
            Real xi[4];
            normals4<Real>(pl, k0 + (uint32_t)g, P.keys, xi);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                if (M == 0) {
                    prev = ph;
                    if constexpr (is_pow_model(MODEL)) {
                        ph = model.advance(ph, xi[q4], s2);
                    } else {
                        ph = model.step(ph, xi[q4]);
                        s2 += xi[q4];
                    }
                    if constexpr (WALL) ph = real_min<Real>(ph, twouv - ph);
                    const int step_index = e.m0 + 4 * g + q4;
                    if (ph <= phi_end) {
                        crossed = true;
                        M = step_index + 1;
                    } else if (step_index + 1 >= S.m_max) {
                        M = step_index + 1;
                    }
                }
            }
            if (__all_sync(mask, M != 0)) break;
        }
    }
    // constant bias: W is the sum of the normals (binary32 sums in rho units);
    // power models: W is ln w itself
    const double Wtot = (sizeof(Real) == 4 && !is_pow_model(MODEL)) ? kXiPerRho * e.W.total(s2)
                                                                     : (double)e.W.total(s2);
    double N;
    if (crossed) {
        // linear interpolation of the crossing inside step M-1, in binary64
        const double a = (double)prev, c = (double)ph, pe = (double)phi_end;
        const double theta = (a - pe) / (a - c);
        N = ((double)(M - 1) + theta) * S.dN;
    } else {
        N = __longlong_as_double(0x7ff0000000000000ll);  // +inf: censored
    }
#if FPT_DEBUG
    if (e.rec >= P.n_total) {
        atomicOr(&P.scratch->status, kStatusRecord);
        return;
    }
#endif
    P.out_N[e.rec] = N;
    P.out_logw[e.rec] = is_pow_model(MODEL) ? Wtot : -S.lw_bsq * Wtot - S.lw_half_b2dN * (double)M;
    my_steps += (unsigned long long)M;
}

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------
// Register cap per thread.  64 is the largest that keeps 32 warps resident per
// SM (4 blocks of 256 or 2 of 512 threads: 65,536 registers), and its spare
// registers hold the next group's Philox words while the current group's
// Box-Muller blocks run.  Measured on the drift-dominated ladder (steps/s of
// the kernel, 64-step blocks): 64 registers, 512 threads (32 warps per SM):
// 1.335e12; 56 registers, 384 threads (36 warps): 1.325e12; 48 registers,
// 256 threads (40 warps): 1.313e12 -- more resident warps do not pay for the
// spills they need.  At 64 the quadratic, constant and
// power-law kernels are spill-free; the polynomial-potential ones (eight
// coefficients per set) spill 12-48 bytes (56-84 at a cap of 56).  The binary64
// reference kernels are built with a larger cap.
#ifndef FPT_STEPPER_MAXNREG
#define FPT_STEPPER_MAXNREG 64
#endif
template <typename Real, int PREC, int MODEL, bool WALL, int KS>
__global__ void __maxnreg__(FPT_STEPPER_MAXNREG)
stepper_kernel(const StepperParams P) {
    static_assert(KS % (sizeof(Real) == 4 ? 16 : 4) == 0,
                  "a scheduling block is a whole number of 16-step groups (binary32) or 4-step blocks (binary64)");
    using Entry = Pending<Real, PREC>;
    // dynamic shared memory: [set table][set starts][per-warp replay queues][parking slots]
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const int n_sets = P.n_sets;
    SetConst* s_sets = reinterpret_cast<SetConst*>(s_dyn);
    long long* s_first = reinterpret_cast<long long*>(s_dyn + (size_t)n_sets * sizeof(SetConst));
    unsigned char* s_queue = s_dyn + stepper_table_bytes(n_sets);
    Entry* q = reinterpret_cast<Entry*>(s_queue) + (threadIdx.x >> 5) * kQueueCap;
    // parking slots follow the queues: kParkWords words per thread, interleaved by thread
    volatile unsigned* park_slot = reinterpret_cast<volatile unsigned*>(
        s_queue + (size_t)(blockDim.x >> 5) * kQueueCap * sizeof(Entry)) + threadIdx.x;
    for (int i = threadIdx.x; i < n_sets; i += blockDim.x) {
        s_sets[i] = P.sets[i];
        s_first[i] = P.sets[i].first;
    }
    if (threadIdx.x == 0) s_first[n_sets] = (long long)P.n_total;
    __syncthreads();

    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;

    // lane state
    bool live = false, exhausted = false;
    int set = 0;
    unsigned long long rec = 0;  // record index (= ticket)
    Real phi = (Real)0, phi_end = (Real)0, twouv = (Real)0;
    int m = 0, m_max = 0;
    PhiloxLane pl{0u, 0u, 0u};
    typename StepOf<Real, MODEL>::type model;
    model.load(s_sets[0]);
    WSum<PREC> W;
    W.reset();
    unsigned long long my_steps = 0;
    int q_count = 0;  // warp-uniform

    for (;;) {
        // ---- refill: lanes without a run take tickets (one atomic per warp) ----
        for (;;) {
            const bool want = !live && !exhausted;
            const unsigned need = __ballot_sync(FULL, want);
            if (need == 0u) break;
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(&P.scratch->ticket, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (want) {
                const unsigned long long t = base + (unsigned long long)__popc(need & lt_mask);
                if (t >= P.n_total) {
                    exhausted = true;
                } else {
                    // set of record t: the last s with first[s] <= t
                    int lo = 0, hi = n_sets - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((long long)t >= s_first[mid]) lo = mid; else hi = mid - 1;
                    }
                    set = lo;
                    bool bad_set = false;
#if FPT_DEBUG
                    bad_set = lo < 0 || lo >= n_sets || (long long)t < s_first[lo] || (long long)t >= s_first[lo + 1];
                    if (bad_set) {
                        atomicOr(&P.scratch->status, kStatusSetIndex);
                        exhausted = true;  // stop this lane rather than write a record of the wrong set
                    }
#endif
                    if (!bad_set) {
                    const SetConst& S = s_sets[set];
                    rec = t;
                    pl = philox_lane(S.traj_offset + (t - (unsigned long long)S.first), S.set_id, P.keys);
                    model.load(S);
                    phi = set_phi_in<Real, MODEL>(S);
                    phi_end = set_phi_end<Real, MODEL>(S);
                    twouv = set_twouv<Real, MODEL>(S);
                    m = 0;
                    m_max = S.m_max;
                    W.reset();
                    if (S.phi_in <= S.phi_end) {
                        // starts at or below the end of inflation: N = 0, w = 1
                        P.out_N[t] = 0.0;
                        P.out_logw[t] = 0.0;
                    } else {
                        live = true;
                    }
                    }  // !bad_set
                }
            }
        }
        if (!__any_sync(FULL, live)) break;

        // ---- one scheduling block of KS steps, no per-step branches ----
        const Real phi0 = phi;
        const int m0 = m;
        Real mn = phi;
        Real sblk = (Real)0;
        if constexpr (sizeof(Real) == 4) {
            const uint32_t G0 = (uint32_t)m0 >> 4;
            if constexpr (is_pow_model(MODEL))
                pipelined_groups<KS>(pl, G0, P.keys, [&](const uint32_t* V, int j) {
                    pow_block_f32<MODEL, WALL>(model, V, j, twouv, phi, mn, sblk);
                });
            else
                pipelined_groups<KS>(pl, G0, P.keys, [&](const uint32_t* V, int j) {
                    quad_block_f32<WALL>(model, V, j, twouv, phi, mn, sblk);
                });
        } else {
            const uint32_t k0 = (uint32_t)m0 >> 2;
#pragma unroll
            for (int g = 0; g < KS / 4; ++g) {
                Real xi[4];
                normals4<Real>(pl, k0 + (uint32_t)g, P.keys, xi);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    if constexpr (is_pow_model(MODEL)) {
                        phi = model.advance(phi, xi[q4], sblk);
                    } else {
                        phi = model.step(phi, xi[q4]);
                        sblk += xi[q4];
                    }
                    if constexpr (WALL) phi = real_min<Real>(phi, twouv - phi);  // mirror at phi_uv
                    mn = real_min<Real>(mn, phi);
                }
            }
        }
        m = m0 + KS;
        const bool event = live && (mn <= phi_end || m >= m_max);
        const unsigned ev = __ballot_sync(FULL, event);
        if (ev) {
            // finished inside this block: queue the block-start state, free the lane
            if (event) {
                const int at = q_count + __popc(ev & lt_mask);
#if FPT_DEBUG
                if (at >= kQueueCap) {
                    atomicOr(&P.scratch->status, kStatusQueueFull);  // the run is dropped, not written
                } else
#endif
                {
                    Entry& slot = q[at];
                    slot.rec = rec;
                    slot.m0 = m0;
                    slot.set = set;
                    slot.phi0 = phi0;
                    slot.W = W;
                }
                live = false;
            }
            q_count += __popc(ev);
#if FPT_DEBUG
            if (q_count > kQueueCap) q_count = kQueueCap;
#endif
            if (q_count >= 32) {
                // park this lane's run (the stride keeps one thread's words in one bank)
                const int stride = (int)blockDim.x;
                volatile unsigned* v = park_slot;
                park_r<Real>(v, 0 * stride, stride, phi);  // words 0, 1
                park_w<PREC>(v, 2 * stride, stride, W);    // words 2, 3
                park(v, 4 * stride, (unsigned)m);
                park(v, 5 * stride, (unsigned)rec);
                park(v, 6 * stride, (unsigned)(rec >> 32));
                park(v, 7 * stride, (unsigned)set | (live ? 0x40000000u : 0u) | (exhausted ? 0x80000000u : 0u));
                park(v, 8 * stride, pl.r1_x0);
                park(v, 9 * stride, pl.r1_x1);
                park(v, 10 * stride, pl.r1_set);
                __syncwarp();
                replay_batch<Real, PREC, MODEL, WALL, KS>(q, 32, P, s_sets, lane, my_steps);
                __syncwarp();
                const int rest = q_count - 32;
                Entry tmp;
                if ((int)lane < rest) tmp = q[32 + lane];
                __syncwarp();
                if ((int)lane < rest) q[lane] = tmp;
                __syncwarp();
                q_count = rest;
                // unpark
                phi = unpark_r<Real>(v, 0 * stride, stride);
                unpark_w<PREC>(v, 2 * stride, stride, W);
                m = (int)unpark(v, 4 * stride);
                rec = (unsigned long long)unpark(v, 5 * stride) |
                      ((unsigned long long)unpark(v, 6 * stride) << 32);
                const unsigned sf = unpark(v, 7 * stride);
                set = (int)(sf & 0x3fffffffu);
                live = (sf & 0x40000000u) != 0u;
                exhausted = (sf & 0x80000000u) != 0u;
                pl.r1_x0 = unpark(v, 8 * stride);
                pl.r1_x1 = unpark(v, 9 * stride);
                pl.r1_set = unpark(v, 10 * stride);
                const SetConst& S = s_sets[set];
                model.load(S);
                phi_end = set_phi_end<Real, MODEL>(S);
                twouv = set_twouv<Real, MODEL>(S);
                m_max = S.m_max;
            }
        }
        if (live) W.add(sblk);
    }
    if (q_count > 0) {
        __syncwarp();
        replay_batch<Real, PREC, MODEL, WALL, KS>(q, q_count, P, s_sets, lane, my_steps);
    }

    // ---- total steps: warp reduce, one atomic per warp ----
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_xor_sync(FULL, my_steps, o);
    if (lane == 0) {
        atomicAdd(&P.scratch->steps, my_steps);
        if (P.steps_out) atomicAdd(P.steps_out, my_steps);
    }
}

}  // namespace fpt
