// Persistent Euler–Maruyama first-passage stepper (arXiv:2206.11234 §2.2).
//
// One lane = one run.  A run's state (phi, step count, the running sum of its
// normals) lives in registers.  Lanes advance in scheduling blocks of KS
// steps with no per-step control flow: each step is the biased EM update of
// §2.2 Eq. (11) followed by the reflecting wall, and the lane keeps the
// minimum phi of the block.  At the block end a lane whose minimum reached
// phi_end (first passage, §2.1 below Eq. (8)) or whose step count reached the
// censoring cap replays the block from its saved start state with a per-step
// test — bit-identical arithmetic, the same Philox counters — to find the
// exact step, interpolates the crossing time in binary64 and writes its
// record.  Finished lanes then refill from a global ticket counter (one
// atomicAdd per warp), so a warp keeps 32 live runs whatever their lengths
// (persistent scheduler).
//
// Log-weight (§2.2 Eqs. (12)-(14), sign as derived from Eqs. (13)-(14)):
// with B = b S the step term is -(b xi sqrt(dN) + b^2 dN / 2), so a run of M
// steps has ln w = -b sqrt(dN) W - b^2 M dN / 2 with W = sum xi.  W is summed
// per block in the state precision and folded into a running sum that is
// either compensated binary32 (Kahan) or binary64.
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

// ---------------------------------------------------------------------------
// Model steps.  phi' = phi + (D + b S) dN + S xi sqrt(dN)   (§2.2 Eq. (11))
// ---------------------------------------------------------------------------
template <typename Real, int MODEL>
struct ModelStep;

// Quadratic potential, binary32.  The increment is formed on its own and then
// added: dphi = phi (b c m dN + c m sqrt(dN) xi) - 2 dN / phi.  (Folding the
// bias into a factor 1 + b c m dN would round b c m dN ~ 1e-6 on the 2^-23
// grid of numbers near 1, i.e. change b by ~1%, which the weights would not
// know about.)  Explicit intrinsics fix the rounding so the replay of a block
// reproduces it bit for bit.
template <>
struct ModelStep<float, FPT_MODEL_QUADRATIC> {
    float bcmdN, cmsq, m2dN;
    __device__ __forceinline__ void load(const SetConst& s) {
        bcmdN = s.f_c1;
        cmsq = s.f_c2;
        m2dN = s.f_c3;
    }
    __device__ __forceinline__ float step(float phi, float xi) const {
        const float inv = rcp_approx(phi);
        const float t = __fmaf_rn(cmsq, xi, bcmdN);
        const float v = __fmul_rn(m2dN, inv);
        return __fadd_rn(phi, __fmaf_rn(phi, t, v));
    }
};

// Constant drift a0 and noise s0, binary32: dphi = (a0 + b s0) dN + s0 sqrt(dN) xi.
template <>
struct ModelStep<float, FPT_MODEL_CONSTANT> {
    float c, s0sq;
    __device__ __forceinline__ void load(const SetConst& s) {
        c = s.f_c1;
        s0sq = s.f_c2;
    }
    __device__ __forceinline__ float step(float phi, float xi) const {
        return __fadd_rn(phi, __fmaf_rn(s0sq, xi, c));
    }
};

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
__device__ __forceinline__ void normals4(const PhiloxLane& l, uint32_t k, uint32_t key0,
                                         uint32_t key1, Real xi[4]);
template <>
__device__ __forceinline__ void normals4<float>(const PhiloxLane& l, uint32_t k, uint32_t key0,
                                                uint32_t key1, float xi[4]) {
    normals4_f32(l, k, key0, key1, xi);
}
template <>
__device__ __forceinline__ void normals4<double>(const PhiloxLane& l, uint32_t k, uint32_t key0,
                                                 uint32_t key1, double xi[4]) {
    normals4_f64(l, k, key0, key1, xi);
}

template <typename Real>
__device__ __forceinline__ Real real_min(Real a, Real b);
template <>
__device__ __forceinline__ float real_min<float>(float a, float b) { return fminf(a, b); }
template <>
__device__ __forceinline__ double real_min<double>(double a, double b) { return fmin(a, b); }

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------
template <typename Real, int PREC, int MODEL, bool WALL, int KS>
__global__ void __launch_bounds__(kStepperMaxThreads)
stepper_kernel(const SetConst* __restrict__ sets, int n_sets, uint64_t n_total, uint32_t key0,
               uint32_t key1, double* __restrict__ out_N, double* __restrict__ out_logw,
               StepperScratch* __restrict__ scratch, unsigned long long* __restrict__ steps_out) {
    static_assert(KS % 4 == 0, "a scheduling block is a whole number of Philox blocks");
    __shared__ SetConst s_sets[FPT_MAX_SETS];
    __shared__ long long s_first[FPT_MAX_SETS + 1];
    for (int i = threadIdx.x; i < n_sets; i += blockDim.x) {
        s_sets[i] = sets[i];
        s_first[i] = sets[i].first;
    }
    if (threadIdx.x == 0) s_first[n_sets] = (long long)n_total;
    __syncthreads();

    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;

    // lane state
    bool live = false, exhausted = false;
    int set = 0;
    uint64_t rec = 0;  // record index (= ticket)
    Real phi = (Real)0, phi_end = (Real)0, twouv = (Real)0;
    int m = 0, m_max = 0;
    PhiloxLane pl{0u, 0u, 0u};
    ModelStep<Real, MODEL> model;
    model.load(s_sets[0]);
    WSum<PREC> W;
    W.reset();
    unsigned long long my_steps = 0;

    for (;;) {
        // ---- refill: lanes without a run take tickets (one atomic per warp) ----
        for (;;) {
            const bool want = !live && !exhausted;
            const unsigned need = __ballot_sync(FULL, want);
            if (need == 0u) break;
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(&scratch->ticket, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (want) {
                const uint64_t t = base + (uint64_t)__popc(need & ((1u << lane) - 1u));
                if (t >= n_total) {
                    exhausted = true;
                } else {
                    // set of record t: the last s with first[s] <= t
                    int lo = 0, hi = n_sets - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((long long)t >= s_first[mid]) lo = mid; else hi = mid - 1;
                    }
                    set = lo;
                    const SetConst& S = s_sets[set];
                    rec = t;
                    const uint64_t id = S.traj_offset + (t - (uint64_t)S.first);
                    pl = philox_lane(id, S.set_id, key0, key1);
                    model.load(S);
                    if constexpr (sizeof(Real) == 4) {
                        phi = S.f_phi_in;
                        phi_end = S.f_phi_end;
                        twouv = S.f_twouv;
                    } else {
                        phi = S.phi_in;
                        phi_end = S.phi_end;
                        twouv = S.twouv;
                    }
                    m = 0;
                    m_max = S.m_max;
                    W.reset();
                    if (S.phi_in <= S.phi_end) {
                        // starts at or below the end of inflation: N = 0, w = 1
                        out_N[t] = 0.0;
                        out_logw[t] = 0.0;
                    } else {
                        live = true;
                    }
                }
            }
        }
        if (!__any_sync(FULL, live)) break;

        // ---- one scheduling block of KS steps, no per-step branches ----
        const Real phi0 = phi;
        const int m0 = m;
        Real mn = phi;
        Real sblk = (Real)0;
        const uint32_t k0 = (uint32_t)m0 >> 2;
#pragma unroll
        for (int g = 0; g < KS / 4; ++g) {
            Real xi[4];
            normals4<Real>(pl, k0 + (uint32_t)g, key0, key1, xi);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                phi = model.step(phi, xi[q]);
                if constexpr (WALL) phi = real_min<Real>(phi, twouv - phi);  // mirror at phi_uv
                mn = real_min<Real>(mn, phi);
                sblk += xi[q];
            }
        }
        m = m0 + KS;
        const bool event = live && (mn <= phi_end || m >= m_max);

        if (__any_sync(FULL, event)) {
            if (event) {
                // replay the block step by step to find the first passage or the cap
                Real ph = phi0, prev = phi0, s2 = (Real)0;
                int M = 0;
                bool crossed = false;
                for (int g = 0; g < KS / 4 && M == 0; ++g) {
                    Real xi[4];
                    normals4<Real>(pl, k0 + (uint32_t)g, key0, key1, xi);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (M == 0) {
                            prev = ph;
                            ph = model.step(ph, xi[q]);
                            if constexpr (WALL) ph = real_min<Real>(ph, twouv - ph);
                            s2 += xi[q];
                            const int step_index = m0 + 4 * g + q;
                            if (ph <= phi_end) {
                                crossed = true;
                                M = step_index + 1;
                            } else if (step_index + 1 >= m_max) {
                                M = step_index + 1;
                            }
                        }
                    }
                }
                const SetConst& S = s_sets[set];
                const double Wtot = W.total(s2);
                double N;
                if (crossed) {
                    // linear interpolation of the crossing inside step M-1, in binary64
                    const double a = (double)prev, c = (double)ph, e = (double)phi_end;
                    const double theta = (a - e) / (a - c);
                    N = ((double)(M - 1) + theta) * S.dN;
                } else {
                    N = __longlong_as_double(0x7ff0000000000000ll);  // +inf: censored
                }
                out_N[rec] = N;
                out_logw[rec] = -S.lw_bsq * Wtot - S.lw_half_b2dN * (double)M;
                my_steps += (unsigned long long)M;
                live = false;
            }
        }
        if (live) W.add(sblk);
    }

    // ---- total steps: warp reduce, one atomic per warp ----
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_xor_sync(FULL, my_steps, o);
    if (lane == 0) {
        atomicAdd(&scratch->steps, my_steps);
        if (steps_out) atomicAdd(steps_out, my_steps);
    }
}

}  // namespace fpt
