// Host/device layout of the stepper's per-set constants and its scratch words.
#pragma once
#include <cstdint>

#include "fpt.h"
#include "rng.cuh"
#include "status.h"

namespace fpt {

constexpr int kStepperMaxThreads = 512;

// Model tags of the quadratic potential with the power-law bias B = A_p phi^p
// (§3.4 Eq. (26)): kModelPow + p for an integer p in 0..4 (phi^(p-1) by
// multiplies), kModelPowReal for any real p (phi^(p-1) = 2^((p-1) log2 phi)).
constexpr int kModelPow = 16;
constexpr int kModelPowReal = kModelPow + 15;
__host__ __device__ constexpr bool is_pow_model(int model) { return model >= kModelPow; }

// Per parameter set, prepared on the host (binary64 originals and the
// binary32 step constants), copied to shared memory by every block.
struct SetConst {
    double phi_in, phi_end, phi_uv, twouv;  // twouv = 2 phi_uv (reflection phi -> 2 phi_uv - phi)
    double dN, sq, b;                       // sq = sqrt(dN)
    double cm;                              // quadratic: c0 m, c0 = 1/(2 pi sqrt 6); constant model: s0
    double a0;                              // constant model drift
    double lw_bsq, lw_half_b2dN;            // ln w = -lw_bsq * W - lw_half_b2dN * M
    long long first;                        // index of this set's first record
    unsigned long long traj_offset;         // Philox id of this set's first run
    int m_max;                              // censoring cap in steps
    uint32_t set_id;                        // Philox counter word 3
    float f_phi_in, f_phi_end, f_twouv;
    // the same three in the binary32 state variable of the quadratic constant-bias
    // stepper, psi = phi / sqrt(2 dN) (stepper.cuh, QuadPsiStep)
    float f_psi_in, f_psi_end, f_psi_twouv;
    float f_c1, f_c2, f_c3;                 // binary32 step constants (see ModelStep)
    float f_cmdN;                           // c0 m dN: the bias part of dphi/phi is b * f_cmdN
    float f_dN, f_sq;                       // dN and sqrt(dN) in binary32 (learned-bias stepper)
    // power-law bias B = A_p phi^p (A_p in b): the exponent, and the binary32
    // weight constants of ModelStep for the power models (stepper.cuh)
    double pw;
    float f_pm1, f_pw1, f_pw2;              // p - 1, -A_p/(c m)^2, -A_p^2 dN/(2 (c m)^2)
    // polynomial potential V = sum_k poly[k] phi^k: binary64 coefficients, and
    // binary32 coefficients of V and V' (f_dpoly[k] = (k + 1) poly[k + 1])
    double poly[FPT_POLY_TERMS];
    float f_poly[FPT_POLY_TERMS], f_dpoly[FPT_POLY_TERMS];
};

// Bytes of the per-set table at the start of the stepper's dynamic shared
// memory: n_sets SetConst plus n_sets + 1 set starts, rounded to 16.
inline __host__ __device__ size_t stepper_table_bytes(int n_sets) {
    const size_t b = (size_t)n_sets * sizeof(SetConst) + (size_t)(n_sets + 1) * sizeof(long long);
    return (b + 15) / 16 * 16;
}

// Device scratch of one stepper launch (zeroed before the launch).
struct StepperScratch {
    unsigned long long ticket;  // next record index to hand out
    unsigned long long steps;   // total Euler–Maruyama steps taken
    unsigned int status;        // error flags (0 = ok)
    unsigned int pad_;
};

// Kernel parameters of one stepper launch (passed by value: constant bank).
struct StepperParams {
    PhiloxKeys keys;                 // round keys of the seed
    const SetConst* sets;            // n_sets entries (device)
    int n_sets;
    unsigned long long n_total;      // records over all sets
    double* out_N;
    double* out_logw;
    StepperScratch* scratch;         // zeroed before the launch
    unsigned long long* steps_out;   // optional
};

}  // namespace fpt
