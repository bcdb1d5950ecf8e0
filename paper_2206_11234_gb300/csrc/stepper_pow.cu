// Binary32-state instantiations of the persistent stepper with the power-law
// bias B = A_p phi^p (§3.4 Eq. (26)): p in 0..4 specialised, any other real p
// through exp2/log2; one scheduling block length (32 steps).
#include "stepper.cuh"
#include "stepper_launch.h"

namespace fpt {
namespace {

constexpr int kPowKS = 32;

template <int PREC, int MODEL, bool WALL>
cudaError_t launch(const StepperParams& a, int grid, int block, cudaStream_t stream) {
    const size_t smem = stepper_table_bytes(a.n_sets) + (size_t)(block / 32) * warp_smem_bytes<float, PREC>();
    stepper_kernel<float, PREC, MODEL, WALL, kPowKS><<<grid, block, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int PREC, int MODEL, bool WALL>
StepperKernel make() {
    return StepperKernel{(const void*)stepper_kernel<float, PREC, MODEL, WALL, kPowKS>,
                         warp_smem_bytes<float, PREC>(), &launch<PREC, MODEL, WALL>};
}

template <int PREC, bool WALL>
StepperKernel by_power(int p_code) {
    switch (p_code) {
        case 0: return make<PREC, kModelPow + 0, WALL>();
        case 1: return make<PREC, kModelPow + 1, WALL>();
        case 2: return make<PREC, kModelPow + 2, WALL>();
        case 3: return make<PREC, kModelPow + 3, WALL>();
        case 4: return make<PREC, kModelPow + 4, WALL>();
        default: return make<PREC, kModelPowReal, WALL>();
    }
}

template <int PREC>
StepperKernel by_wall(bool wall, int p_code) {
    return wall ? by_power<PREC, true>(p_code) : by_power<PREC, false>(p_code);
}

}  // namespace

int pow_code(double p) {
    for (int k = 0; k <= 4; ++k)
        if (p == (double)k) return k;
    return kModelPowReal - kModelPow;
}

StepperKernel stepper_f32_pow(int precision, double p, bool wall, int k_steps) {
    if (k_steps != kPowKS) return StepperKernel{nullptr, 0, nullptr};
    if (precision == FPT_PREC_F32_KAHAN) return by_wall<FPT_PREC_F32_KAHAN>(wall, pow_code(p));
    if (precision == FPT_PREC_F32_F64ACC) return by_wall<FPT_PREC_F32_F64ACC>(wall, pow_code(p));
    return StepperKernel{nullptr, 0, nullptr};
}

}  // namespace fpt
