// Binary32-state instantiations of the persistent stepper.
#include "stepper.cuh"
#include "stepper_launch.h"

namespace fpt {
namespace {

template <int PREC, int MODEL, bool WALL, int KS>
cudaError_t launch(const StepperParams& a, int grid, int block, cudaStream_t stream) {
    const size_t smem = stepper_table_bytes(a.n_sets) + (size_t)(block / 32) * warp_smem_bytes<float, PREC>();
    stepper_kernel<float, PREC, MODEL, WALL, KS><<<grid, block, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int PREC, int MODEL, bool WALL, int KS>
StepperKernel make() {
    return StepperKernel{(const void*)stepper_kernel<float, PREC, MODEL, WALL, KS>,
                         warp_smem_bytes<float, PREC>(), &launch<PREC, MODEL, WALL, KS>};
}

template <int PREC, int MODEL, bool WALL>
StepperKernel by_ks(int ks) {
    switch (ks) {
        case 16: return make<PREC, MODEL, WALL, 16>();
        case 32: return make<PREC, MODEL, WALL, 32>();
        case 64: return make<PREC, MODEL, WALL, 64>();
        default: return StepperKernel{nullptr, 0, nullptr};
    }
}

template <int PREC, int MODEL>
StepperKernel by_wall(bool wall, int ks) {
    return wall ? by_ks<PREC, MODEL, true>(ks) : by_ks<PREC, MODEL, false>(ks);
}

template <int PREC>
StepperKernel by_model(int model, bool wall, int ks) {
    if (model == FPT_MODEL_QUADRATIC) return by_wall<PREC, FPT_MODEL_QUADRATIC>(wall, ks);
    if (model == FPT_MODEL_CONSTANT) return by_wall<PREC, FPT_MODEL_CONSTANT>(wall, ks);
    if (model == FPT_MODEL_POLYNOMIAL) return by_wall<PREC, FPT_MODEL_POLYNOMIAL>(wall, ks);
    return StepperKernel{nullptr, 0, nullptr};
}

}  // namespace

StepperKernel stepper_f32(int precision, int model, bool wall, int k_steps) {
    if (precision == FPT_PREC_F32_KAHAN) return by_model<FPT_PREC_F32_KAHAN>(model, wall, k_steps);
    if (precision == FPT_PREC_F32_F64ACC) return by_model<FPT_PREC_F32_F64ACC>(model, wall, k_steps);
    return StepperKernel{nullptr, 0, nullptr};
}

}  // namespace fpt
