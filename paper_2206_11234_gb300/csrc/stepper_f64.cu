// Binary64 (reference) instantiations of the persistent stepper.  Built with
// FMA contraction off (-fmad=false) so that every operation of the update is
// rounded exactly as written, like the FP64 CPU definition it is checked
// against.
#include "stepper.cuh"
#include "stepper_launch.h"

namespace fpt {
namespace {

template <int MODEL, bool WALL, int KS>
cudaError_t launch(const StepperParams& a, int grid, int block, cudaStream_t stream) {
    const size_t smem = stepper_table_bytes(a.n_sets) + (size_t)(block / 32) * warp_smem_bytes<double, FPT_PREC_F64>();
    stepper_kernel<double, FPT_PREC_F64, MODEL, WALL, KS><<<grid, block, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int MODEL, bool WALL, int KS>
StepperKernel make() {
    return StepperKernel{(const void*)stepper_kernel<double, FPT_PREC_F64, MODEL, WALL, KS>,
                         warp_smem_bytes<double, FPT_PREC_F64>(), &launch<MODEL, WALL, KS>};
}

template <int MODEL, bool WALL>
StepperKernel by_ks(int ks) {
    switch (ks) {
        case 4: return make<MODEL, WALL, 4>();
        case 8: return make<MODEL, WALL, 8>();
        default: return StepperKernel{nullptr, 0, nullptr};
    }
}

template <int MODEL>
StepperKernel by_wall(bool wall, int ks) {
    return wall ? by_ks<MODEL, true>(ks) : by_ks<MODEL, false>(ks);
}

}  // namespace

StepperKernel stepper_f64(int model, bool wall, int k_steps) {
    if (model == FPT_MODEL_QUADRATIC) return by_wall<FPT_MODEL_QUADRATIC>(wall, k_steps);
    if (model == FPT_MODEL_CONSTANT) return by_wall<FPT_MODEL_CONSTANT>(wall, k_steps);
    if (model == FPT_MODEL_POLYNOMIAL) return by_wall<FPT_MODEL_POLYNOMIAL>(wall, k_steps);
    if (model == kModelPowReal) return by_wall<kModelPowReal>(wall, k_steps);
    return StepperKernel{nullptr, 0, nullptr};
}

}  // namespace fpt
