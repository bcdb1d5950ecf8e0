// Type-erased access to the stepper instantiations (one per precision, model,
// wall and block length), used by the C ABI layer.
#pragma once
#include <cuda_runtime.h>

#include "stepper_types.h"

namespace fpt {

struct StepperKernel {
    const void* func;     // for occupancy queries; nullptr = no such instantiation
    int warp_smem_bytes;  // dynamic shared memory per warp (replay queue + parking)
    cudaError_t (*launch)(const StepperParams&, int grid, int block, cudaStream_t stream);
};

inline size_t stepper_smem(const StepperKernel& k, int block, int n_sets) {
    return stepper_table_bytes(n_sets) + (size_t)(block / 32) * (size_t)k.warp_smem_bytes;
}

// Block lengths with an instantiation: binary32 8/16/32/64, binary64 4/8; the
// power-law bias (model = kModelPowReal in binary64): binary32 32, binary64 4/8.
StepperKernel stepper_f32(int precision, int model, bool wall, int k_steps);
StepperKernel stepper_f64(int model, bool wall, int k_steps);
StepperKernel stepper_f32_pow(int precision, double p, bool wall, int k_steps);

}  // namespace fpt
