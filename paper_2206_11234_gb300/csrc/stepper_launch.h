// Type-erased access to the stepper instantiations (one per precision, model,
// wall and block length), used by the C ABI layer.
#pragma once
#include <cuda_runtime.h>

#include "stepper_types.h"

namespace fpt {

struct StepperArgs {
    const SetConst* sets;
    int n_sets;
    unsigned long long n_total;
    uint32_t key0, key1;
    double* out_N;
    double* out_logw;
    StepperScratch* scratch;
    unsigned long long* steps_out;
};

struct StepperKernel {
    const void* func;  // for occupancy queries; nullptr = no such instantiation
    cudaError_t (*launch)(const StepperArgs&, int grid, int block, cudaStream_t stream);
};

// Block lengths with an instantiation: binary32 8/16/32, binary64 4/8.
StepperKernel stepper_f32(int precision, int model, bool wall, int k_steps);
StepperKernel stepper_f64(int model, bool wall, int k_steps);

}  // namespace fpt
