// fpt_normals: the normals the stepper draws, written out for inspection
// (RNG parity checks).  Built with FMA contraction off like the binary64
// stepper, so the binary64 Box–Muller here is the stepper's bit for bit.
#include <cuda_runtime.h>

#include "abi_internal.h"
#include "fpt.h"
#include "rng.cuh"

namespace fpt {
namespace {

__global__ void philox_words_kernel(uint32_t key0, uint32_t key1, const PhiloxKeys K, unsigned long long traj,
                                    uint32_t set_id, uint32_t k0, long long n_blocks,
                                    uint32_t* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_blocks) return;
    const uint32_t c[4] = {k0 + (uint32_t)i, (uint32_t)traj, (uint32_t)(traj >> 32), set_id};
    uint32_t w[4];
    philox4x32_10(c, key0, key1, w);
    // the stepper's folded form with the host key schedule must give the same words
    const PhiloxLane l = philox_lane(traj, set_id, K);
    uint32_t v[4];
    philox_block(l, k0 + (uint32_t)i, K, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[4 * i + q] = (w[q] == v[q]) ? w[q] : 0xDEADBEEFu ^ w[q] ^ v[q];
}

template <typename Real>
__global__ void normals_kernel(const PhiloxKeys K, unsigned long long traj, uint32_t set_id,
                               uint32_t k0, long long n_blocks, Real* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_blocks) return;
    const PhiloxLane l = philox_lane(traj, set_id, K);
    Real xi[4];
    if constexpr (sizeof(Real) == 8)
        normals4_f64(l, k0 + (uint32_t)i, K, xi);
    else
        normals4_f32(l, k0 + (uint32_t)i, K, xi);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[4 * i + q] = xi[q];
}

}  // namespace
}  // namespace fpt

using namespace fpt;

extern "C" int fpt_normals(uint64_t seed, uint64_t traj, uint32_t set_id, uint32_t k0, int64_t n_blocks,
                           int32_t precision, void* out, void* stream) {
    if (n_blocks < 0 || (n_blocks > 0 && !out)) return fail(FPT_EINVAL, "n_blocks < 0 or out is NULL");
    if ((unsigned long long)k0 + (unsigned long long)n_blocks > 0x100000000ull)
        return fail(FPT_EINVAL, "k0 + n_blocks exceeds the 32-bit block counter");
    if (n_blocks == 0) return FPT_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int threads = 128;
    const long long blocks = (n_blocks + threads - 1) / threads;
    const PhiloxKeys K = philox_keys(seed);
    if (precision == FPT_NORMALS_RAW_BITS)
        philox_words_kernel<<<(unsigned)blocks, threads, 0, st>>>(
            (uint32_t)seed, (uint32_t)(seed >> 32), K, traj, set_id, k0, n_blocks, static_cast<uint32_t*>(out));
    else if (precision == FPT_PREC_F64)
        normals_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(K, traj, set_id, k0, n_blocks,
                                                                      static_cast<double*>(out));
    else if (precision == FPT_PREC_F32_KAHAN || precision == FPT_PREC_F32_F64ACC)
        normals_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(K, traj, set_id, k0, n_blocks,
                                                                     static_cast<float*>(out));
    else
        return fail(FPT_EINVAL, "unknown precision %d", precision);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "normals launch");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return FPT_OK;
}
