// Autotuner of the stepper's launch shape: threads per block and steps per
// scheduling block (k_steps).  Pilot launches over a sample of the caller's
// own parameter sets, timed with CUDA events on the caller's stream; the
// fastest shape (EM steps per second) is cached per (device, precision,
// model, wall) and used by every call that leaves block_dim or k_steps at 0.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "abi_internal.h"
#include "fpt.h"
#include "stepper_launch.h"

namespace fpt {
namespace {

using TuneKey = std::tuple<int, int, int, int>;  // device, precision, model, wall
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;  // -> (block_dim, k_steps)

}  // namespace

bool tuned_shape(int precision, int model, bool wall, int* block, int* ks) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(TuneKey{dev, precision, model, wall ? 1 : 0});
    if (it == g_tune.end()) return false;
    *block = it->second.first;
    *ks = it->second.second;
    return true;
}

void clear_tuned_shapes() {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

}  // namespace fpt

using namespace fpt;

extern "C" int fpt_autotune(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                            double fraction, int32_t* block_dim_out, int32_t* k_steps_out,
                            double* steps_per_s_out) {
    NvtxRange nvtx_range("fpt_autotune");
    int rc = check_params(p);
    if (rc) return rc;
    if (!sets) return fail(FPT_EINVAL, "sets is NULL");
    if (!(fraction > 0.0 && fraction <= 1.0)) return fail(FPT_EINVAL, "fraction %g not in (0, 1]", fraction);
    if (n_sets < 1 || n_sets > FPT_MAX_SETS) return fail(FPT_EINVAL, "n_sets %d not in [1, %d]", n_sets, FPT_MAX_SETS);
    int n_sm = 0;
    rc = device_sm_count(&n_sm);
    if (rc) return rc;
    // pilot: each set scaled by `fraction`, but at least enough runs to fill
    // every SM several times over (the full set at most)
    long long full = 0;
    for (int i = 0; i < n_sets; ++i) full += sets[i].n_traj;
    if (full <= 0) return fail(FPT_EINVAL, "no runs to tune on");
    const double min_runs = 4.0 * n_sm * 2048.0;
    double f = fraction;
    if (f * (double)full < min_runs) f = std::fmin(1.0, min_runs / (double)full);
    std::vector<fpt_set> pilot(sets, sets + n_sets);
    for (auto& s : pilot) s.n_traj = s.n_traj > 0 ? (int64_t)std::ceil((double)s.n_traj * f) : 0;
    Prepared P;
    rc = prepare(p, pilot.data(), n_sets, false, &P);
    if (rc) return rc;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(p->stream);
    WorkspaceLayout L;
    workspace_layout(P, &L);
    std::vector<unsigned char> img;
    workspace_image(P, L, &img);
    const size_t rec_bytes = (size_t)P.n_total * sizeof(double);
    unsigned char* dev = nullptr;
    cudaError_t e = lib_malloc_async(reinterpret_cast<void**>(&dev), L.bytes + 2 * rec_bytes + 512, st);
    if (e != cudaSuccess) return cuda_fail(e, "autotune buffers");
    unsigned char* ws = dev;
    double* outN = reinterpret_cast<double*>(dev + (L.bytes + 255) / 256 * 256);
    double* outL = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(outN) + (rec_bytes + 255) / 256 * 256);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);

    const int blocks[3] = {128, 256, 512};
    const int ks32[3] = {16, 32, 64};     // binary32 block lengths (whole 16-step groups)
    const int ks64[2] = {4, 8};           // binary64
    const int ks_pow[1] = {32};          // binary32 power-law bias kernels
    const bool pw = p->bias_kind == FPT_BIAS_POWER && p->precision != FPT_PREC_F64;
    const int* kss = p->precision == FPT_PREC_F64 ? ks64 : (pw ? ks_pow : ks32);
    const int nks = p->precision == FPT_PREC_F64 ? 2 : (pw ? 1 : 3);
    double best = -1.0;
    int best_b = 256, best_k = kss[0];
    fpt_params q = *p;
    q.steps_out = nullptr;
    for (int bi = 0; bi < 3 && !rc; ++bi) {
        for (int ki = 0; ki < nks && !rc; ++ki) {
            q.block_dim = blocks[bi];
            q.k_steps = kss[ki];
            double t_best = 1e300;
            unsigned long long steps = 0;
            for (int rep = 0; rep < 3 && !rc; ++rep) {  // rep 0 warms up
                e = cudaMemcpyAsync(ws, img.data(), L.bytes, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) { rc = cuda_fail(e, "autotune upload"); break; }
                cudaEventRecord(e0, st);
                rc = enqueue_run(&q, P, L, ws, seed, outN, outL, nullptr, nullptr, st);
                if (rc) break;
                cudaEventRecord(e1, st);
                StepperScratch host;
                e = cudaMemcpyAsync(&host, ws + L.off_scratch, sizeof(host), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) { rc = cuda_fail(e, "autotune launch"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < t_best) t_best = ms;
                steps = host.steps;
            }
            if (!rc) {
                const double rate = (double)steps / (t_best * 1e-3);
                if (rate > best) {
                    best = rate;
                    best_b = blocks[bi];
                    best_k = kss[ki];
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t ef = cudaFreeAsync(dev, st);
    cudaStreamSynchronize(st);
    if (rc) return rc;
    if (ef != cudaSuccess) return cuda_fail(ef, "autotune free");
    int devi = 0;
    cudaGetDevice(&devi);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[TuneKey{devi, p->precision, p->model, P.wall ? 1 : 0}] = {best_b, best_k};
    }
    if (block_dim_out) *block_dim_out = best_b;
    if (k_steps_out) *k_steps_out = best_k;
    if (steps_per_s_out) *steps_per_s_out = best;
    return FPT_OK;
}

extern "C" void fpt_autotune_reset(void) { clear_tuned_shapes(); }
