// One training step of the learned bias on the GPU.
//
// Objective: the second moment of the importance-sampling estimator of the
// tail probability P(N > N*) (§2.2 Eq. (16) summed over the tail bins),
//   L(theta) = E_S[w^2 1{N > N*}],
// whose minimiser over the sample process minimises the estimator's variance
// (P itself does not depend on theta).  Differentiating at a fixed path (the
// target measure does not depend on theta) gives
//   dL/dtheta = E_S[w^2 1_E d ln w/dtheta],  d ln w/d b_k = -sqrt(dN) Xi_k
// for the bias b_k held over block k (Xi_k = its sum of normals).  The step
// descends log L, i.e. uses the normalised coefficients c_i / sum_j c_j with
// c_i = w_i^2 1_E(i), computed with a max shift so that weights spanning
// hundreds of e-folds stay finite.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "abi_internal.h"
#include "fpt.h"

namespace fpt {
namespace {

__device__ __forceinline__ unsigned long long ord_key(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_value(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

struct TailAcc {
    unsigned long long max_key;  // ordered key of the largest ln w in the tail
    double s1, s2;               // sum exp(lw - max), sum exp(2 (lw - max)) over the tail
    unsigned long long count;    // runs in the tail
    unsigned long long n_rows;   // rows written by records_to_rows
};

__device__ __forceinline__ bool in_tail(double N, double tail_N) {
    return N > tail_N;  // +inf (censored) counts: the run lasted longer than N*
}

__global__ void tail_max(const double* __restrict__ N, const double* __restrict__ lw, long long n, double tail_N,
                         TailAcc* acc) {
    unsigned long long best = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (in_tail(N[i], tail_N)) {
            const unsigned long long k = ord_key(lw[i]);
            best = k > best ? k : best;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&acc->max_key, best);
}

__global__ void tail_sums(const double* __restrict__ N, const double* __restrict__ lw, long long n, double tail_N,
                          TailAcc* acc, double* __restrict__ coef) {
    const double mx = ord_value(acc->max_key);
    double s1 = 0.0, s2 = 0.0;
    unsigned long long c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double ci = 0.0;
        if (in_tail(N[i], tail_N)) {
            const double e = exp(lw[i] - mx);
            ci = e * e;
            s1 += e;
            s2 += ci;
            ++c;
        }
        coef[i] = ci;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0 && c) {
        atomicAdd(&acc->s1, s1);
        atomicAdd(&acc->s2, s2);
        atomicAdd(&acc->count, c);
    }
}

// Rows of the batched MLP backward: inputs of block k and
// g_k = (c_run / sum c) (-sqrt(dN) Xi_k), for the blocks of runs with c != 0
// only.  The others (runs outside the tail, or whose w^2 underflows) have
// g_k = 0 exactly and add nothing to the gradient, so they are left out: the
// rows are compacted, one atomic per warp, in no particular order (the
// backward's sums do not depend on it beyond rounding).  acc->n_rows counts
// them.
__global__ void records_to_rows(const fpt_mlp_record* __restrict__ rec, long long n_rec,
                                const double* __restrict__ coef, TailAcc* acc, double sq,
                                float* __restrict__ phi, float* __restrict__ Nin, float* __restrict__ g) {
    const double inv = acc->s2 > 0.0 ? 1.0 / acc->s2 : 0.0;
    const unsigned lane = threadIdx.x & 31u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // warp-uniform loop: every lane of a warp runs the same iterations
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31u); base < n_rec;
         base += stride) {
        const long long r = base + lane;
        fpt_mlp_record x{};
        double c = 0.0;
        if (r < n_rec) {
            x = rec[r];
            c = coef[x.run];
        }
        const bool keep = c != 0.0;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (m == 0u) continue;
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(&acc->n_rows, (unsigned long long)__popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (keep) {
            const long long o = (long long)at + __popc(m & ((1u << lane) - 1u));
            phi[o] = x.phi;
            Nin[o] = x.N;
            g[o] = (float)(c * inv * (-sq * (double)x.xi_sum));
        }
    }
}

__global__ void adam_update(float* __restrict__ master, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2, fpt_mlp_params* __restrict__ w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float p = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        master[i] = p;
        const __nv_bfloat16 h = __float2bfloat16_rn(p);
        w->w[i] = *reinterpret_cast<const uint16_t*>(&h);
    }
}

double ord_value_host(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double d;
    std::memcpy(&d, &u, sizeof(d));
    return d;
}

}  // namespace
}  // namespace fpt

using namespace fpt;

extern "C" int fpt_mlp_train_step(const fpt_params* p, const fpt_set* set, uint64_t seed, double tail_N,
                                  double lr, fpt_mlp_train_state* S, fpt_mlp_train_stats* stats) {
    NvtxRange nvtx_range("fpt_mlp_train_step");
    if (!p || !set || !S) return fail(FPT_EINVAL, "NULL argument");
    if (p->mlp != S->w) return fail(FPT_EINVAL, "p->mlp must be the state's BF16 parameters");
    if (!S->master || !S->adam_m || !S->adam_v || !S->grad || !S->w || !S->records || !S->out_N ||
        !S->out_logw || !S->coef || !S->rows)
        return fail(FPT_EINVAL, "a training buffer is NULL");
    if (!(lr > 0.0) || !std::isfinite(lr) || !std::isfinite(tail_N)) return fail(FPT_EINVAL, "bad lr or tail_N");
    if (set->n_traj < 2) return fail(FPT_EINVAL, "need at least 2 runs per step");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(p->stream);
    int64_t n_rec = 0;
    int rc = fpt_simulate_mlp(p, set, 1, seed, S->out_N, S->out_logw, S->records, S->record_capacity, &n_rec);
    if (rc) return rc;
    const long long n = set->n_traj;
    TailAcc* acc = nullptr;
    cudaError_t e = lib_malloc_async(reinterpret_cast<void**>(&acc), sizeof(TailAcc), st);
    if (e != cudaSuccess) return cuda_fail(e, "training scratch");
    cudaMemsetAsync(acc, 0, sizeof(TailAcc), st);
    int n_sm = 0;
    rc = device_sm_count(&n_sm);
    const int grid = 2 * (n_sm > 0 ? n_sm : 1);
    if (!rc) {
        tail_max<<<grid, 256, 0, st>>>(S->out_N, S->out_logw, n, tail_N, acc);
        tail_sums<<<grid, 256, 0, st>>>(S->out_N, S->out_logw, n, tail_N, acc, S->coef);
        float* rphi = S->rows;
        float* rN = S->rows + S->record_capacity;
        float* rg = S->rows + 2 * S->record_capacity;
        records_to_rows<<<4 * grid, 256, 0, st>>>(S->records, n_rec, S->coef, acc, std::sqrt(set->dN), rphi, rN, rg);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "training kernels");
        if (!rc) e = cudaMemsetAsync(S->grad, 0, sizeof(float) * FPT_MLP_NPARAM, st);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "gradient clear");
    }
    // the tail sums and the number of rows (the backward's size) on the host
    TailAcc h;
    std::memset(&h, 0, sizeof(h));
    if (!rc) {
        e = cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "tail sums");
    }
    if (!rc && h.n_rows > (unsigned long long)n_rec) rc = fail(FPT_ECUDA, "%llu rows from %lld records", h.n_rows, (long long)n_rec);
    if (!rc && h.n_rows > 0)
        rc = fpt_mlp_backward(S->w, S->rows, S->rows + S->record_capacity, S->rows + 2 * S->record_capacity,
                              (int64_t)h.n_rows, S->grad, p->stream);
    if (!rc) {
        S->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)S->step), c2 = 1.f - std::pow(b2, (float)S->step);
        adam_update<<<(FPT_MLP_NPARAM + 255) / 256, 256, 0, st>>>(S->master, S->grad, S->adam_m, S->adam_v,
                                                                 FPT_MLP_NPARAM, (float)lr, b1, b2, 1e-8f, c1, c2,
                                                                 S->w);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "Adam update");
    }
    cudaFreeAsync(acc, st);
    if (rc) return rc;
    if (stats) {
        const double mx = h.count ? ord_value_host(h.max_key) : 0.0;
        const double P = h.count ? std::exp(mx) * h.s1 / (double)n : 0.0;
        const double L = h.count ? std::exp(2.0 * mx) * h.s2 / (double)n : 0.0;
        const double var = (L - P * P) / (double)(n - 1);
        stats->log_second_moment = h.count ? 2.0 * mx + std::log(h.s2 / (double)n) : -INFINITY;
        stats->p_hat = P;
        stats->n_eff = var > 0.0 ? P * P / var : 0.0;
        stats->frac_in_tail = (double)h.count / (double)n;
        stats->n_records = n_rec;
    }
    return FPT_OK;
}
