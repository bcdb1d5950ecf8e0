// Per-bin estimates of the first-passage-time density from a weighted
// histogram (arXiv:2206.11234): the direct / weighted estimate (§2.1 Eq. (9),
// §2.2 Eq. (16)) with its standard error, the lognormal estimate and its error
// bars (§2.4 Eqs. (22)-(24)), the D'Agostino-Pearson normality test of ln w
// that decides whether the lognormal estimate applies (§2.4), and jackknife
// errors over the histogram's n_sub subsets (§2.1); the multi-bias
// reconstruction of §3.2 (estimates of the same bins from several bias
// amplitudes, combined where they overlap); and Pearson's r of (N, ln w) over
// all runs, the measure of §3.4's search for the power-law bias.
//
// One thread per bin, binary64 throughout.  The thread reads the bin's n_sub
// subset entries, each holding max-shifted sums about its own maximum, and
// merges them about the common maximum M: s1, s2 rescale by exp(m_k - M), and
// the moments sum x^r (x = ln w - m_k) re-centre binomially with
// delta_k = m_k - M:  sum (x + delta)^r = sum_i C(r, i) delta^(r-i) sum x^i.
// Central moments then follow from the moments about M; since every x is
// within the bin's spread of M, the cancellation is mild in binary64.
//
// The normality statistics: sqrt(b1) = m3 / m2^1.5 is mapped to a normal
// deviate with D'Agostino's (1970) Johnson S_U transform, b2 = m4 / m2^2 with
// Anscombe and Glynn's (1983) cube-root transform, and K^2 = Z1^2 + Z2^2 is
// chi^2 with 2 degrees of freedom, so p = exp(-K^2 / 2) (D'Agostino, Belanger
// and D'Agostino 1990).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "abi_internal.h"
#include "fpt.h"

namespace fpt {
namespace {

struct BinSums {
    double mx, s1, s2, n;
    double l[5];  // l[0] = n, l[r] = sum x^r about mx
};

__device__ __forceinline__ BinSums load_bin(const fpt_bin& b) {
    BinSums s;
    s.mx = b.max_lw;
    s.s1 = b.s1;
    s.s2 = b.s2;
    s.n = (double)b.count;
    s.l[0] = s.n;
    s.l[1] = b.l1;
    s.l[2] = b.l2;
    s.l[3] = b.l3;
    s.l[4] = b.l4;
    return s;
}

// runs of subset k among ids id_offset .. id_offset + n_total - 1 (subset = id mod n_sub)
__device__ __forceinline__ double subset_total(long long n_total, unsigned long long id_offset, int n_sub, int k) {
    const long long base = n_total / n_sub, rem = n_total % n_sub;
    const int first = (int)(id_offset % (unsigned long long)n_sub);
    const int pos = (k - first + n_sub) % n_sub;
    return (double)(base + (pos < rem ? 1 : 0));
}

__device__ __forceinline__ double direct_p(const BinSums& s, double n_total, double d) {
    return s.n > 0.0 ? exp(s.mx) * s.s1 / (n_total * d) : 0.0;
}

// mean and unbiased variance of x (about mx) from the moments
__device__ __forceinline__ void mean_var(const BinSums& s, double* mean, double* var) {
    const double a1 = s.l[1] / s.n, a2 = s.l[2] / s.n;
    *mean = a1;
    *var = fmax(a2 - a1 * a1, 0.0) * s.n / (s.n - 1.0);
}

__device__ __forceinline__ double lognormal_p(const BinSums& s, double n_total, double d) {
    if (s.n == 0.0) return 0.0;
    if (s.n < 2.0) return nan("");
    double mean, var;
    mean_var(s, &mean, &var);
    return s.n * exp(s.mx + mean + 0.5 * var) / (n_total * d);
}

__device__ double skew_z(double g, double n) {
    const double y = g * sqrt((n + 1.0) * (n + 3.0) / (6.0 * (n - 2.0)));
    const double beta2 = 3.0 * (n * n + 27.0 * n - 70.0) * (n + 1.0) * (n + 3.0) /
                         ((n - 2.0) * (n + 5.0) * (n + 7.0) * (n + 9.0));
    const double w2 = -1.0 + sqrt(2.0 * (beta2 - 1.0));
    const double delta = 1.0 / sqrt(0.5 * log(w2));
    const double alpha = sqrt(2.0 / (w2 - 1.0));
    return delta * asinh(y / alpha);
}

__device__ double kurt_z(double b2, double n) {
    const double mean = 3.0 * (n - 1.0) / (n + 1.0);
    const double var = 24.0 * n * (n - 2.0) * (n - 3.0) / ((n + 1.0) * (n + 1.0) * (n + 3.0) * (n + 5.0));
    const double x = (b2 - mean) / sqrt(var);
    const double sb1 = 6.0 * (n * n - 5.0 * n + 2.0) / ((n + 7.0) * (n + 9.0)) *
                       sqrt(6.0 * (n + 3.0) * (n + 5.0) / (n * (n - 2.0) * (n - 3.0)));
    const double A = 6.0 + 8.0 / sb1 * (2.0 / sb1 + sqrt(1.0 + 4.0 / (sb1 * sb1)));
    const double t = (1.0 - 2.0 / A) / (1.0 + x * sqrt(2.0 / (A - 4.0)));
    return ((1.0 - 2.0 / (9.0 * A)) - cbrt(t)) / sqrt(2.0 / (9.0 * A));
}

__global__ void estimate_kernel(const fpt_bin* __restrict__ bins, int n_bins, int n_sub, double lo, double hi,
                                long long n_total, unsigned long long id_offset, fpt_estimate_bin* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_bins) return;
    const double d = (hi - lo) / n_bins;
    const double nt = (double)n_total;
    const double qnan = nan("");
    fpt_estimate_bin o;
    // ---- merge the subsets about the common maximum ----
    double M = -INFINITY;
    for (int k = 0; k < n_sub; ++k) {
        const fpt_bin& b = bins[(long long)k * n_bins + j];
        if (b.count > 0) M = fmax(M, b.max_lw);
    }
    BinSums A{M, 0.0, 0.0, 0.0, {0.0, 0.0, 0.0, 0.0, 0.0}};
    for (int k = 0; k < n_sub; ++k) {
        const fpt_bin& b = bins[(long long)k * n_bins + j];
        if (b.count <= 0) continue;
        const BinSums s = load_bin(b);
        const double dl = s.mx - M, sc = exp(dl);
        A.s1 += s.s1 * sc;
        A.s2 += s.s2 * sc * sc;
        A.n += s.n;
        // binomial re-centring, Horner in delta: sum_i C(r, i) delta^(r - i) l_i
        const double d2 = dl * dl;
        A.l[1] += s.l[1] + dl * s.l[0];
        A.l[2] += s.l[2] + 2.0 * dl * s.l[1] + d2 * s.l[0];
        A.l[3] += s.l[3] + 3.0 * dl * s.l[2] + 3.0 * d2 * s.l[1] + d2 * dl * s.l[0];
        A.l[4] += s.l[4] + 4.0 * dl * s.l[3] + 6.0 * d2 * s.l[2] + 4.0 * d2 * dl * s.l[1] + d2 * d2 * s.l[0];
    }
    A.l[0] = A.n;
    o.count = A.n;
    // ---- direct / weighted estimate (Eqs. (9), (16)) ----
    if (A.n > 0.0) {
        const double e = exp(M);
        o.p_direct = e * A.s1 / (nt * d);
        const double v = A.s2 / nt - (A.s1 / nt) * (A.s1 / nt);
        o.se_direct = e * sqrt(fmax(v, 0.0) / nt) / d;
    } else {
        o.p_direct = 0.0;
        o.se_direct = 0.0;
    }
    // ---- lognormal estimate (Eqs. (22)-(24)) ----
    o.mean_lw = qnan;
    o.var_lw = qnan;
    if (A.n == 0.0) {
        o.p_lognormal = o.eps_lo = o.eps_hi = 0.0;
    } else if (A.n < 2.0) {
        o.mean_lw = M + A.l[1] / A.n;
        o.p_lognormal = o.eps_lo = o.eps_hi = qnan;
    } else {
        double mean, var;
        mean_var(A, &mean, &var);
        o.mean_lw = M + mean;
        o.var_lw = var;
        const double p = A.n * exp(o.mean_lw + 0.5 * var) / (nt * d);
        const double a = sqrt(var / A.n + var * var / (2.0 * A.n - 2.0));
        o.p_lognormal = p;
        o.eps_hi = p * expm1(a);
        o.eps_lo = -p * expm1(-a);
    }
    // ---- D'Agostino-Pearson normality of ln w ----
    o.skew = o.kurt = o.z_skew = o.z_kurt = o.k2 = o.p_normal = qnan;
    if (A.n >= 8.0 && o.var_lw > 0.0) {
        const double n = A.n;
        const double a1 = A.l[1] / n, a2 = A.l[2] / n, a3 = A.l[3] / n, a4 = A.l[4] / n;
        const double m2 = a2 - a1 * a1;
        const double m3 = a3 - 3.0 * a1 * a2 + 2.0 * a1 * a1 * a1;
        const double m4 = a4 - 4.0 * a1 * a3 + 6.0 * a1 * a1 * a2 - 3.0 * a1 * a1 * a1 * a1;
        if (m2 > 0.0) {
            o.skew = m3 / (m2 * sqrt(m2));
            o.kurt = m4 / (m2 * m2);
            o.z_skew = skew_z(o.skew, n);
            o.z_kurt = kurt_z(o.kurt, n);
            o.k2 = o.z_skew * o.z_skew + o.z_kurt * o.z_kurt;
            o.p_normal = exp(-0.5 * o.k2);
        }
    }
    // ---- the next cumulant terms of ln <w>: k3/6 + k4/24 (k-statistics) ----
    o.bias_ln = o.bias_se = qnan;
    if (A.n >= 4.0 && o.var_lw > 0.0) {
        const double n = A.n;
        const double a1 = A.l[1] / n, a2 = A.l[2] / n, a3 = A.l[3] / n, a4 = A.l[4] / n;
        const double m2 = a2 - a1 * a1;
        const double m3 = a3 - 3.0 * a1 * a2 + 2.0 * a1 * a1 * a1;
        const double m4 = a4 - 4.0 * a1 * a3 + 6.0 * a1 * a1 * a2 - 3.0 * a1 * a1 * a1 * a1;
        if (m2 > 0.0) {
            const double k2 = n / (n - 1.0) * m2;
            const double k3 = n * n / ((n - 1.0) * (n - 2.0)) * m3;
            const double k4 = n * n * ((n + 1.0) * m4 - 3.0 * (n - 1.0) * m2 * m2) / ((n - 1.0) * (n - 2.0) * (n - 3.0));
            const double v3 = 6.0 * n * k2 * k2 * k2 / ((n - 1.0) * (n - 2.0));
            const double v4 = 24.0 * n * (n + 1.0) * k2 * k2 * k2 * k2 / ((n - 1.0) * (n - 2.0) * (n - 3.0));
            o.bias_ln = k3 / 6.0 + k4 / 24.0;
            o.bias_se = sqrt(v3 / 36.0 + v4 / 576.0);
        }
    }
    // ---- jackknife over the subsets (§2.1) ----
    o.jk_direct = o.jk_lognormal = qnan;
    if (n_sub >= 2) {
        double sd = 0.0, sl = 0.0;
        for (int k = 0; k < n_sub; ++k) {
            const BinSums s = load_bin(bins[(long long)k * n_bins + j]);
            const double tk = subset_total(n_total, id_offset, n_sub, k);
            sd += tk > 0.0 ? direct_p(s, tk, d) : qnan;
            sl += tk > 0.0 ? lognormal_p(s, tk, d) : qnan;
        }
        const double md = sd / n_sub, ml = sl / n_sub;
        double vd = 0.0, vl = 0.0;
        for (int k = 0; k < n_sub; ++k) {
            const BinSums s = load_bin(bins[(long long)k * n_bins + j]);
            const double tk = subset_total(n_total, id_offset, n_sub, k);
            const double pd = tk > 0.0 ? direct_p(s, tk, d) : qnan;
            const double pl = tk > 0.0 ? lognormal_p(s, tk, d) : qnan;
            vd += (pd - md) * (pd - md);
            vl += (pl - ml) * (pl - ml);
        }
        o.jk_direct = sqrt(vd / (n_sub - 1)) / sqrt((double)n_sub);
        o.jk_lognormal = sqrt(vl / (n_sub - 1)) / sqrt((double)n_sub);
    }
    out[j] = o;
}

// ---- multi-bias reconstruction: inverse-variance combination in log space ----

__global__ void stitch_kernel(const fpt_estimate_bin* __restrict__ est, int n_runs, int n_bins, int estimator,
                              long long min_count, double p_threshold, fpt_stitch_bin* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_bins) return;
    double sw = 0.0, swl = 0.0, best_a = INFINITY;
    int used = 0, best = -1;
    for (int k = 0; k < n_runs; ++k) {
        const fpt_estimate_bin& e = est[(long long)k * n_bins + j];
        if (!(e.count >= (double)min_count)) continue;
        double p, a;
        if (estimator == FPT_ESTIMATOR_LOGNORMAL) {
            // w = 1 throughout the bin (var_lw = 0): a degenerate normal, the test is undefined, not failed
            if (p_threshold > 0.0 && !(e.p_normal >= p_threshold) && !(e.var_lw == 0.0)) continue;
            p = e.p_lognormal;
            // Eq. (24)'s spread of ln w plus the count's own relative fluctuation 1/n_j
            a = sqrt(e.var_lw / e.count + e.var_lw * e.var_lw / (2.0 * e.count - 2.0) + 1.0 / e.count);
        } else {
            p = e.p_direct;
            a = e.se_direct / e.p_direct;
        }
        if (!(p > 0.0) || !(a > 0.0) || !isfinite(p) || !isfinite(a)) continue;
        const double w = 1.0 / (a * a);
        sw += w;
        swl += w * log(p);
        ++used;
        if (a < best_a) {
            best_a = a;
            best = k;
        }
    }
    fpt_stitch_bin o;
    if (used > 0) {
        const double a = 1.0 / sqrt(sw);
        o.p = exp(swl / sw);
        o.log_err = a;
        o.eps_lo = -o.p * expm1(-a);
        o.eps_hi = o.p * expm1(a);
    } else {
        o.p = o.eps_lo = o.eps_hi = o.log_err = nan("");
    }
    o.n_used = (double)used;
    o.best = (double)best;
    out[j] = o;
}

// ---- Pearson's r of (N, ln w) over the finite runs ----

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // sh is reused by consecutive calls
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// pass 1: count, sum N, sum ln w -> out[1..3]
__global__ void pearson_pass1(const double* __restrict__ N, const double* __restrict__ lw, long long n,
                              double* __restrict__ out) {
    __shared__ double sh[32];
    double c = 0.0, sn = 0.0, sl = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = N[i];
        if (isfinite(x)) {
            c += 1.0;
            sn += x;
            sl += lw[i];
        }
    }
    c = block_sum(c, sh);
    sn = block_sum(sn, sh);
    sl = block_sum(sl, sh);
    if (threadIdx.x == 0 && c > 0.0) {
        atomicAdd(&out[1], c);
        atomicAdd(&out[2], sn);
        atomicAdd(&out[3], sl);
    }
}

// pass 2: centred sums of squares and products -> out[4..6]
__global__ void pearson_pass2(const double* __restrict__ N, const double* __restrict__ lw, long long n,
                              double* __restrict__ out) {
    __shared__ double sh[32];
    const double cnt = out[1];
    if (cnt == 0.0) return;
    const double mn = out[2] / cnt, ml = out[3] / cnt;
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = N[i];
        if (isfinite(x)) {
            const double dx = x - mn, dy = lw[i] - ml;
            sxx += dx * dx;
            syy += dy * dy;
            sxy += dx * dy;
        }
    }
    sxx = block_sum(sxx, sh);
    syy = block_sum(syy, sh);
    sxy = block_sum(sxy, sh);
    if (threadIdx.x == 0) {
        atomicAdd(&out[4], sxx);
        atomicAdd(&out[5], syy);
        atomicAdd(&out[6], sxy);
    }
}

__global__ void pearson_final(double* out) {
    const double c = out[1], sxx = out[4], syy = out[5], sxy = out[6];
    const double qnan = nan("");
    out[0] = (c >= 2.0 && sxx > 0.0 && syy > 0.0) ? sxy / sqrt(sxx * syy) : qnan;
    out[2] = c > 0.0 ? out[2] / c : qnan;
    out[3] = c > 0.0 ? out[3] / c : qnan;
    out[4] = c >= 2.0 ? sxx / (c - 1.0) : qnan;
    out[5] = c >= 2.0 ? syy / (c - 1.0) : qnan;
    out[6] = c >= 2.0 ? sxy / (c - 1.0) : qnan;
    out[7] = 0.0;
}

}  // namespace
}  // namespace fpt

using namespace fpt;

extern "C" int fpt_stitch(const fpt_estimate_bin* est, int32_t n_runs, int32_t n_bins, int32_t estimator,
                          int64_t min_count, double p_threshold, fpt_stitch_bin* out, void* stream) {
    NvtxRange nvtx_range("fpt_stitch");
    if (!est || !out) return fail(FPT_EINVAL, "pointer is NULL");
    if (n_runs < 1 || n_bins < 1) return fail(FPT_EINVAL, "n_runs %d and n_bins %d must be >= 1", n_runs, n_bins);
    if (estimator != FPT_ESTIMATOR_DIRECT && estimator != FPT_ESTIMATOR_LOGNORMAL)
        return fail(FPT_EINVAL, "unknown estimator %d", estimator);
    if (min_count < 2) return fail(FPT_EINVAL, "min_count %lld < 2", (long long)min_count);
    if (!(p_threshold >= 0.0 && p_threshold < 1.0)) return fail(FPT_EINVAL, "p_threshold must be in [0, 1)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int threads = 128;
    stitch_kernel<<<(n_bins + threads - 1) / threads, threads, 0, st>>>(est, n_runs, n_bins, estimator,
                                                                        (long long)min_count, p_threshold, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "stitch launch");
    return FPT_OK;
}

extern "C" int fpt_pearson(const double* N, const double* logw, int64_t n, double* out, void* stream) {
    NvtxRange nvtx_range("fpt_pearson");
    if (n < 0) return fail(FPT_EINVAL, "n %lld < 0", (long long)n);
    if (!out || (n > 0 && (!N || !logw))) return fail(FPT_EINVAL, "pointer is NULL");
    int n_sm = 0;
    int rc = device_sm_count(&n_sm);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(out, 0, 8 * sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, "pearson reset");
    const int threads = 256;
    long long want = (n + threads - 1) / threads;
    const int grid = (int)std::max(1LL, std::min(want, 2LL * n_sm));
    if (n > 0) {
        pearson_pass1<<<grid, threads, 0, st>>>(N, logw, (long long)n, out);
        pearson_pass2<<<grid, threads, 0, st>>>(N, logw, (long long)n, out);
    }
    pearson_final<<<1, 1, 0, st>>>(out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pearson launch");
    return FPT_OK;
}

extern "C" int fpt_estimate(const fpt_bin* bins, int32_t n_bins, int32_t n_sub, double lo, double hi,
                            int64_t n_total, uint64_t id_offset, fpt_estimate_bin* out, void* stream) {
    NvtxRange nvtx_range("fpt_estimate");
    if (!bins || !out) return fail(FPT_EINVAL, "pointer is NULL");
    if (n_bins < 1 || n_sub < 1 || (int64_t)n_bins * n_sub > FPT_MAX_HIST_BINS)
        return fail(FPT_EINVAL, "n_bins %d x n_sub %d not in [1, %d]", n_bins, n_sub, FPT_MAX_HIST_BINS);
    if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi)) return fail(FPT_EINVAL, "need finite lo < hi");
    if (n_total < 1) return fail(FPT_EINVAL, "n_total %lld < 1", (long long)n_total);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int threads = 128;
    estimate_kernel<<<(n_bins + threads - 1) / threads, threads, 0, st>>>(bins, n_bins, n_sub, lo, hi,
                                                                          (long long)n_total, id_offset, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "estimate launch");
    return FPT_OK;
}
