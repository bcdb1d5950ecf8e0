// Weighted histogram of first-passage times (arXiv:2206.11234 §2.1 Eq. (9),
// §2.2 Eq. (16)), several histograms (one per parameter set) per launch.
//
// Per bin: n_j, max ln w and, with x = ln w - max <= 0, s1 = sum exp(x),
// s2 = sum exp(2 x), l_k = sum x^k for k = 1..4 (the moments of ln w behind the
// lognormal estimator and normality test of §2.4).  Two streaming passes over the
// records (HBM-resident; the passes are bound by the binary64 arithmetic, not
// by the bytes):
//   pass 1: classify each record (16 B read), per-bin max of ln w (shared-memory
//           atomicMax on an order-preserving 64-bit key, one global atomic per bin
//           and block); with a bin-index buffer, store each record's bin (4 B);
//   pass 2: read ln w and the stored bin (or classify again without the buffer),
//           max-shifted sums into shared-memory bins, lanes of a warp that hit
//           the same bin (__match_any_sync) combined by their lowest lane, one
//           peer per shuffle round, before one shared atomic per bin and warp.
// Bins are right-closed: j = ceil((N - lo)/d) - 1, clamped to [0, n_bins).
#include <cuda_runtime.h>

#include <cstdint>

#include "histogram.h"

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

constexpr unsigned long long kKeyNegInf = 0x000fffffffffffffull;  // ord_key(-inf)
constexpr int kSums = 6;  // s1, s2, l1 .. l4 per bin

// 0: in range (bin set), 1: N <= lo, 2: finite N > hi, 3: N not finite
__device__ __forceinline__ int classify(double N, const HistSeg& h, unsigned long long gid, int& bin,
                                        unsigned* status) {
    if (!(N < __longlong_as_double(0x7ff0000000000000ll))) return 3;
    if (N <= h.lo) return 1;
    if (N > h.hi) return 2;
    long long j = (long long)ceil((N - h.lo) / h.d) - 1;
#if FPT_DEBUG
    // rounding at the edges gives -1 or n_bins, which the clamp absorbs; more is a broken segment
    if ((j < -1 || j > h.n_bins) && status) atomicOr(status, kStatusHistBin);
#else
    (void)status;
#endif
    if (j < 0) j = 0;
    if (j > h.n_bins - 1) j = h.n_bins - 1;
    const int sub = (int)(gid % (unsigned long long)h.n_sub);
    bin = sub * h.n_bins + (int)j;
    return 0;
}

__global__ void hist_init(const HistSeg* __restrict__ segs, int n_segs, fpt_bin* __restrict__ bins,
                          fpt_hist_counts* __restrict__ counts) {
    const HistSeg h = segs[blockIdx.y];
    const int nb = h.n_bins * h.n_sub;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        fpt_bin* o = bins + h.bin0 + b;
        o->max_lw = __longlong_as_double((long long)kKeyNegInf);  // holds the key until hist_final
        o->s1 = 0.0;
        o->s2 = 0.0;
        o->l1 = 0.0;
        o->l2 = 0.0;
        o->l3 = 0.0;
        o->l4 = 0.0;
        o->count = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counts[blockIdx.y].under = 0;
        counts[blockIdx.y].over = 0;
        counts[blockIdx.y].censored = 0;
        counts[blockIdx.y].total = h.n;
    }
}

__global__ void hist_pass_max(const double* __restrict__ N, const double* __restrict__ lw,
                              const HistSeg* __restrict__ segs, fpt_bin* __restrict__ bins,
                              fpt_hist_counts* __restrict__ counts, unsigned* status,
                              int* __restrict__ bin_idx) {
    extern __shared__ unsigned long long s_key[];
    const HistSeg h = segs[blockIdx.y];
    const int nb = h.n_bins * h.n_sub;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s_key[b] = kKeyNegInf;
    __syncthreads();
    unsigned long long under = 0, over = 0, cens = 0;
    const unsigned lane = threadIdx.x & 31u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // warp-uniform loop: every lane of a warp runs the same iterations
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < h.n;
         base += stride) {
        const long long i = base + lane;
        int bin = -1;
        unsigned long long key = 0;
        if (i < h.n) {
            const long long r = h.first + i;
            const int cat = classify(N[r], h, h.id_offset + (unsigned long long)i, bin, status);
            under += (cat == 1);
            over += (cat == 2);
            cens += (cat == 3);
            if (cat == 0) key = ord_key(lw[r]);
            if (bin_idx) bin_idx[r] = bin;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        // the group leader (lowest lane of the bin) takes the max over its peers,
        // one peer per round: as many rounds as the largest group has members - 1
        const bool leader = (int)lane == __ffs(peers) - 1;
        unsigned rem = (leader && bin >= 0) ? (peers & ~(1u << lane)) : 0u;
        unsigned long long best = key;
        while (__any_sync(0xffffffffu, rem != 0u)) {
            const int src = rem ? __ffs(rem) - 1 : (int)lane;
            const unsigned long long v = __shfl_sync(0xffffffffu, key, src);
            if (rem) best = v > best ? v : best;
            rem &= rem - 1u;
        }
        if (bin >= 0 && leader) atomicMax(&s_key[bin], best);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (s_key[b] != kKeyNegInf)
            atomicMax(reinterpret_cast<unsigned long long*>(&bins[h.bin0 + b].max_lw), s_key[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        under += __shfl_xor_sync(0xffffffffu, under, o);
        over += __shfl_xor_sync(0xffffffffu, over, o);
        cens += __shfl_xor_sync(0xffffffffu, cens, o);
    }
    if (lane == 0 && (under | over | cens)) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&counts[blockIdx.y].under), under);
        atomicAdd(reinterpret_cast<unsigned long long*>(&counts[blockIdx.y].over), over);
        atomicAdd(reinterpret_cast<unsigned long long*>(&counts[blockIdx.y].censored), cens);
    }
}

__global__ void hist_pass_sum(const double* __restrict__ N, const double* __restrict__ lw,
                              const HistSeg* __restrict__ segs, fpt_bin* __restrict__ bins, unsigned* status,
                              const int* __restrict__ bin_idx) {
    extern __shared__ double s_acc[];  // [nb][kSums] sums, then [nb] counts
    const HistSeg h = segs[blockIdx.y];
    const int nb = h.n_bins * h.n_sub;
    unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_acc + kSums * nb);
    for (int b = threadIdx.x; b < kSums * nb; b += blockDim.x) s_acc[b] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s_cnt[b] = 0ull;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < h.n;
         base += stride) {
        const long long i = base + lane;
        int bin = -1;
        double v[kSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (i < h.n) {
            const long long r = h.first + i;
            if (bin_idx)
                bin = bin_idx[r];
            else if (classify(N[r], h, h.id_offset + (unsigned long long)i, bin, status) != 0)
                bin = -1;
            if (bin >= 0) {
                const unsigned long long k =
                    (unsigned long long)__double_as_longlong(bins[h.bin0 + bin].max_lw);
                const double x = lw[r] - ord_value(k);
                const double e = exp(x), x2 = x * x;
                v[0] = e;
                v[1] = e * e;
                v[2] = x;
                v[3] = x2;
                v[4] = x2 * x;
                v[5] = x2 * x2;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        // the group leader sums its peers' values, one peer per round (no
        // rounds when every lane of the warp has a bin of its own)
        const bool leader = (int)lane == __ffs(peers) - 1;
        unsigned rem = (leader && bin >= 0) ? (peers & ~(1u << lane)) : 0u;
        double acc[kSums];
#pragma unroll
        for (int f = 0; f < kSums; ++f) acc[f] = v[f];
        while (__any_sync(0xffffffffu, rem != 0u)) {
            const int src = rem ? __ffs(rem) - 1 : (int)lane;
#pragma unroll
            for (int f = 0; f < kSums; ++f) {
                const double y = __shfl_sync(0xffffffffu, v[f], src);
                if (rem) acc[f] += y;
            }
            rem &= rem - 1u;
        }
        if (bin >= 0 && leader) {
#pragma unroll
            for (int f = 0; f < kSums; ++f) atomicAdd(&s_acc[kSums * bin + f], acc[f]);
            atomicAdd(&s_cnt[bin], (unsigned long long)__popc(peers));
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        if (s_cnt[b] == 0ull) continue;
        fpt_bin* o = bins + h.bin0 + b;
        atomicAdd(&o->s1, s_acc[kSums * b + 0]);
        atomicAdd(&o->s2, s_acc[kSums * b + 1]);
        atomicAdd(&o->l1, s_acc[kSums * b + 2]);
        atomicAdd(&o->l2, s_acc[kSums * b + 3]);
        atomicAdd(&o->l3, s_acc[kSums * b + 4]);
        atomicAdd(&o->l4, s_acc[kSums * b + 5]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&o->count), s_cnt[b]);
    }
}

__global__ void hist_final(const HistSeg* __restrict__ segs, fpt_bin* __restrict__ bins) {
    const HistSeg h = segs[blockIdx.y];
    const int nb = h.n_bins * h.n_sub;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        fpt_bin* o = bins + h.bin0 + b;
        o->max_lw = ord_value((unsigned long long)__double_as_longlong(o->max_lw));
    }
}

}  // namespace

size_t hist_smem_bytes(int max_nb) { return (size_t)max_nb * (kSums * sizeof(double) + 8); }

cudaError_t hist_launch(const HistSeg* d_segs, int n_segs, int max_nb, long long max_n,
                        const double* N, const double* lw, fpt_bin* bins, fpt_hist_counts* counts,
                        int n_sm, cudaStream_t stream, unsigned* status, int* bin_idx) {
    const size_t smem_sum = hist_smem_bytes(max_nb);
    const size_t smem_max = (size_t)max_nb * sizeof(unsigned long long);
    // opt in to large dynamic shared memory (per device; cheap to repeat)
    cudaError_t e = cudaFuncSetAttribute(hist_pass_sum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)hist_smem_bytes(FPT_MAX_HIST_BINS));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(hist_pass_max, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(FPT_MAX_HIST_BINS * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int init_blocks = (max_nb + threads - 1) / threads;
    hist_init<<<dim3(init_blocks, n_segs), threads, 0, stream>>>(d_segs, n_segs, bins, counts);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // about two waves of blocks over all segments, at least one block per segment
    long long want = (max_n + threads * 8 - 1) / (threads * 8);
    int per_seg = (int)(want < 1 ? 1 : want);
    const int cap = (2 * n_sm + n_segs - 1) / n_segs;
    if (per_seg > cap) per_seg = cap < 1 ? 1 : cap;
    hist_pass_max<<<dim3(per_seg, n_segs), threads, smem_max, stream>>>(N, lw, d_segs, bins, counts, status,
                                                                        bin_idx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    hist_pass_sum<<<dim3(per_seg, n_segs), threads, smem_sum, stream>>>(N, lw, d_segs, bins, status, bin_idx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    hist_final<<<dim3(init_blocks, n_segs), threads, 0, stream>>>(d_segs, bins);
    return cudaGetLastError();
}

}  // namespace fpt
