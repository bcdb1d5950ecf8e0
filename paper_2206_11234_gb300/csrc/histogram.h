// Launch interface of the weighted-histogram kernels.
#pragma once
#include <cuda_runtime.h>

#include "fpt.h"
#include "status.h"

namespace fpt {

// One histogram over records [first, first + n) of (N, ln w).
struct HistSeg {
    long long first;              // first record
    long long n;                  // number of records
    unsigned long long id_offset; // global id of record `first` (jackknife subset = id mod n_sub)
    double lo, hi, d;             // range (lo, hi], bin width d = (hi - lo)/n_bins
    int n_bins, n_sub;
    long long bin0;               // first output bin of this histogram
};

size_t hist_smem_bytes(int max_nb);

// Enqueue the four histogram kernels for n_segs segments (device array
// d_segs).  max_nb = max over segments of n_bins * n_sub, max_n = max records.
// status: device status word (nullable), written only by FPT_DEBUG checks.
// bin_idx (nullable): one int per record, indexed like N; pass 1 stores each
// record's bin there (-1 outside the range) and pass 2 reads it instead of
// classifying the record again.
cudaError_t hist_launch(const HistSeg* d_segs, int n_segs, int max_nb, long long max_n,
                        const double* N, const double* lw, fpt_bin* bins, fpt_hist_counts* counts,
                        int n_sm, cudaStream_t stream, unsigned* status, int* bin_idx = nullptr);

}  // namespace fpt
