// Internal helpers shared by the C ABI translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <functional>
#include <vector>

#include "fpt.h"
#include "histogram.h"
#include "stepper_launch.h"

namespace fpt {

// Device allocations of the library's scratch.  While failures are pending
// (fpt_inject_alloc_failures) each call consumes one and returns
// cudaErrorMemoryAllocation without allocating, as a full device would.
cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t st);
cudaError_t lib_malloc_from_pool_async(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t st);
// From the library's pool, which keeps freed memory mapped (per device).
cudaError_t library_pool(cudaMemPool_t* out);
cudaError_t lib_malloc_retained_async(void** p, size_t bytes, cudaStream_t st);
cudaError_t lib_malloc(void** p, size_t bytes);
// Status bits to pre-set in the next uploaded stepper scratch (fpt_inject_status), consumed.
unsigned take_injected_status();

// NVTX range over one entry point (shows the library's calls on a profiler's
// timeline; free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Record a failure message for fpt_last_error() and return `code`.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
int device_sm_count(int* n_sm);
int check_params(const fpt_params* p);
// CTAs of `func` that fit on one SM by registers, shared memory, threads and
// (tmem_cols > 0) the 512 TMEM columns; computed from the kernel's attributes,
// since the occupancy API is conservative for kernels that allocate TMEM.
int resident_ctas(const void* func, int threads, size_t dyn_smem, int tmem_cols, int* per_sm);

// Host-side image of one batched call.
struct Prepared {
    std::vector<SetConst> sets;
    std::vector<HistSeg> segs;
    unsigned long long n_total;
    bool wall;
    int max_nb;
    long long max_n;
    long long total_bins;
};

// bytes: the part uploaded from the host image (scratch, set table, histogram
// segments); total: bytes plus, with histograms, a region that is not
// uploaded: one int per record (the bin index of histogram pass 1).
struct WorkspaceLayout {
    size_t off_scratch, off_sets, off_segs, bytes;
    size_t off_bin_idx, total;
};

int prepare(const fpt_params* p, const fpt_set* sets, int n_sets, bool with_hist, Prepared* P);
int make_set_const(const fpt_params* p, const fpt_set& s, long long first, SetConst* out);
int pick_stepper(const fpt_params* p, bool wall, StepperKernel* k, int* block);
// Launch shape chosen by fpt_autotune for this device and kind of launch, if any.
bool tuned_shape(int precision, int model, bool wall, int* block, int* ks);
void clear_tuned_shapes();
int stepper_grid(const StepperKernel& k, int block, int n_sets, unsigned long long n_total, int* grid);
void workspace_layout(const Prepared& P, WorkspaceLayout* L);
void workspace_image(const Prepared& P, const WorkspaceLayout& L, std::vector<unsigned char>* img);
// Enqueues the stepper and, with bins, the histogram kernels on `stream`.
// after_stepper (optional) is called between the two, when the records are
// final and only read from then on; a nonzero return stops the enqueue.
int enqueue_run(const fpt_params* p, const Prepared& P, const WorkspaceLayout& L, unsigned char* ws,
                uint64_t seed, double* out_N, double* out_logw, fpt_bin* bins, fpt_hist_counts* counts,
                cudaStream_t stream, const std::function<int()>& after_stepper = {});

}  // namespace fpt
