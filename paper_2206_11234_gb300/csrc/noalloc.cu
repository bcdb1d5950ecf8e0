// fpt_simulate_batch_noalloc: the batched stepper with its scratch in a
// fixed, file-scope device array instead of a per-call allocation.
//
// Who needs this: callers that are not allowed to allocate device memory
// while they run — a process whose device memory is entirely reserved by its
// own pool allocator or a fixed memory budget, or a latency-bound loop that
// cannot accept an allocation failing half-way through a run or the implicit
// device synchronisation of releasing memory.  They pass their own output
// buffers; the scratch the stepper needs (ticket counter, step total and
// status word in a 256-byte header, then the per-set constants of up to
// FPT_NOALLOC_MAX_SETS sets: 15,232 bytes in all) lives in g_noalloc_scratch.
//
// The array is part of the library image: every GPU that loads the library
// holds it until the process exits.  All calls share it and it keeps the last
// call's contents, so each call rewrites the whole region it uses (zeroed
// counters, fresh per-set constants) before launching.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "abi_internal.h"
#include "fpt.h"
#include "stepper_launch.h"

namespace fpt {
namespace {

constexpr size_t kScratchHeader = 256;  // StepperScratch, padded to the set table's alignment
constexpr size_t kNoAllocBytes = kScratchHeader + FPT_NOALLOC_MAX_SETS * sizeof(SetConst);
static_assert(sizeof(StepperScratch) <= kScratchHeader, "scratch header");
static_assert(kNoAllocBytes == 15232, "the size stated in fpt.h (FPT_NOALLOC_MAX_SETS) is out of date");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Identity of the calling thread's current CUDA context, through the driver
// entry points the runtime hands out (no link-time dependency on the driver
// library); 0 when it cannot be determined.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

struct CachedAddress {
    unsigned long long context;  // context the address belongs to
    void* addr;
};
std::mutex g_addr_mu;
CachedAddress g_addr[64] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol itself is only a host-side handle, so the address is looked up with
// the device current (cudaGetSymbolAddress, which also makes sure the module is
// loaded there) at set-up, the first call on a device, and cached.  The cache
// is keyed on the device's current context as well, so a new context on the
// same device (after cudaDeviceReset, or a non-primary context) repeats the
// set-up instead of reusing an address of the old one.
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(FPT_EUNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev].addr || g_addr[dev].context != current_context_id()) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // creates the device's context if needed
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_addr[dev] = CachedAddress{current_context_id(), p};
    }
    *out = static_cast<unsigned char*>(g_addr[dev].addr);
    return FPT_OK;
}

}  // namespace
}  // namespace fpt

using namespace fpt;

extern "C" int fpt_simulate_batch_noalloc(const fpt_params* p, const fpt_set* sets, int32_t n_sets,
                                          uint64_t seed, double* out_N, double* out_logw) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!sets) return fail(FPT_EINVAL, "sets is NULL");
    if (n_sets < 1 || n_sets > FPT_NOALLOC_MAX_SETS)
        return fail(FPT_EINVAL,
                    "n_sets %d: the no-alloc entry holds at most %d parameter sets in its fixed scratch",
                    n_sets, FPT_NOALLOC_MAX_SETS);
    // host image of the scratch region, on the stack
    alignas(256) unsigned char img[kNoAllocBytes];
    std::memset(img, 0, kScratchHeader);  // ticket, step total and status start at zero
    SetConst* table = reinterpret_cast<SetConst*>(img + kScratchHeader);
    unsigned long long n_total = 0;
    bool wall = false;
    for (int i = 0; i < n_sets; ++i) {
        rc = make_set_const(p, sets[i], (long long)n_total, &table[i]);
        if (rc) return rc;
        wall = wall || std::isfinite(sets[i].phi_uv);
        n_total += (unsigned long long)sets[i].n_traj;
    }
    if (n_total == 0) return FPT_OK;
    if (!out_N || !out_logw) return fail(FPT_EINVAL, "output pointer is NULL");

    StepperKernel k;
    int block = 0, grid = 0;
    rc = pick_stepper(p, wall, &k, &block);
    if (rc) return rc;
    rc = stepper_grid(k, block, n_sets, n_total, &grid);
    if (rc) return rc;
    unsigned char* ws = nullptr;
    rc = scratch_address(&ws);
    if (rc) return rc;

    cudaStream_t stream = reinterpret_cast<cudaStream_t>(p->stream);
    const size_t bytes = kScratchHeader + (size_t)n_sets * sizeof(SetConst);
    // pageable source: the runtime has taken the data before this returns
    cudaError_t e = cudaMemcpyAsync(ws, img, bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc scratch upload");

    StepperParams a;
    a.keys = philox_keys(seed);
    a.sets = reinterpret_cast<const SetConst*>(ws + kScratchHeader);
    a.n_sets = n_sets;
    a.n_total = n_total;
    a.out_N = out_N;
    a.out_logw = out_logw;
    a.scratch = reinterpret_cast<StepperScratch*>(ws);
    a.steps_out = reinterpret_cast<unsigned long long*>(p->steps_out);
    e = k.launch(a, grid, block, stream);
    if (e != cudaSuccess) return cuda_fail(e, "stepper launch");

    StepperScratch host;
    e = cudaMemcpyAsync(&host, ws, sizeof(StepperScratch), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "status readback");
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (host.status != 0u) return fail(FPT_EDEVICE_STATUS, "device status 0x%x", host.status);
    return FPT_OK;
}
