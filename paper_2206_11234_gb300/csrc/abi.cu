// C ABI of the library (include/fpt.h): argument checks, per-set constants,
// stream-ordered workspace, kernel dispatch and the device status readback.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "abi_internal.h"
#include "fpt.h"
#include "histogram.h"
#include "stepper_launch.h"

namespace fpt {

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

namespace {
std::atomic<int> g_fail_allocs{0};
std::atomic<unsigned> g_inject_status{0u};

bool take_alloc_failure() {
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    return false;
}
}  // namespace

cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    if (take_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

cudaError_t lib_malloc_from_pool_async(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t st) {
    if (take_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

// The library's stream-ordered memory pool, one per device, created on first
// use, for the allocations made afresh at every call (call workspaces, the
// host-buffer entry's device buffers).  Its release threshold is the maximum,
// so what one call frees stays mapped for the next; the default pool returns
// memory to the system at every synchronisation, and mapping tens or hundreds
// of megabytes again costs milliseconds per call.
cudaError_t library_pool(cudaMemPool_t* out) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

cudaError_t lib_malloc_retained_async(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool;
    cudaError_t e = library_pool(&pool);
    if (e != cudaSuccess) return e;
    return lib_malloc_from_pool_async(p, bytes, pool, st);
}

cudaError_t lib_malloc(void** p, size_t bytes) {
    if (take_alloc_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

unsigned take_injected_status() { return g_inject_status.exchange(0u); }

int cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) return fail(FPT_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FPT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int device_sm_count(int* n_sm) {
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(FPT_EUNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        cache[dev] = v;
    }
    *n_sm = cache[dev];
    return FPT_OK;
}

// c0 = 1/(2 pi sqrt 6): S = H/(2 pi) with H = m phi / sqrt 6 for V = m^2 phi^2 / 2, M_Pl = 1
// (§1 Eq. (4), §2.3 Eq. (17), §3 Eq. (25)).
static const double kC0 = 1.0 / (2.0 * 3.14159265358979323846 * std::sqrt(6.0));

int check_params(const fpt_params* p) {
    if (!p) return fail(FPT_EINVAL, "params is NULL");
    if (p->abi_version != FPT_ABI_VERSION)
        return fail(FPT_EINVAL, "abi_version %d, library is %d", p->abi_version, FPT_ABI_VERSION);
    if (p->model != FPT_MODEL_QUADRATIC && p->model != FPT_MODEL_CONSTANT && p->model != FPT_MODEL_POLYNOMIAL)
        return fail(FPT_EINVAL, "unknown model %d", p->model);
    if (p->model == FPT_MODEL_POLYNOMIAL) {
        bool any = false;
        for (int k = 0; k < FPT_POLY_TERMS; ++k) {
            if (!std::isfinite(p->poly[k])) return fail(FPT_EINVAL, "poly[%d] is not finite", k);
            any = any || p->poly[k] != 0.0;
        }
        if (!any) return fail(FPT_EINVAL, "the polynomial potential is zero");
    }
    if (p->precision != FPT_PREC_F64 && p->precision != FPT_PREC_F32_KAHAN &&
        p->precision != FPT_PREC_F32_F64ACC)
        return fail(FPT_EINVAL, "unknown precision %d", p->precision);
    if (p->bias_kind != FPT_BIAS_CONST && p->bias_kind != FPT_BIAS_POWER && p->bias_kind != FPT_BIAS_MLP)
        return fail(FPT_EINVAL, "unknown bias_kind %d", p->bias_kind);
    if (p->bias_kind == FPT_BIAS_MLP)
        return fail(FPT_EUNSUPPORTED, "the learned bias runs through fpt_simulate_mlp");
    if (p->bias_kind == FPT_BIAS_POWER) {
        if (p->model != FPT_MODEL_QUADRATIC)
            return fail(FPT_EUNSUPPORTED, "the power-law bias is defined for the quadratic model");
        if (!std::isfinite(p->bias_p) || std::fabs(p->bias_p) > 64.0)
            return fail(FPT_EINVAL, "bias_p %g must be finite with |p| <= 64", p->bias_p);
    }
    if (p->model == FPT_MODEL_CONSTANT && !(p->s0 > 0.0 && std::isfinite(p->s0) && std::isfinite(p->a0)))
        return fail(FPT_EINVAL, "constant model needs finite a0 and s0 > 0");
    if (p->block_dim != 0 && (p->block_dim < 32 || p->block_dim > kStepperMaxThreads || p->block_dim % 32))
        return fail(FPT_EINVAL, "block_dim %d (0 or a multiple of 32 in [32, %d])", p->block_dim,
                    kStepperMaxThreads);
    if (p->k_steps < 0) return fail(FPT_EINVAL, "k_steps %d < 0", p->k_steps);
    return FPT_OK;
}

int make_set_const(const fpt_params* p, const fpt_set& s, long long first, SetConst* out) {
    if (s.n_traj < 0) return fail(FPT_EINVAL, "n_traj %lld < 0", (long long)s.n_traj);
    if (!(s.dN > 0.0) || !std::isfinite(s.dN)) return fail(FPT_EINVAL, "dN must be finite and > 0");
    if (!(s.n_max > 0.0) || !std::isfinite(s.n_max)) return fail(FPT_EINVAL, "n_max must be finite and > 0");
    if (!std::isfinite(s.phi_in) || !std::isfinite(s.phi_end) || std::isnan(s.phi_uv))
        return fail(FPT_EINVAL, "phi_in, phi_end must be finite and phi_uv not NaN");
    if (s.phi_in > s.phi_uv) return fail(FPT_EINVAL, "phi_in %g above the wall phi_uv %g", s.phi_in, s.phi_uv);
    if (!std::isfinite(s.b)) return fail(FPT_EINVAL, "bias must be finite");
    if (p->model == FPT_MODEL_QUADRATIC && !(s.m > 0.0 && std::isfinite(s.m) && s.phi_end > 0.0))
        return fail(FPT_EINVAL, "quadratic model needs m > 0 and phi_end > 0");
    if (p->model == FPT_MODEL_POLYNOMIAL) {
        auto V = [&](double x) {
            double v = 0.0;
            for (int k = FPT_POLY_TERMS - 1; k >= 0; --k) v = v * x + p->poly[k];
            return v;
        };
        if (!(V(s.phi_in) > 0.0) || !(V(s.phi_end) > 0.0))
            return fail(FPT_EINVAL, "the potential must be positive at phi_in and phi_end");
        if (std::isfinite(s.phi_uv) && !(V(s.phi_uv) > 0.0))
            return fail(FPT_EINVAL, "the potential must be positive at the wall");
    }
    const double steps = std::ceil(s.n_max / s.dN);
    if (!(steps <= 2147483647.0 - 64.0))
        return fail(FPT_EINVAL, "n_max/dN = %g steps exceeds the 2^31 step limit", steps);
    SetConst c;
    std::memset(&c, 0, sizeof(c));
    c.phi_in = s.phi_in;
    c.phi_end = s.phi_end;
    c.phi_uv = s.phi_uv;
    c.twouv = 2.0 * s.phi_uv;
    c.dN = s.dN;
    c.sq = std::sqrt(s.dN);
    c.b = s.b;
    c.a0 = p->a0;
    c.cm = (p->model == FPT_MODEL_QUADRATIC) ? kC0 * s.m : p->s0;
    c.lw_bsq = s.b * c.sq;
    c.lw_half_b2dN = 0.5 * s.b * s.b * s.dN;
    c.first = first;
    c.traj_offset = s.traj_offset;
    c.m_max = (int)steps;
    c.set_id = s.set_id;
    c.f_cmdN = (float)(c.cm * s.dN);
    c.f_dN = (float)s.dN;
    c.f_sq = (float)c.sq;
    c.f_phi_in = (float)s.phi_in;
    c.f_phi_end = (float)s.phi_end;
    c.f_twouv = (float)c.twouv;
    const double psi_per_phi = 1.0 / std::sqrt(2.0 * s.dN);
    c.f_psi_in = (float)(psi_per_phi * s.phi_in);
    c.f_psi_end = (float)(psi_per_phi * s.phi_end);
    c.f_psi_twouv = (float)(psi_per_phi * c.twouv);
    // binary32 step constants; the noise coefficient carries -sqrt(2 ln 2), the
    // factor between the stepper's Box–Muller radius rho and the normal (rng.cuh)
    const double neg_sqrt2ln2 = -1.1774100225154747;
    if (p->bias_kind == FPT_BIAS_POWER) {
        // B = A_p phi^p: dphi/phi = A_p dN phi^(p-1) + c m sqrt(dN) xi - 2 dN / phi^2;
        // the step's log-weight is -beta sqrt(dN) xi - beta^2 dN / 2 with beta = B/S = (A_p/c m) phi^(p-1)
        c.pw = p->bias_p;
        c.f_c1 = (float)(s.b * s.dN);                        // A_p dN, times phi^(p-1)
        c.f_c2 = (float)(neg_sqrt2ln2 * c.cm * c.sq);
        c.f_c3 = (float)(-2.0 * s.dN);
        c.f_pm1 = (float)(p->bias_p - 1.0);
        c.f_pw1 = (float)(-s.b / (c.cm * c.cm));
        c.f_pw2 = (float)(-0.5 * s.b * s.b * s.dN / (c.cm * c.cm));
    } else if (p->model == FPT_MODEL_POLYNOMIAL) {
        // dphi = S (b dN + sqrt(dN) xi) + D dN with D = -V'/V and S = sqrt(V) / (2 pi sqrt 3)
        c.cm = 0.0;
        for (int k = 0; k < FPT_POLY_TERMS; ++k) {
            c.poly[k] = p->poly[k];
            c.f_poly[k] = (float)p->poly[k];
            c.f_dpoly[k] = k + 1 < FPT_POLY_TERMS ? (float)((double)(k + 1) * p->poly[k + 1]) : 0.0f;
        }
        c.f_c1 = (float)(s.b * s.dN);                        // bias part of dphi / S
        c.f_c2 = (float)(neg_sqrt2ln2 * c.sq);               // noise part of dphi / S per unit rho cos
        c.f_c3 = (float)s.dN;
    } else if (p->model == FPT_MODEL_QUADRATIC) {
        c.f_c1 = (float)(s.b * c.cm * s.dN);                 // bias part of dphi/phi
        c.f_c2 = (float)(neg_sqrt2ln2 * c.cm * c.sq);        // noise part of dphi/phi per unit rho cos
        c.f_c3 = (float)(-2.0 * s.dN);                       // drift part of dphi, times phi
    } else {
        c.f_c1 = (float)((p->a0 + s.b * p->s0) * s.dN);
        c.f_c2 = (float)(neg_sqrt2ln2 * p->s0 * c.sq);
        c.f_c3 = 0.0f;
    }
    *out = c;
    return FPT_OK;
}

int check_hist(int32_t n_bins, double lo, double hi, int32_t n_sub) {
    if (n_bins < 1 || n_sub < 1) return fail(FPT_EINVAL, "n_bins %d and n_sub %d must be >= 1", n_bins, n_sub);
    if ((long long)n_bins * n_sub > FPT_MAX_HIST_BINS)
        return fail(FPT_EINVAL, "n_sub * n_bins = %lld exceeds %d", (long long)n_bins * n_sub,
                    FPT_MAX_HIST_BINS);
    if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi))
        return fail(FPT_EINVAL, "histogram range needs finite lo < hi");
    return FPT_OK;
}

int prepare(const fpt_params* p, const fpt_set* sets, int n_sets, bool with_hist, Prepared* P) {
    if (!sets) return fail(FPT_EINVAL, "sets is NULL");
    if (n_sets < 1 || n_sets > FPT_MAX_SETS) return fail(FPT_EINVAL, "n_sets %d not in [1, %d]", n_sets, FPT_MAX_SETS);
    P->sets.resize(n_sets);
    P->segs.clear();
    P->n_total = 0;
    P->wall = false;
    P->max_nb = 1;
    P->max_n = 0;
    P->total_bins = 0;
    for (int i = 0; i < n_sets; ++i) {
        int rc = make_set_const(p, sets[i], (long long)P->n_total, &P->sets[i]);
        if (rc) return rc;
        P->wall = P->wall || std::isfinite(sets[i].phi_uv);
        if (with_hist) {
            rc = check_hist(sets[i].n_bins, sets[i].hist_lo, sets[i].hist_hi, 1);
            if (rc) return rc;
            HistSeg h;
            h.first = (long long)P->n_total;
            h.n = sets[i].n_traj;
            h.id_offset = sets[i].traj_offset;
            h.lo = sets[i].hist_lo;
            h.hi = sets[i].hist_hi;
            h.d = (h.hi - h.lo) / (double)sets[i].n_bins;
            h.n_bins = sets[i].n_bins;
            h.n_sub = 1;
            h.bin0 = P->total_bins;
            P->segs.push_back(h);
            P->total_bins += sets[i].n_bins;
            if (sets[i].n_bins > P->max_nb) P->max_nb = sets[i].n_bins;
            if (sets[i].n_traj > P->max_n) P->max_n = sets[i].n_traj;
        }
        P->n_total += (unsigned long long)sets[i].n_traj;
    }
    return FPT_OK;
}

int pick_stepper(const fpt_params* p, bool wall, StepperKernel* k, int* block) {
    int b = p->block_dim;
    int s = p->k_steps;
    if (p->bias_kind == FPT_BIAS_POWER) {
        if (b == 0) b = 256;
        if (p->precision == FPT_PREC_F64) {
            *k = stepper_f64(kModelPowReal, wall, s == 0 ? 4 : s);
        } else {
            *k = stepper_f32_pow(p->precision, p->bias_p, wall, s == 0 ? 32 : s);
        }
        if (!k->func) return fail(FPT_EINVAL, "k_steps %d not available for the power-law bias", s);
        *block = b;
        return FPT_OK;
    }
    if (b == 0 || s == 0) {
        int tb = 0, ts = 0;
        if (tuned_shape(p->precision, p->model, wall, &tb, &ts)) {
            if (b == 0) b = tb;
            if (s == 0) s = ts;
        }
    }
    if (b == 0) b = 256;
    if (p->precision == FPT_PREC_F64) {
        if (s == 0) s = 4;
        *k = stepper_f64(p->model, wall, s);
    } else {
        if (s == 0) s = 16;
        *k = stepper_f32(p->precision, p->model, wall, s);
    }
    if (!k->func) return fail(FPT_EINVAL, "k_steps %d not available for precision %d", s, p->precision);
    *block = b;
    return FPT_OK;
}

int stepper_grid(const StepperKernel& k, int block, int n_sets, unsigned long long n_total, int* grid) {
    int n_sm = 0;
    int rc = device_sm_count(&n_sm);
    if (rc) return rc;
    int per_sm = 0;
    const size_t smem = stepper_smem(k, block, n_sets);
    cudaError_t e = cudaFuncSetAttribute(k.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "stepper shared memory");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.func, block, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const unsigned long long full = (unsigned long long)per_sm * n_sm;
    const unsigned long long need = (n_total + block - 1) / block;
    *grid = (int)(need < full ? (need < 1 ? 1 : need) : full);
    return FPT_OK;
}

int resident_ctas(const void* func, int threads, size_t dyn_smem, int tmem_cols, int* per_sm) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    int dev = 0, smem_sm = 0, reserved = 0, max_blocks = 0, regs_sm = 0, max_threads = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&max_blocks, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const size_t smem_block = dyn_smem + fa.sharedSizeBytes + (size_t)reserved;
    const int warps = (threads + 31) / 32;
    const int regs_block = ((fa.numRegs * 32 + 255) / 256) * 256 * warps;  // 256-register warp granules
    int n = max_blocks;
    n = std::min(n, (int)((size_t)smem_sm / smem_block));
    n = std::min(n, regs_block > 0 ? regs_sm / regs_block : n);
    n = std::min(n, max_threads / threads);
    if (tmem_cols > 0) n = std::min(n, 512 / tmem_cols);
    *per_sm = n;
    return FPT_OK;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void workspace_layout(const Prepared& P, WorkspaceLayout* L) {
    L->off_scratch = 0;
    L->off_sets = align_up(sizeof(StepperScratch), 256);
    L->off_segs = align_up(L->off_sets + P.sets.size() * sizeof(SetConst), 256);
    L->bytes = align_up(L->off_segs + P.segs.size() * sizeof(HistSeg), 256);
    L->off_bin_idx = L->bytes;
    L->total = P.segs.empty() ? L->bytes : L->bytes + align_up((size_t)P.n_total * sizeof(int), 256);
}

void workspace_image(const Prepared& P, const WorkspaceLayout& L, std::vector<unsigned char>* img) {
    img->assign(L.bytes, 0);
    std::memcpy(img->data() + L.off_sets, P.sets.data(), P.sets.size() * sizeof(SetConst));
    if (!P.segs.empty()) std::memcpy(img->data() + L.off_segs, P.segs.data(), P.segs.size() * sizeof(HistSeg));
}

// Enqueue stepper (+ histogram) on `stream` using a workspace whose image has
// already been copied to `ws`.
int enqueue_run(const fpt_params* p, const Prepared& P, const WorkspaceLayout& L, unsigned char* ws,
                uint64_t seed, double* out_N, double* out_logw, fpt_bin* bins, fpt_hist_counts* counts,
                cudaStream_t stream, const std::function<int()>& after_stepper) {
    StepperKernel k;
    int block = 0, grid = 0;
    int rc = pick_stepper(p, P.wall, &k, &block);
    if (rc) return rc;
    rc = stepper_grid(k, block, (int)P.sets.size(), P.n_total, &grid);
    if (rc) return rc;
    StepperParams a;
    a.keys = philox_keys(seed);
    a.sets = reinterpret_cast<const SetConst*>(ws + L.off_sets);
    a.n_sets = (int)P.sets.size();
    a.n_total = P.n_total;
    a.out_N = out_N;
    a.out_logw = out_logw;
    a.scratch = reinterpret_cast<StepperScratch*>(ws + L.off_scratch);
    a.steps_out = reinterpret_cast<unsigned long long*>(p->steps_out);
    if (P.n_total > 0) {
        cudaError_t e = k.launch(a, grid, block, stream);
        if (e != cudaSuccess) return cuda_fail(e, "stepper launch");
    }
    if (after_stepper) {
        rc = after_stepper();
        if (rc) return rc;
    }
    if (bins) {
        int n_sm = 0;
        rc = device_sm_count(&n_sm);
        if (rc) return rc;
        unsigned* status = reinterpret_cast<unsigned*>(ws + L.off_scratch + offsetof(StepperScratch, status));
        int* bin_idx = L.total > L.bytes ? reinterpret_cast<int*>(ws + L.off_bin_idx) : nullptr;
        cudaError_t e = hist_launch(reinterpret_cast<const HistSeg*>(ws + L.off_segs), (int)P.segs.size(),
                                    P.max_nb, P.max_n, out_N, out_logw, bins, counts, n_sm, stream, status,
                                    bin_idx);
        if (e != cudaSuccess) return cuda_fail(e, "histogram launch");
    }
    return FPT_OK;
}

int read_status(const unsigned char* ws, const WorkspaceLayout& L, cudaStream_t stream,
                StepperScratch* host) {
    cudaError_t e = cudaMemcpyAsync(host, ws + L.off_scratch, sizeof(StepperScratch),
                                    cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "status readback");
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (host->status != 0u) return fail(FPT_EDEVICE_STATUS, "device status 0x%x", host->status);
    return FPT_OK;
}

// One complete call: stream-ordered workspace, upload, enqueue, status, free.
// after_stepper: as for enqueue_run.
int run_once(const fpt_params* p, const Prepared& P, uint64_t seed, double* out_N, double* out_logw,
             fpt_bin* bins, fpt_hist_counts* counts, const std::function<int()>& after_stepper = {}) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(p->stream);
    WorkspaceLayout L;
    workspace_layout(P, &L);
    std::vector<unsigned char> img;
    workspace_image(P, L, &img);
    // status bits injected by the host (fpt_inject_status) start the call's status word
    const unsigned injected = take_injected_status();
    std::memcpy(img.data() + L.off_scratch + offsetof(StepperScratch, status), &injected, sizeof(injected));
    unsigned char* ws = nullptr;
    cudaError_t e = lib_malloc_retained_async(reinterpret_cast<void**>(&ws), L.total, stream);
    if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    // pageable source: the copy is staged before the call returns
    e = cudaMemcpyAsync(ws, img.data(), L.bytes, cudaMemcpyHostToDevice, stream);
    int rc = (e != cudaSuccess) ? cuda_fail(e, "workspace upload") : FPT_OK;
    if (!rc) rc = enqueue_run(p, P, L, ws, seed, out_N, out_logw, bins, counts, stream, after_stepper);
    StepperScratch host;
    if (!rc) rc = read_status(ws, L, stream, &host);
    cudaError_t ef = cudaFreeAsync(ws, stream);
    if (!rc && ef != cudaSuccess) rc = cuda_fail(ef, "workspace free");
    return rc;
}

}  // namespace fpt

using namespace fpt;

extern "C" {

int fpt_simulate(const fpt_params* p, int64_t n_traj, double phi_in, double phi_end, double phi_uv,
                 double dN, double bias, uint64_t seed, double* out_N, double* out_logw) {
    NvtxRange nvtx_range("fpt_simulate");
    int rc = check_params(p);
    if (rc) return rc;
    if (n_traj < 0) return fail(FPT_EINVAL, "n_traj %lld < 0", (long long)n_traj);
    if (n_traj > 0 && (!out_N || !out_logw)) return fail(FPT_EINVAL, "output pointer is NULL");
    fpt_set s;
    std::memset(&s, 0, sizeof(s));
    s.phi_in = phi_in;
    s.phi_end = phi_end;
    s.phi_uv = phi_uv;
    s.m = p->m;
    s.b = bias;
    s.dN = dN;
    s.n_max = p->n_max;
    s.n_traj = n_traj;
    s.traj_offset = p->traj_offset;
    s.set_id = p->set_id;
    Prepared P;
    rc = prepare(p, &s, 1, false, &P);
    if (rc) return rc;
    if (n_traj == 0) return FPT_OK;
    return run_once(p, P, seed, out_N, out_logw, nullptr, nullptr);
}

int fpt_simulate_batch(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                       double* out_N, double* out_logw, fpt_bin* out_bins, fpt_hist_counts* out_counts) {
    NvtxRange nvtx_range("fpt_simulate_batch");
    int rc = check_params(p);
    if (rc) return rc;
    if ((out_bins == nullptr) != (out_counts == nullptr))
        return fail(FPT_EINVAL, "out_bins and out_counts must both be set or both be NULL");
    Prepared P;
    rc = prepare(p, sets, n_sets, out_bins != nullptr, &P);
    if (rc) return rc;
    if (P.n_total > 0 && (!out_N || !out_logw)) return fail(FPT_EINVAL, "output pointer is NULL");
    return run_once(p, P, seed, out_N, out_logw, out_bins, out_counts);
}

int fpt_histogram(const double* N, const double* logw, int64_t n, int32_t n_bins, double lo, double hi,
                  int32_t n_sub, uint64_t id_offset, fpt_bin* bins, fpt_hist_counts* counts, void* stream) {
    NvtxRange nvtx_range("fpt_histogram");
    if (n < 0) return fail(FPT_EINVAL, "n %lld < 0", (long long)n);
    int rc = check_hist(n_bins, lo, hi, n_sub);
    if (rc) return rc;
    if (!bins || !counts || (n > 0 && (!N || !logw))) return fail(FPT_EINVAL, "pointer is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HistSeg h;
    h.first = 0;
    h.n = n;
    h.id_offset = id_offset;
    h.lo = lo;
    h.hi = hi;
    h.d = (hi - lo) / (double)n_bins;
    h.n_bins = n_bins;
    h.n_sub = n_sub;
    h.bin0 = 0;
    // workspace: the segment, then the status word (zero), then (not uploaded)
    // one int per record for the bin index of pass 1
    struct HistWork {
        HistSeg seg;
        unsigned status;
    } hw{};
    hw.seg = h;
    const size_t off_idx = align_up(sizeof(HistWork), 256);
    HistWork* d_w = nullptr;
    cudaError_t e = lib_malloc_retained_async(reinterpret_cast<void**>(&d_w), off_idx + (size_t)n * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "histogram workspace");
    int* bin_idx = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(d_w) + off_idx);
    e = cudaMemcpyAsync(d_w, &hw, sizeof(HistWork), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "histogram upload");
    int n_sm = 0;
    if (!rc) rc = device_sm_count(&n_sm);
    if (!rc) {
        e = hist_launch(&d_w->seg, 1, n_bins * n_sub, n, N, logw, bins, counts, n_sm, st, &d_w->status,
                        bin_idx);
        if (e != cudaSuccess) rc = cuda_fail(e, "histogram launch");
    }
    unsigned status = 0u;
    if (!rc) {
        e = cudaMemcpyAsync(&status, &d_w->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "status readback");
    }
    cudaError_t ef = cudaFreeAsync(d_w, st);
    if (!rc) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "stream synchronize");
    }
    if (!rc && ef != cudaSuccess) rc = cuda_fail(ef, "histogram workspace free");
    if (!rc && status != 0u) rc = fail(FPT_EDEVICE_STATUS, "device status 0x%x", status);
    return rc;
}

namespace {

// A non-blocking stream per device for the host entry's record copies,
// created on first use and kept for the life of the process.
cudaError_t copy_stream(cudaStream_t* out) {
    static std::mutex mu;
    static std::vector<cudaStream_t> streams;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)streams.size() <= dev) streams.resize(dev + 1, nullptr);
    if (!streams[dev]) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        streams[dev] = s;
    }
    *out = streams[dev];
    return cudaSuccess;
}
}  // namespace

int fpt_simulate_batch_host(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                            double* host_N, double* host_logw, fpt_bin* host_bins,
                            fpt_hist_counts* host_counts) {
    NvtxRange nvtx_range("fpt_simulate_batch_host");
    int rc = check_params(p);
    if (rc) return rc;
    if (!host_bins || !host_counts) return fail(FPT_EINVAL, "host_bins and host_counts are required");
    Prepared P;
    rc = prepare(p, sets, n_sets, true, &P);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(p->stream);
    const size_t rec_bytes = (size_t)P.n_total * sizeof(double);
    const size_t bin_bytes = (size_t)P.total_bins * sizeof(fpt_bin);
    const size_t cnt_bytes = (size_t)n_sets * sizeof(fpt_hist_counts);
    unsigned char* dev = nullptr;
    const size_t o_N = 0, o_lw = (rec_bytes + 255) / 256 * 256;
    const size_t o_bins = o_lw + (rec_bytes + 255) / 256 * 256;
    const size_t o_cnt = o_bins + (bin_bytes + 255) / 256 * 256;
    const size_t total = o_cnt + cnt_bytes;
    cudaMemPool_t pool;
    cudaError_t e = library_pool(&pool);
    if (e != cudaSuccess) return cuda_fail(e, "memory pool");
    e = lib_malloc_from_pool_async(reinterpret_cast<void**>(&dev), total, pool, st);
    if (e != cudaSuccess) return cuda_fail(e, "device buffers");
    double* dN_ = reinterpret_cast<double*>(dev + o_N);
    double* dlw = reinterpret_cast<double*>(dev + o_lw);
    fpt_bin* db = reinterpret_cast<fpt_bin*>(dev + o_bins);
    fpt_hist_counts* dc = reinterpret_cast<fpt_hist_counts*>(dev + o_cnt);
    // The records are final when the stepper ends: copy them to the host on a
    // second stream while the histogram kernels (which only read them) run.
    cudaStream_t side = nullptr;
    cudaEvent_t stepper_done = nullptr, copied = nullptr;
    e = copy_stream(&side);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&stepper_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy stream");
    bool side_used = false;
    if (!rc) {
        // the side stream waits for the stepper; it is enqueued before the
        // histogram so that the copies start as soon as the stepper ends
        rc = run_once(p, P, seed, dN_, dlw, db, dc, [&]() -> int {
            cudaError_t ec = cudaEventRecord(stepper_done, st);
            if (ec != cudaSuccess) return cuda_fail(ec, "event record");
            ec = cudaStreamWaitEvent(side, stepper_done, 0);
            if (ec != cudaSuccess) return cuda_fail(ec, "copy stream wait");
            side_used = true;
            if (host_N && rec_bytes) {
                ec = cudaMemcpyAsync(host_N, dN_, rec_bytes, cudaMemcpyDeviceToHost, side);
                if (ec != cudaSuccess) return cuda_fail(ec, "copy N to host");
            }
            if (host_logw && rec_bytes) {
                ec = cudaMemcpyAsync(host_logw, dlw, rec_bytes, cudaMemcpyDeviceToHost, side);
                if (ec != cudaSuccess) return cuda_fail(ec, "copy logw to host");
            }
            return FPT_OK;
        });
    }
    if (side_used) {
        // the buffers are freed on `st` only after the side stream's copies
        cudaError_t ec = cudaEventRecord(copied, side);
        if (ec == cudaSuccess) ec = cudaStreamWaitEvent(st, copied, 0);
        if (!rc && ec != cudaSuccess) rc = cuda_fail(ec, "copy stream join");
        if (ec != cudaSuccess) cudaStreamSynchronize(side);
    }
    if (!rc) {
        e = cudaMemcpyAsync(host_bins, db, bin_bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy bins to host");
    }
    if (!rc) {
        e = cudaMemcpyAsync(host_counts, dc, cnt_bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy counts to host");
    }
    cudaError_t ef = cudaFreeAsync(dev, st);
    e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "stream synchronize");
    if (!rc && ef != cudaSuccess) rc = cuda_fail(ef, "device buffers free");
    if (stepper_done) cudaEventDestroy(stepper_done);
    if (copied) cudaEventDestroy(copied);
    return rc;
}

const char* fpt_strerror(int code) {
    switch (code) {
        case FPT_OK: return "ok";
        case FPT_EINVAL: return "invalid argument";
        case FPT_ECUDA: return "CUDA error";
        case FPT_ENOMEM: return "out of device memory";
        case FPT_EUNSUPPORTED: return "unsupported";
        case FPT_EDEVICE_STATUS: return "device status error";
        default: return "unknown error";
    }
}

const char* fpt_last_error(void) { return g_last_error.c_str(); }

int fpt_abi_version(void) { return FPT_ABI_VERSION; }

int fpt_inject_alloc_failures(int32_t count) {
    if (count < 0) return fail(FPT_EINVAL, "count %d < 0", count);
    g_fail_allocs.store(count);
    return FPT_OK;
}

int fpt_inject_status(uint32_t bits) {
    g_inject_status.store(bits);
    return FPT_OK;
}

}  // extern "C"
