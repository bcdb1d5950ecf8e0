// Persistent stepper with the learned bias b(phi, N) (FPT_BIAS_MLP).
//
// Same scheme as the constant-bias stepper (stepper.cuh: one lane per run,
// blocks of KS steps without per-step branches, a per-warp queue of finished
// runs replayed 32 at a time, refills from a ticket counter), with one CTA of
// 128 threads = one tensor-core tile: at the start of every block all 128
// lanes evaluate b at their own (phi, N elapsed) (mlp.cuh: one tcgen05 MMA for
// the hidden layer, the rest on the CUDA cores) and hold it for the block.  With B = b S the weight term of a step is
// -(b xi sqrt(dN) + b^2 dN / 2) (arXiv:2206.11234 §2.2 Eqs. (12)-(14)), so a
// block adds -b sqrt(dN) Xi - b^2 n dN / 2 with Xi its sum of normals and n
// its steps; the running ln w is kept in binary64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "abi_internal.h"
#include "fpt.h"
#include "mlp.cuh"
#include "stepper.cuh"

namespace fpt {
namespace {

constexpr int kMlpTmemCols = 64;

struct PendingMlp {
    unsigned long long rec;  // record index
    double lw;               // ln w before the block
    int m0;                  // step count at the block start
    int set;
    float phi0;              // phi at the block start
    float b;                 // bias amplitude of the block
};

struct RecordSink {
    fpt_mlp_record* out;
    unsigned long long cap;
    unsigned long long* count;
};

// Append one record per lane with `want` set (one atomic per warp).
__device__ __forceinline__ void emit_records(const RecordSink& sink, bool want, float phi0, float N0, float xi,
                                             unsigned long long rec) {
    if (!sink.count) return;
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mask = __ballot_sync(FULL, want);
    if (!mask) return;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(sink.count, (unsigned long long)__popc(mask));
    base = __shfl_sync(FULL, base, leader);
    if (want) {
        const unsigned long long at = base + __popc(mask & ((1u << lane) - 1u));
        if (at < sink.cap) sink.out[at] = fpt_mlp_record{phi0, N0, xi, (uint32_t)rec};
    }
}

template <int KS>
__device__ __forceinline__ void replay_mlp(const PendingMlp* q, int cnt, const StepperParams& P,
                                           const SetConst* s_sets, const RecordSink& sink, unsigned lane,
                                           unsigned long long& my_steps) {
    const unsigned mask = cnt >= 32 ? 0xffffffffu : ((1u << cnt) - 1u);
    bool have = (int)lane < cnt;
    PendingMlp e{};
    if (have) e = q[lane];
    const SetConst& S = s_sets[have ? e.set : 0];
    ModelStep<float, FPT_MODEL_QUADRATIC> model;
    model.load(S);
    model.tc = __fmul_rn(e.b, S.f_cmdN);
    const float phi_end = S.f_phi_end, twouv = S.f_twouv;
    const PhiloxLane pl = philox_lane(S.traj_offset + (e.rec - (unsigned long long)S.first), S.set_id, P.keys);
    float ph = e.phi0, prev = e.phi0, s2 = 0.f;
    int M = 0;
    bool crossed = false;
    if (have) {
        for (int gg = 0; gg < KS / 16; ++gg) {
            uint32_t V[12];
            philox_group(pl, ((uint32_t)e.m0 >> 4) + (uint32_t)gg, P.keys, V);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const NormalPair np = group_pair_f32(V, j, p);
                    const float q = __fmul_rn(model.kq, np.rho);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (M == 0) {
                            const float trig = h == 0 ? np.c : np.s;
                            prev = ph;
                            ph = model.step(ph, __fmaf_rn(q, trig, model.tc));
                            ph = fminf(ph, twouv - ph);
                            s2 = __fmaf_rn(np.rho, trig, s2);
                            const int step_index = e.m0 + 16 * gg + 4 * j + 2 * p + h;
                            if (ph <= phi_end) {
                                crossed = true;
                                M = step_index + 1;
                            } else if (step_index + 1 >= S.m_max) {
                                M = step_index + 1;
                            }
                        }
                    }
                }
            }
            if (__all_sync(mask, M != 0)) break;
        }
    }
    __syncwarp();
    const float xisum = -kSqrt2Ln2 * s2;  // the block's sum of normals up to the last step
    emit_records(sink, have, e.phi0, __fmul_rn((float)e.m0, S.f_dN), xisum, e.rec);
    if (!have) return;
    const float bsq = __fmul_rn(e.b, S.f_sq);
    const float hb2 = __fmul_rn(0.5f * e.b, __fmul_rn(e.b, S.f_dN));
    const double lw = e.lw + (double)(-bsq * xisum - hb2 * (float)(M - e.m0));
    double N;
    if (crossed) {
        const double a = (double)prev, c = (double)ph, pe = (double)phi_end;
        N = ((double)(M - 1) + (a - pe) / (a - c)) * S.dN;
    } else {
        N = __longlong_as_double(0x7ff0000000000000ll);
    }
    P.out_N[e.rec] = N;
    P.out_logw[e.rec] = lw;
    my_steps += (unsigned long long)M;
}

// The bound caps the kernel at 64 registers (16 bytes spilled; 72 without
// it), for a schedule that waits less on dependencies (6.93e11 against
// 6.80e11 steps/s on the learned-bias workload when measured).  Residency is
// 6 CTAs per SM, set by the ~34.5 KB of shared memory each holds (the tile's
// 26 KB of operands and parameters and 8 KB of replay queues); at 5 CTAs,
// with the earlier three-MMA tile of 44 KB, the kernel ran at the same speed.
template <int KS>
__global__ void __launch_bounds__(128, 8) stepper_mlp_kernel(const StepperParams P, const fpt_mlp_params* __restrict__ W,
                                                          const RecordSink sink) {
    extern __shared__ __align__(1024) unsigned char s_dyn[];
    MlpTile& F = *reinterpret_cast<MlpTile*>(s_dyn);
    const size_t off_sets = (sizeof(MlpTile) + 15) / 16 * 16;
    SetConst* s_sets = reinterpret_cast<SetConst*>(s_dyn + off_sets);
    const int n_sets = P.n_sets;
    long long* s_first = reinterpret_cast<long long*>(s_dyn + off_sets + (size_t)n_sets * sizeof(SetConst));
    unsigned char* s_queue = s_dyn + off_sets + stepper_table_bytes(n_sets);
    const unsigned tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u, lt_mask = (1u << lane) - 1u;
    PendingMlp* q = reinterpret_cast<PendingMlp*>(s_queue) + warp * kQueueCap;
    // lane state parked during a replay lives in the MLP's A tile, which holds
    // nothing between two bias evaluations (mlp_tile_forward waits for the
    // last MMA that reads it)
    static_assert(sizeof(F.A) >= 128 * 10 * 4, "park area");
    static_assert(KS % 16 == 0, "a bias block is a whole number of 16-step Philox groups");
    volatile unsigned* v = reinterpret_cast<volatile unsigned*>(F.A) + tid;

    if (warp == 0) {
        tc::tmem_alloc(&F.tmem, kMlpTmemCols);
        tc::tmem_relinquish();
        tc::fence_before_sync();
    }
    for (int i = tid; i < n_sets; i += blockDim.x) {
        s_sets[i] = P.sets[i];
        s_first[i] = P.sets[i].first;
    }
    if (tid == 0) s_first[n_sets] = (long long)P.n_total;
    mlp_tile_load(F, W);  // ends with __syncthreads
    tc::fence_after_sync();

    const unsigned FULL = 0xffffffffu;
    bool live = false, exhausted = false;
    int set = 0, m = 0, m_max = 0;
    unsigned long long rec = 0;
    float phi = 2.f, phi_end = 0.f, twouv = 0.f;
    double lw = 0.0;
    PhiloxLane pl{0u, 0u, 0u};
    ModelStep<float, FPT_MODEL_QUADRATIC> model;
    model.load(s_sets[0]);
    unsigned long long my_steps = 0;
    int q_count = 0;
    uint32_t phase = 0;

    for (;;) {
        // ---- refill (per warp) ----
        for (;;) {
            const bool want = !live && !exhausted;
            const unsigned need = __ballot_sync(FULL, want);
            if (need == 0u) break;
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(&P.scratch->ticket, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (want) {
                const unsigned long long t = base + (unsigned long long)__popc(need & lt_mask);
                if (t >= P.n_total) {
                    exhausted = true;
                } else {
                    int lo = 0, hi = n_sets - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((long long)t >= s_first[mid]) lo = mid; else hi = mid - 1;
                    }
                    set = lo;
                    const SetConst& S = s_sets[set];
                    rec = t;
                    pl = philox_lane(S.traj_offset + (t - (unsigned long long)S.first), S.set_id, P.keys);
                    model.load(S);
                    phi = S.f_phi_in;
                    phi_end = S.f_phi_end;
                    twouv = S.f_twouv;
                    m = 0;
                    m_max = S.m_max;
                    lw = 0.0;
                    if (S.phi_in <= S.phi_end) {
                        P.out_N[t] = 0.0;
                        P.out_logw[t] = 0.0;
                    } else {
                        live = true;
                    }
                }
            }
        }
        if (!__syncthreads_or(live)) break;

        // ---- the learned bias at the block start, 128 runs per tensor-core tile ----
        const SetConst& S = s_sets[set];
        const float b = mlp_tile_forward(F, phi, __fmul_rn((float)m, S.f_dN), phase);
        model.tc = __fmul_rn(b, S.f_cmdN);

        // ---- one block of KS steps ----
        const float phi0 = phi;
        const int m0 = m;
        float mn = phi, srho = 0.f;
        const uint32_t G0 = (uint32_t)m0 >> 4;
        pipelined_groups<KS>(pl, G0, P.keys, [&](const uint32_t* V, int j) {
            quad_block_f32<true>(model, V, j, twouv, phi, mn, srho);
        });
        const float sblk = -kSqrt2Ln2 * srho;  // the block's sum of normals
        m = m0 + KS;
        const bool event = live && (mn <= phi_end || m >= m_max);
        const bool through = live && !event;
        // a block that did not end the run: fold its weight and (training) record it
        if (through) {
            const float bsq = __fmul_rn(b, S.f_sq);
            const float hb2 = __fmul_rn(0.5f * b, __fmul_rn(b, S.f_dN));
            lw += (double)(-bsq * sblk - hb2 * (float)KS);
        }
        emit_records(sink, through, phi0, __fmul_rn((float)m0, S.f_dN), sblk, rec);
        const unsigned ev = __ballot_sync(FULL, event);
        if (ev) {
            if (event) {
                PendingMlp& slot = q[q_count + __popc(ev & lt_mask)];
                slot.rec = rec;
                slot.lw = lw;
                slot.m0 = m0;
                slot.set = set;
                slot.phi0 = phi0;
                slot.b = b;
                live = false;
            }
            q_count += __popc(ev);
            if (q_count >= 32) {
                const int stride = (int)blockDim.x;
                park_f(v, 0 * stride, phi);
                park_d(v, 1 * stride, stride, lw);  // words 1, 2
                park(v, 3 * stride, (unsigned)m);
                park(v, 4 * stride, (unsigned)rec);
                park(v, 5 * stride, (unsigned)(rec >> 32));
                park(v, 6 * stride, (unsigned)set | (live ? 0x40000000u : 0u) | (exhausted ? 0x80000000u : 0u));
                park(v, 7 * stride, pl.r1_x0);
                park(v, 8 * stride, pl.r1_x1);
                park(v, 9 * stride, pl.r1_set);
                __syncwarp();
                replay_mlp<KS>(q, 32, P, s_sets, sink, lane, my_steps);
                __syncwarp();
                const int rest = q_count - 32;
                PendingMlp tmp;
                if ((int)lane < rest) tmp = q[32 + lane];
                __syncwarp();
                if ((int)lane < rest) q[lane] = tmp;
                __syncwarp();
                q_count = rest;
                phi = unpark_f(v, 0 * stride);
                lw = unpark_d(v, 1 * stride, stride);
                m = (int)unpark(v, 3 * stride);
                rec = (unsigned long long)unpark(v, 4 * stride) | ((unsigned long long)unpark(v, 5 * stride) << 32);
                const unsigned sf = unpark(v, 6 * stride);
                set = (int)(sf & 0x3fffffffu);
                live = (sf & 0x40000000u) != 0u;
                exhausted = (sf & 0x80000000u) != 0u;
                pl.r1_x0 = unpark(v, 7 * stride);
                pl.r1_x1 = unpark(v, 8 * stride);
                pl.r1_set = unpark(v, 9 * stride);
                const SetConst& S2 = s_sets[set];
                model.load(S2);
                phi_end = S2.f_phi_end;
                twouv = S2.f_twouv;
                m_max = S2.m_max;
            }
        }
    }
    if (q_count > 0) {
        __syncwarp();
        replay_mlp<KS>(q, q_count, P, s_sets, sink, lane, my_steps);
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_xor_sync(FULL, my_steps, o);
    if (lane == 0) {
        atomicAdd(&P.scratch->steps, my_steps);
        if (P.steps_out) atomicAdd(P.steps_out, my_steps);
    }
    __syncthreads();
    if (tid == 0 && F.status) atomicOr(&P.scratch->status, F.status);
    if (warp == 0) {
        // after an expired wait the last commit may still be pending: wait for
        // it once more (bounded) before the columns are released
        if (F.status) tc::mbar_wait(&F.mbar, phase ^ 1u);
        tc::tmem_dealloc(F.tmem, kMlpTmemCols);
    }
}

size_t stepper_mlp_smem(int n_sets) {
    return (sizeof(MlpTile) + 15) / 16 * 16 + stepper_table_bytes(n_sets) + 4 * kQueueCap * sizeof(PendingMlp);
}

template <int KS>
int launch_mlp(const StepperParams& a, const fpt_mlp_params* W, const RecordSink& sink, int n_sets,
               cudaStream_t st) {
    const void* func = (const void*)stepper_mlp_kernel<KS>;
    const size_t smem = stepper_mlp_smem(n_sets);
    int n_sm = 0;
    int rc = device_sm_count(&n_sm);
    if (rc) return rc;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "learned-bias stepper shared memory");
    // every resident CTA holds kMlpTmemCols TMEM columns until it exits
    int per_sm = 0;
    rc = resident_ctas(func, 128, smem, kMlpTmemCols, &per_sm);
    if (rc) return rc;
    if (per_sm < 1) return fail(FPT_EUNSUPPORTED, "learned-bias stepper does not fit on an SM");
    const unsigned long long full = (unsigned long long)per_sm * n_sm;
    const unsigned long long need = (a.n_total + 127) / 128;
    const int grid = (int)(need < full ? (need < 1 ? 1 : need) : full);
    stepper_mlp_kernel<KS><<<grid, 128, smem, st>>>(a, W, sink);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "learned-bias stepper launch");
    return FPT_OK;
}

}  // namespace
}  // namespace fpt

using namespace fpt;

extern "C" int fpt_simulate_mlp(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                                double* out_N, double* out_logw, fpt_mlp_record* records,
                                int64_t record_capacity, int64_t* n_records_out) {
    NvtxRange nvtx_range("fpt_simulate_mlp");
    if (!p) return fail(FPT_EINVAL, "params is NULL");
    if (p->bias_kind != FPT_BIAS_MLP) return fail(FPT_EINVAL, "fpt_simulate_mlp needs bias_kind FPT_BIAS_MLP");
    if (!p->mlp) return fail(FPT_EINVAL, "mlp parameters are NULL");
    if ((reinterpret_cast<uintptr_t>(p->mlp) & 15u) != 0) return fail(FPT_EINVAL, "mlp parameters must be 16-byte aligned");
    if (p->precision != FPT_PREC_F32_F64ACC)
        return fail(FPT_EUNSUPPORTED, "the learned bias runs with FPT_PREC_F32_F64ACC");
    if (p->model != FPT_MODEL_QUADRATIC) return fail(FPT_EUNSUPPORTED, "the learned bias runs on the quadratic model");
    const int ks = p->k_eval ? p->k_eval : 32;
    if (ks != 16 && ks != 32 && ks != 64 && ks != 128)
        return fail(FPT_EINVAL, "k_eval %d not in {16, 32, 64, 128}", ks);
    if (record_capacity < 0) return fail(FPT_EINVAL, "record_capacity < 0");
    fpt_params q = *p;
    q.bias_kind = FPT_BIAS_CONST;  // the generic checks below treat the set data only
    int rc = check_params(&q);
    if (rc) return rc;
    Prepared P;
    rc = prepare(&q, sets, n_sets, false, &P);
    if (rc) return rc;
    if (P.n_total >= (1ull << 32)) return fail(FPT_EINVAL, "at most 2^32 - 1 runs per call");
    if (P.n_total > 0 && (!out_N || !out_logw)) return fail(FPT_EINVAL, "output pointer is NULL");
    if (n_records_out) *n_records_out = 0;
    if (P.n_total == 0) return FPT_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(p->stream);
    WorkspaceLayout L;
    workspace_layout(P, &L);
    std::vector<unsigned char> img;
    workspace_image(P, L, &img);
    const size_t off_cnt = L.bytes;
    unsigned char* ws = nullptr;
    cudaError_t e = lib_malloc_async(reinterpret_cast<void**>(&ws), L.bytes + 256, st);
    if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    std::vector<unsigned char> img2(img);
    img2.resize(L.bytes + 256, 0);
    e = cudaMemcpyAsync(ws, img2.data(), img2.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "workspace upload");
    StepperParams a;
    a.keys = philox_keys(seed);
    a.sets = reinterpret_cast<const SetConst*>(ws + L.off_sets);
    a.n_sets = (int)P.sets.size();
    a.n_total = P.n_total;
    a.out_N = out_N;
    a.out_logw = out_logw;
    a.scratch = reinterpret_cast<StepperScratch*>(ws + L.off_scratch);
    a.steps_out = reinterpret_cast<unsigned long long*>(p->steps_out);
    RecordSink sink;
    sink.out = records;
    sink.cap = (unsigned long long)record_capacity;
    sink.count = records ? reinterpret_cast<unsigned long long*>(ws + off_cnt) : nullptr;
    const fpt_mlp_params* W = static_cast<const fpt_mlp_params*>(p->mlp);
    if (!rc) {
        if (ks == 16) rc = launch_mlp<16>(a, W, sink, a.n_sets, st);
        else if (ks == 32) rc = launch_mlp<32>(a, W, sink, a.n_sets, st);
        else if (ks == 64) rc = launch_mlp<64>(a, W, sink, a.n_sets, st);
        else rc = launch_mlp<128>(a, W, sink, a.n_sets, st);
    }
    StepperScratch host;
    unsigned long long count = 0;
    if (!rc) {
        e = cudaMemcpyAsync(&host, ws + L.off_scratch, sizeof(host), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&count, ws + off_cnt, sizeof(count), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "status readback");
    }
    cudaError_t ef = cudaFreeAsync(ws, st);
    if (rc) return rc;
    if (ef != cudaSuccess) return cuda_fail(ef, "workspace free");
    if (host.status) return fail(FPT_EDEVICE_STATUS, "learned-bias stepper: a tensor-core wait expired");
    if (n_records_out) *n_records_out = (int64_t)count;
    if (records && count > (unsigned long long)record_capacity)
        return fail(FPT_ENOMEM, "record buffer holds %lld records, the run produced %llu",
                    (long long)record_capacity, count);
    return FPT_OK;
}
