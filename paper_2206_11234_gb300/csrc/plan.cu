// Reusable, graph-captured launch of a batched simulation (fpt_plan_*).
//
// The per-set constants are validated and uploaded once into a plan-owned
// workspace; the sequence [scratch reset, persistent stepper, histogram
// kernels, status copy to pinned host memory] is captured once into a CUDA
// graph.  Each launch only rewrites the stepper node's Philox round keys (the
// seed) and replays the graph, so a batch of many parameter sets costs one
// graph launch.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "abi_internal.h"
#include "fpt.h"
#include "stepper_launch.h"

struct fpt_plan {
    int device;
    fpt::Prepared P;
    fpt::WorkspaceLayout L;
    unsigned char* ws;
    fpt::StepperScratch* host_status;  // pinned
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t stepper_node;
    cudaKernelNodeParams knp;
    fpt::StepperParams sp;
    void* args[1];
};

using namespace fpt;

static void plan_free(fpt_plan* pl) {
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->ws) cudaFree(pl->ws);
    if (pl->host_status) cudaFreeHost(pl->host_status);
    delete pl;
}

extern "C" int fpt_plan_create(const fpt_params* p, const fpt_set* sets, int32_t n_sets, double* out_N,
                               double* out_logw, fpt_bin* out_bins, fpt_hist_counts* out_counts,
                               fpt_plan** plan_out) {
    NvtxRange nvtx_range("fpt_plan_create");
    if (!plan_out) return fail(FPT_EINVAL, "plan_out is NULL");
    *plan_out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    if ((out_bins == nullptr) != (out_counts == nullptr))
        return fail(FPT_EINVAL, "out_bins and out_counts must both be set or both be NULL");
    fpt_plan* pl = new (std::nothrow) fpt_plan();
    if (!pl) return fail(FPT_ENOMEM, "host allocation");
    rc = prepare(p, sets, n_sets, out_bins != nullptr, &pl->P);
    if (!rc && pl->P.n_total > 0 && (!out_N || !out_logw)) rc = fail(FPT_EINVAL, "output pointer is NULL");
    if (!rc && pl->P.n_total == 0) rc = fail(FPT_EINVAL, "a plan needs at least one run");
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaGetDevice(&pl->device);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGetDevice");
    }
    std::vector<unsigned char> img;
    if (!rc) {
        workspace_layout(pl->P, &pl->L);
        workspace_image(pl->P, pl->L, &img);
        e = lib_malloc(reinterpret_cast<void**>(&pl->ws), pl->L.total);
        if (e != cudaSuccess) rc = cuda_fail(e, "plan workspace");
    }
    if (!rc) {
        e = cudaMemcpy(pl->ws, img.data(), pl->L.bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&pl->host_status), sizeof(StepperScratch));
        if (e != cudaSuccess) rc = cuda_fail(e, "plan setup");
    }
    cudaStream_t cs = nullptr;
    if (!rc) {
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = cuda_fail(e, "capture stream");
    }
    if (!rc) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(e, "begin capture");
        if (!rc) {
            e = cudaMemsetAsync(pl->ws + pl->L.off_scratch, 0, sizeof(StepperScratch), cs);
            if (e != cudaSuccess) rc = cuda_fail(e, "captured scratch reset");
        }
        if (!rc) rc = enqueue_run(p, pl->P, pl->L, pl->ws, 0, out_N, out_logw, out_bins, out_counts, cs);
        if (!rc) {
            e = cudaMemcpyAsync(pl->host_status, pl->ws + pl->L.off_scratch, sizeof(StepperScratch),
                                cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) rc = cuda_fail(e, "captured status copy");
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "end capture");
        pl->graph = g;
    }
    if (cs) cudaStreamDestroy(cs);
    if (!rc) {
        e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "graph instantiate");
    }
    if (!rc) {
        // the stepper is the kernel node whose parameter is a StepperParams
        StepperKernel k;
        int block = 0;
        rc = pick_stepper(p, pl->P.wall, &k, &block);
        size_t nn = 0;
        if (!rc) e = cudaGraphGetNodes(pl->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (!rc && e == cudaSuccess) e = cudaGraphGetNodes(pl->graph, nodes.data(), &nn);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "graph nodes");
        for (size_t i = 0; !rc && i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            if (cudaGraphKernelNodeGetParams(nodes[i], &kp) != cudaSuccess) continue;
            if (kp.func == k.func) {
                pl->stepper_node = nodes[i];
                pl->knp = kp;
                std::memcpy(&pl->sp, kp.kernelParams[0], sizeof(StepperParams));
            }
        }
        if (!rc && !pl->stepper_node) rc = fail(FPT_ECUDA, "stepper node not found in the captured graph");
    }
    if (rc) {
        plan_free(pl);
        return rc;
    }
    pl->args[0] = &pl->sp;
    pl->knp.kernelParams = pl->args;
    pl->knp.extra = nullptr;
    *plan_out = pl;
    return FPT_OK;
}

extern "C" int fpt_plan_launch(fpt_plan* pl, uint64_t seed, void* stream) {
    NvtxRange nvtx_range("fpt_plan_launch");
    if (!pl) return fail(FPT_EINVAL, "plan is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != pl->device) return fail(FPT_EINVAL, "plan belongs to device %d, current is %d", pl->device, dev);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    pl->sp.keys = philox_keys(seed);
    cudaError_t e = cudaGraphExecKernelNodeSetParams(pl->exec, pl->stepper_node, &pl->knp);
    if (e != cudaSuccess) return cuda_fail(e, "set stepper seed");
    e = cudaGraphLaunch(pl->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (pl->host_status->status != 0u)
        return fail(FPT_EDEVICE_STATUS, "device status 0x%x", pl->host_status->status);
    return FPT_OK;
}

extern "C" int fpt_plan_destroy(fpt_plan* pl) {
    plan_free(pl);
    return FPT_OK;
}
