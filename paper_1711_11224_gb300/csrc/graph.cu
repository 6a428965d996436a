// CUDA graph of a whole projected-gradient run: prologue -> WHILE(trial slot) -> epilogue.
//
// The trial slot's last kernel evaluates the step rule on the device and sets
// the loop condition (continue while the run is not done), so the graph runs
// exactly the trials the run needs, with no spare slots.  The prologue is
// captured into the graph, the conditional node is appended after its tail,
// its body graph is filled by a second capture, and the epilogue is captured
// after the conditional node.
#include <stdio.h>

#include <vector>

#include "cdv_internal.h"

namespace cdv {

cdv_status build_loop_graph(cudaStream_t cap, PhaseFn phase, void* ctx, cudaGraph_t* out)
{
    *out = nullptr;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaGraph_t g = nullptr;
    cudaError_t e0 = cudaGraphCreate(&g, 0);
    if (e0 != cudaSuccess) {
        set_last_error(cudaGetErrorString(e0));
        return CDV_ERR_CUDA;
    }
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    cdv_status st = CDV_OK;
    std::vector<cudaGraphNode_t> tail;
    cudaGraphNode_t cn = nullptr;
    cudaGraph_t tmp = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, mode);
    if (e == cudaSuccess) {
        st = phase(ctx, 0, true, (unsigned long long)h, cap);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(cap, &cs, nullptr, nullptr, &deps, nullptr, &nd);
        if (e == cudaSuccess && deps) tail.assign(deps, deps + nd);
        const cudaError_t e2 = cudaStreamEndCapture(cap, &tmp);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && st == CDV_OK) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&cn, g, tail.data(), nullptr, tail.size(), &cp);
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, mode);
            if (e == cudaSuccess) {
                st = phase(ctx, 1, true, (unsigned long long)h, cap);
                const cudaError_t e2 = cudaStreamEndCapture(cap, &tmp);
                if (e == cudaSuccess) e = e2;
            }
        }
    }
    if (e == cudaSuccess && st == CDV_OK) {
        e = cudaStreamBeginCaptureToGraph(cap, g, &cn, nullptr, 1, mode);
        if (e == cudaSuccess) {
            st = phase(ctx, 2, true, (unsigned long long)h, cap);
            const cudaError_t e2 = cudaStreamEndCapture(cap, &tmp);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e != cudaSuccess || st != CDV_OK) {
        cudaGraphDestroy(g);
        if (st != CDV_OK) return st;
        char buf[256];
        snprintf(buf, sizeof buf, "building the iteration graph: %s", cudaGetErrorString(e));
        set_last_error(buf);
        return CDV_ERR_CUDA;
    }
    *out = g;
    return CDV_OK;
}

}  // namespace cdv
