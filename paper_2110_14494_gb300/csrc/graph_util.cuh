// Helpers for recording device-driven loops into CUDA graphs (conditional
// nodes added at the capture point of a stream).
#pragma once
#include <cuda_runtime.h>

namespace pic {

// Adds a conditional node with handle h at the capture point of stream cs
// (which must be capturing) and makes it the stream's only dependency;
// bodies receives its body graphs (owned by the node).
inline cudaError_t add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                   unsigned size, cudaGraph_t* bodies) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, &ed, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, ed, nd, &p);
    if (e != cudaSuccess) return e;
    for (unsigned q = 0; q < size; ++q) bodies[q] = p.conditional.phGraph_out[q];
    return cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Ends a capture into a body graph (the graph stays owned by its node).
inline cudaError_t end_body_capture(cudaStream_t s) {
    cudaGraph_t g = nullptr;
    return cudaStreamEndCapture(s, &g);
}

// The graph a capturing stream records into (null if it is not capturing).
inline cudaGraph_t capturing_graph(cudaStream_t cs) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    if (cudaStreamGetCaptureInfo(cs, &st, nullptr, &g) != cudaSuccess || st != cudaStreamCaptureStatusActive)
        return nullptr;
    return g;
}

}  // namespace pic
