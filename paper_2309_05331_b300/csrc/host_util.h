// host_util.h -- host helpers shared by the library's translation units:
// error text of context-free entry points, and creation of the CUDA graph
// skeleton WHILE(cond) { body } that drives every step loop.
#pragma once
#include <cuda_runtime.h>

#include <cstring>

void set_global_error(cudaError_t e, const char* where);

// Creates graph *g holding one conditional WHILE node (default condition 1,
// reset at every launch) and returns its handle and its empty body graph.
inline cudaError_t make_while_graph(cudaGraph_t* g, cudaGraphConditionalHandle* h, cudaGraph_t* body) {
    *g = nullptr;
    cudaError_t e = cudaGraphCreate(g, 0);
    if (e != cudaSuccess) return e;
    e = cudaGraphConditionalHandleCreate(h, *g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = *h;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, *g, nullptr, nullptr, 0, np);
    if (e != cudaSuccess) return e;
    *body = np->conditional.phGraph_out[0];
    return cudaSuccess;
}
