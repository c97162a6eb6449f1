// forest_dev.cuh -- device helpers shared by the assignment-graph kernels.
#pragma once

#include "slm_internal.cuh"

namespace slm {

__device__ __forceinline__ void add64(long long *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

#define SLM_GRID_STRIDE(v, n)                                                      \
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < (n); \
         v += (long long)gridDim.x * blockDim.x)

// Lowest common ancestor of two nodes with the same entry: walk up by depth.
// Every loop is bounded by the depths, so it ends even on inconsistent input.
__device__ __forceinline__ int lca_walk(int x, int y, const int32_t *a, const int32_t *depth) {
    int dx = depth[x], dy = depth[y];
    while (dx > dy) { x = a[x]; dx--; }
    while (dy > dx) { y = a[y]; dy--; }
    while (dx > 0 && x != y) { x = a[x]; y = a[y]; dx--; }
    return x;
}

}  // namespace slm
