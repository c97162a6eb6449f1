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

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

namespace {

// Grid barrier with a time limit (the kernel is launched cooperatively, so
// every block is resident).  One word serves every barrier of a launch:
// block 0 adds 2^31 - (blocks - 1) and every other block adds 1, so the top
// bit flips exactly when the last block arrives and the low bits return to
// their value before the barrier.  Thread 0 of each block waits for the flip
// for at most `limit_ns` of global time, then sets the failure word.  Returns
// false once any block has failed: the caller leaves the kernel, and every
// other block does the same at its next barrier, which is bounded the same
// way, so the launch always ends.  A grid of one block needs the block
// barrier only.
struct GridBarrier {
    unsigned word;
    int failed;
};
// longest a block waits at a grid barrier before the launch is abandoned
constexpr long long kBarrierLimitNs = 4000000000LL;

// The arrival is one acq_rel atomic at GPU scope and the wait reads the word
// with acquire loads: the block barrier before the arrival orders every
// thread's writes before thread 0's release, and the block barrier after the
// wait orders thread 0's acquire before every thread's reads, so the writes
// of every block before the barrier are visible to every block after it
// (release and acquire are cumulative), without a full fence on either side.
__device__ __forceinline__ unsigned gbar_arrive(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned gbar_load(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __noinline__ bool gbar(GridBarrier *b, long long limit_ns) {
    __syncthreads();
    if (gridDim.x > 1) {
        if (threadIdx.x == 0) {
            const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
            const unsigned old = gbar_arrive(&b->word, add);
            long long t0 = 0;
            for (unsigned spin = 0; ((old ^ gbar_load(&b->word)) & 0x80000000u) == 0; spin++) {
                if ((spin & 255u) == 0) {  // read the clock now and then
                    const long long t = global_ns();
                    if (t0 == 0) t0 = t;
                    else if (t - t0 > limit_ns) {
                        atomicExch(&b->failed, 1);
                        break;
                    }
                }
            }
        }
        __syncthreads();
    }
    return *((volatile int *)&b->failed) == 0;
}

}  // namespace

}  // namespace slm
