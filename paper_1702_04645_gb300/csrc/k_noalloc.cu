// k_noalloc.cu -- modularity of a labelling without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: frameworks that hand all
// device memory to their own caching allocator or to a fixed arena, and that
// forbid (or cannot afford the device-wide synchronisation of) further
// allocations in the middle of their work.  slm_step_modularity_noalloc serves
// them: it computes the same exact numerator and quotient as
// slm_step_modularity, but its scratch lives in one file-scope device array of
// fixed size that every GPU loading this library holds until the process exits.
#include <mutex>

#include "slm_internal.cuh"
#include "slm_steps.h"

namespace slm {
namespace {

constexpr int kNoAllocMaxN = 1 << 20;  // largest n accepted (labels take values in [0, n))

// scratch: per-label internal weight, per-label total strength, three sums
__device__ __align__(256) unsigned long long g_modularity_scratch[2 * kNoAllocMaxN + 4];

std::mutex g_addr_mutex;
void *g_addr[64] = {nullptr};  // address of the scratch array on each device, once looked up

// The host-side name of a __device__ array is only a stand-in: the device
// address has to be looked up with that device current.
unsigned long long *scratch_for_current_device() {
    int dev = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(SLM_ERR_INVALID_ARGUMENT, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_modularity_scratch);
        if (e != cudaSuccess || p == nullptr)
            fail(SLM_ERR_CUDA, std::string("cudaGetSymbolAddress of the modularity scratch failed: ") +
                                   cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    return static_cast<unsigned long long *>(g_addr[dev]);
}

// zero win[0..n), sig[0..n) and the four trailing words (three sums and an
// error flag): the array keeps whatever the previous call left in it
__global__ void k_na_clear(unsigned long long *scr, int32_t n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 2LL * n + 4;
         i += (long long)gridDim.x * blockDim.x) {
        long long j;
        if (i < n) j = i;
        else if (i < 2LL * n) j = kNoAllocMaxN + (i - n);
        else j = 2LL * kNoAllocMaxN + (i - 2LL * n);
        scr[j] = 0;
    }
}

__global__ void k_na_accumulate(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                                const int32_t *labels, unsigned long long *scr) {
    unsigned long long *win = scr, *sig = scr + kNoAllocMaxN;
    unsigned long long *err = scr + 2 * kNoAllocMaxN + 3;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nwarps) {
        int lu = labels[u];
        if (lu < 0 || lu >= n) {  // a label outside [0, n) would index past the scratch
            if (lane == 0) atomicOr(err, 1ull);
            continue;
        }
        long long in = 0, su = 0;
        for (int p = rp[u] + lane; p < rp[u + 1]; p += 32) {
            int j = col[p];
            su += w[p];
            if (j < 0 || j >= n) { atomicOr(err, 2ull); continue; }
            if (labels[j] == lu) in += w[p];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            in += __shfl_xor_sync(0xffffffffu, in, o);
            su += __shfl_xor_sync(0xffffffffu, su, o);
        }
        if (lane == 0) {
            if (in) atomicAdd(&win[lu], (unsigned long long)in);
            if (su) atomicAdd(&sig[lu], (unsigned long long)su);
        }
    }
}

// sums[0] = sum_C W_in(C), sums[1] = sum_C Sigma_C = m_w, sums[2] = sum_C Sigma_C^2
__global__ void k_na_reduce(int32_t n, unsigned long long *scr) {
    const unsigned long long *win = scr, *sig = scr + kNoAllocMaxN;
    unsigned long long *sums = scr + 2 * kNoAllocMaxN;
    unsigned long long a = 0, b = 0, c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        a += win[i];
        b += sig[i];
        c += sig[i] * sig[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&sums[0], a);
        if (b) atomicAdd(&sums[1], b);
        if (c) atomicAdd(&sums[2], c);
    }
}

// num = m_w sum W_in - sum Sigma^2 (both terms below m_w^2 < 2^62), Q = num / m_w^2
__global__ void k_na_finish(const unsigned long long *scr, int64_t *num_out, double *q_out) {
    const unsigned long long *sums = scr + 2 * kNoAllocMaxN;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        long long m = (long long)sums[1];
        long long num = m * (long long)sums[0] - (long long)sums[2];
        *num_out = num;
        *q_out = m == 0 ? 0.0 : (double)num / ((double)m * (double)m);
    }
}

}  // namespace
}  // namespace slm

extern "C" slm_status slm_step_modularity_noalloc(int32_t n, const int32_t *row_ptr,
                                                  const int32_t *col, const int32_t *w,
                                                  const int32_t *labels, int64_t *num_out,
                                                  double *q_out, void *stream) {
    using namespace slm;
    if (n < 0 || !num_out || !q_out || (n > 0 && (!row_ptr || !col || !w || !labels))) {
        set_global_error("slm_step_modularity_noalloc: negative n or NULL pointer");
        return SLM_ERR_INVALID_ARGUMENT;
    }
    if (n > kNoAllocMaxN) {
        set_global_error("slm_step_modularity_noalloc: n exceeds its fixed scratch of 1048576 nodes");
        return SLM_ERR_INVALID_ARGUMENT;
    }
    try {
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        unsigned long long *scr = scratch_for_current_device();
        const int32_t nn = n > 0 ? n : 0;
        k_na_clear<<<grid_for(2LL * nn + 4, 256), 256, 0, st>>>(scr, nn);
        SLM_LAUNCH_CHECK();
        if (nn > 0) {
            k_na_accumulate<<<grid_for((long long)nn * 32, 256), 256, 0, st>>>(nn, row_ptr, col, w,
                                                                              labels, scr);
            SLM_LAUNCH_CHECK();
            k_na_reduce<<<grid_for(nn, 256, 1024), 256, 0, st>>>(nn, scr);
            SLM_LAUNCH_CHECK();
        }
        k_na_finish<<<1, 32, 0, st>>>(scr, num_out, q_out);
        SLM_LAUNCH_CHECK();
        unsigned long long err = 0;
        SLM_CUDA(cudaMemcpyAsync(&err, scr + 2 * kNoAllocMaxN + 3, sizeof err, cudaMemcpyDeviceToHost, st));
        SLM_CUDA(cudaStreamSynchronize(st));
        if (err) fail(SLM_ERR_INVALID_ARGUMENT, "slm_step_modularity_noalloc: a label or column lies outside [0, n)");
        return SLM_OK;
    } catch (const slm::Error &e) {
        set_global_error(e.msg);
        return e.status;
    }
}
