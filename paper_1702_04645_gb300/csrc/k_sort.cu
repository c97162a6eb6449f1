// k_sort.cu -- stable LSD radix sort and AGGREGATE (Section 3.5).
//
// AGGREGATE turns every community into a super node: W'_AB is the sum of W_uv
// over u in A and v in B (the diagonal keeps the internal weight), so the
// strengths and m_w are preserved.  Each stored entry (u, v, w) becomes the
// key id[u] * K + id[v]; the keys are sorted by a radix sort (8-bit digits,
// per-tile histograms, stable scatter ranked by warp match) and equal keys are
// reduced by segment into the new CSR, whose columns come out sorted.
#include "slm_internal.cuh"

namespace slm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const K *keys, long long n, int shift, int32_t *hist, int ntiles) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; r++) {
        long long i = base + (long long)r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 255)], 1);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K *kin, const int32_t *vin, K *kout, int32_t *vout, long long n,
                             int shift, const int32_t *offs, int ntiles) {
    __shared__ int base[256];
    __shared__ int run[256];
    __shared__ int wcnt[kRsWarps][257];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    base[tid] = offs[(long long)tid * ntiles + blockIdx.x];
    run[tid] = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long t0 = (long long)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; r++) {
        long long i = t0 + (long long)r * kRsThreads + tid;
        bool valid = i < n;
        K key = valid ? kin[i] : K(0);
        int val = valid ? vin[i] : 0;
        int d = valid ? (int)((key >> shift) & 255) : 256;
        for (int k = tid; k < kRsWarps * 257; k += kRsThreads) (&wcnt[0][0])[k] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(FULL, d);
        int rk = __popc(peers & lt_mask);
        if (valid && rk == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        {
            int acc = run[tid];
            for (int w = 0; w < kRsWarps; w++) {
                int c = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += c;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            int pos = base[d] + wcnt[wid][d] + rk;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

template <class K>
void radix_sort_impl(K *keys, int32_t *vals, K *ktmp, int32_t *vtmp, long long n, int bits,
                     cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
    DevBuf hist(sizeof(int32_t) * 256 * (size_t)ntiles, s);
    K *ka = keys, *kb = ktmp;
    int32_t *va = vals, *vb = vtmp;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, passes++) {
        k_rs_hist<K><<<ntiles, kRsThreads, 0, s>>>(ka, n, shift, hist.as<int32_t>(), ntiles);
        SLM_LAUNCH_CHECK();
        exclusive_scan_i32(hist.as<int32_t>(), hist.as<int32_t>(), 256LL * ntiles, nullptr, s);
        k_rs_scatter<K><<<ntiles, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist.as<int32_t>(), ntiles);
        SLM_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (passes & 1) {
        SLM_CUDA(cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
        SLM_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
}

// ---------------------------------------------------------------------------
// Aggregation
// ---------------------------------------------------------------------------
// rows of nodes whose graph is marked in drop_graph (a forest) get the key
// K*K, one past every real key, so that they sort last and are cut off
__global__ void k_agg_keys(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                           const int32_t *id, long long K, unsigned long long *keys,
                           int32_t *vals, const int32_t *gid, const int32_t *drop_graph) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = warp; u < n; u += nwarps) {
        const bool drop = drop_graph && drop_graph[gid[u]];
        unsigned long long hi = (unsigned long long)id[u] * (unsigned long long)K;
        for (int p = rp[u] + lane; p < rp[u + 1]; p += 32) {
            keys[p] = drop ? (unsigned long long)K * (unsigned long long)K
                           : hi + (unsigned long long)id[col[p]];
            vals[p] = w[p];
        }
    }
}

__global__ void k_agg_heads(long long nnz, const unsigned long long *keys, int32_t *head) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (long long)gridDim.x * blockDim.x)
        head[p] = (p == 0 || keys[p] != keys[p - 1]) ? 1 : 0;
}

// seg[p] = exclusive scan of heads; a warp-level segmented sum issues one
// atomic per segment piece.
__global__ void k_agg_reduce(long long nnz, const unsigned long long *keys, const int32_t *vals,
                             const int32_t *seg, long long K, int32_t *w_out, int32_t *col_out,
                             int32_t *rowcnt) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nnz; base += stride) {
        long long p = base + threadIdx.x;
        bool valid = p < nnz;
        int sg = valid ? seg[p] + ((p == 0 || keys[p] != keys[p - 1]) ? 1 : 0) - 1 : -1;
        // seg[] is the exclusive scan of heads, so segment id = seg + head - 1
        int v = valid ? vals[p] : 0;
        // inclusive segmented scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int ov = __shfl_up_sync(FULL, v, o);
            int os = __shfl_up_sync(FULL, sg, o);
            if (lane >= o && os == sg) v += ov;
        }
        int nsg = __shfl_down_sync(FULL, sg, 1);
        bool last = (lane == 31) || (nsg != sg);
        if (valid && last) atomicAdd(&w_out[sg], v);
        if (valid && (p == 0 || keys[p] != keys[p - 1])) {
            unsigned long long k = keys[p];
            col_out[sg] = (int32_t)(k % (unsigned long long)K);
            atomicAdd(&rowcnt[(int)(k / (unsigned long long)K)], 1);
        }
    }
}

}  // namespace

void radix_sort_u64(unsigned long long *keys, int32_t *vals, unsigned long long *keys_tmp,
                    int32_t *vals_tmp, long long n, int bits, cudaStream_t s) {
    radix_sort_impl<unsigned long long>(keys, vals, keys_tmp, vals_tmp, n, bits, s);
}
void radix_sort_u32(uint32_t *keys, int32_t *vals, uint32_t *keys_tmp, int32_t *vals_tmp,
                    long long n, int bits, cudaStream_t s) {
    radix_sort_impl<uint32_t>(keys, vals, keys_tmp, vals_tmp, n, bits, s);
}

int32_t aggregate_graph(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                        const int32_t *id, int32_t K, DevBuf &rp_out, DevBuf &col_out,
                        DevBuf &w_out, cudaStream_t st, const int32_t *gid,
                        const int32_t *drop_graph, long long dropped) {
    int32_t nnz_all = 0;
    SLM_CUDA(cudaMemcpyAsync(&nnz_all, rp + n, sizeof nnz_all, cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    const int32_t nnz = nnz_all - (int32_t)dropped;  // entries kept after the sort
    rp_out.alloc(sizeof(int32_t) * ((size_t)K + 1), st);
    SLM_CUDA(cudaMemsetAsync(rp_out.get(), 0, sizeof(int32_t) * ((size_t)K + 1), st));
    if (nnz == 0 || K == 0) {
        col_out.alloc(16, st);
        w_out.alloc(16, st);
        return 0;
    }
    DevBuf keys(8 * (size_t)nnz_all, st), ktmp(8 * (size_t)nnz_all, st), vals(4 * (size_t)nnz_all, st),
        vtmp(4 * (size_t)nnz_all, st), seg(4 * (size_t)nnz, st), tot(8, st);
    k_agg_keys<<<grid_for((long long)n * 32, 256, kNumSMs * 16), 256, 0, st>>>(
        n, rp, col, w, id, K, keys.as<unsigned long long>(), vals.as<int32_t>(), gid, drop_graph);
    SLM_LAUNCH_CHECK();
    unsigned long long maxkey = (unsigned long long)K * (unsigned long long)K + (dropped > 0 ? 1 : 0);
    int bits = 0;
    while (bits < 64 && (1ull << bits) < maxkey) bits++;
    radix_sort_u64(keys.as<unsigned long long>(), vals.as<int32_t>(), ktmp.as<unsigned long long>(),
                   vtmp.as<int32_t>(), nnz_all, bits, st);
    k_agg_heads<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, keys.as<unsigned long long>(), seg.as<int32_t>());
    SLM_LAUNCH_CHECK();
    exclusive_scan_i32(seg.as<int32_t>(), seg.as<int32_t>(), nnz, tot.as<int32_t>(), st);
    int32_t nnz2 = 0;
    SLM_CUDA(cudaMemcpyAsync(&nnz2, tot.get(), sizeof nnz2, cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    col_out.alloc(4 * (size_t)nnz2, st);
    w_out.alloc(4 * (size_t)nnz2, st);
    SLM_CUDA(cudaMemsetAsync(w_out.get(), 0, 4 * (size_t)nnz2, st));
    k_agg_reduce<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, keys.as<unsigned long long>(),
                                                     vals.as<int32_t>(), seg.as<int32_t>(), K,
                                                     w_out.as<int32_t>(), col_out.as<int32_t>(),
                                                     rp_out.as<int32_t>());
    SLM_LAUNCH_CHECK();
    exclusive_scan_i32(rp_out.as<int32_t>(), rp_out.as<int32_t>(), (long long)K + 1, nullptr, st);
    return nnz2;
}

}  // namespace slm
