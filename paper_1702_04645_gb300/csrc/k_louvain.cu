// k_louvain.cu -- colour-synchronous Louvain on the scan kernels: the
// parallel form of classical Louvain that Section 6 leaves for later work,
// built for comparison with the Synchronised Louvain Method.
//
// The nodes of one colour class of a distance-1 colouring share no edge, so
// their classical moves (leave the own community, join the neighbouring one
// of largest positive gain, ties to the smallest name) can be decided
// together: every class is one MAXIMAL scan over its nodes (the gain that
// scan computes is exactly Louvain's), followed by one write of the class's
// moves and of the totals they change.
//
// Colouring: node v at level t has the key mix64(seed ^ mix64((t << 32) | v));
// u precedes v when its key is larger, or the keys are equal and u < v.  The
// result is the first-fit colouring in that order (each node takes the
// smallest colour no preceding neighbour holds), computed in Jones-Plassmann
// rounds: an uncoloured node whose uncoloured neighbours all come after it is
// coloured in the current round.  Its neighbours that precede it were all
// coloured in earlier rounds, and no neighbour that follows it is coloured
// before it, so each node sees exactly the neighbours the sequential order
// would show it.
#include "slm_internal.cuh"

namespace slm {
namespace {

__device__ __forceinline__ unsigned long long colour_key(unsigned long long seed, int t, int v) {
    return mix64(seed ^ mix64(((unsigned long long)(unsigned)t << 32) | (unsigned long long)(unsigned)v));
}

// cr[v] = -1 while v is uncoloured, then (round << 32) | colour.  A neighbour
// coloured in the current round counts as uncoloured, so a decision never
// depends on the order in which the round's writes land (64-bit stores are
// seen whole).  One warp per node.
__global__ void k_colour_round(int32_t n, const int32_t *rp, const int32_t *col,
                               unsigned long long seed, int t, int round, long long *cr,
                               int32_t *left) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int blocked_nodes = 0;
    for (long long v = warp; v < n; v += nw) {
        if (cr[v] >= 0) continue;  // uniform over the warp
        const unsigned long long kv = colour_key(seed, t, (int)v);
        const int b = rp[v], e = rp[v + 1];
        bool blocked = false;
        for (int p = b + lane; p < e && !blocked; p += 32) {
            const int u = col[p];
            if (u == v) continue;
            const long long c = cr[u];
            const bool unc = c < 0 || (int)(c >> 32) == round;
            if (unc) {
                const unsigned long long ku = colour_key(seed, t, u);
                blocked = ku > kv || (ku == kv && u < (int)v);
            }
        }
        if (__any_sync(0xffffffffu, blocked)) {
            blocked_nodes++;
            continue;
        }
        // the smallest colour held by no neighbour coloured before this round,
        // 64 colours per look at the row
        int colour = 0;
        for (int base = 0;; base += 64) {
            unsigned long long mask = 0;
            for (int p = b + lane; p < e; p += 32) {
                const int u = col[p];
                if (u == v) continue;
                const long long c = cr[u];
                if (c >= 0 && (int)(c >> 32) != round) {
                    const int cu = (int)(c & 0xffffffffll);
                    if (cu >= base && cu < base + 64) mask |= 1ull << (cu - base);
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
            if (mask != ~0ull) {
                colour = base + __ffsll((long long)~mask) - 1;
                break;
            }
        }
        if (lane == 0) cr[v] = ((long long)round << 32) | (long long)colour;
    }
    if (lane == 0 && blocked_nodes) atomicAdd(left, blocked_nodes);
}

__global__ void k_colour_take(int32_t n, const long long *cr, int32_t *colour, uint32_t *key,
                              int32_t *node, int32_t *ncol) {
    int mx = -1;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(cr[v] & 0xffffffffll);
        colour[v] = c;
        key[v] = (uint32_t)c;
        node[v] = (int32_t)v;
        mx = max(mx, c);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx >= 0) atomicMax(ncol, mx + 1);
}

__global__ void k_colour_count(int32_t n, const int32_t *colour, int32_t *cnt) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[colour[v]], 1);
}

// The moves of one colour class: best[i] differs from comm[i] exactly when
// the scan found a positive gain.
__global__ void k_louvain_move(const int32_t *list, int32_t cnt, const int32_t *best,
                               int32_t *comm, const int32_t *s, int32_t *sigma,
                               unsigned long long *moves) {
    unsigned mv = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < cnt;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = list[k];
        const int to = best[i], from = comm[i];
        if (to != from) {
            atomicSub(&sigma[from], s[i]);
            atomicAdd(&sigma[to], s[i]);
            comm[i] = to;
            mv++;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mv += __shfl_xor_sync(0xffffffffu, mv, o);
    if ((threadIdx.x & 31) == 0 && mv) atomicAdd(moves, (unsigned long long)mv);
}

__global__ void k_louvain_init(int32_t n, const int32_t *s, int32_t *comm, int32_t *sigma) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        comm[v] = (int32_t)v;
        sigma[v] = s[v];
    }
}

__global__ void k_name_used(int32_t n, const int32_t *comm, int32_t *used) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        used[comm[v]] = 1;
}

__global__ void k_name_rank(int32_t n, const int32_t *comm, const int32_t *rank, int32_t *id) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        id[v] = rank[comm[v]];
}

}  // namespace

std::vector<int32_t> colour_nodes(int32_t n, const int32_t *rp, const int32_t *col,
                                  unsigned long long seed, int32_t level, int32_t *colour,
                                  int32_t *order, cudaStream_t st) {
    std::vector<int32_t> class_off(1, 0);
    if (n <= 0) return class_off;
    DevBuf cr(8 * (size_t)n, st), left(16, st), key(4 * (size_t)n, st), ktmp(4 * (size_t)n, st),
        vtmp(4 * (size_t)n, st);
    SLM_CUDA(cudaMemsetAsync(cr.get(), 0xff, 8 * (size_t)n, st));
    int32_t *lp = left.as<int32_t>();
    const int grid = grid_for((long long)n * 32, 256, kNumSMs * 16);
    // every round colours at least the first uncoloured node of the order
    for (int round = 0;; round++) {
        if (round > n) fail(SLM_ERR_CUDA, "colouring did not finish");
        SLM_CUDA(cudaMemsetAsync(lp, 0, 8, st));
        k_colour_round<<<grid, 256, 0, st>>>(n, rp, col, seed, level, round, cr.as<long long>(), lp);
        SLM_LAUNCH_CHECK();
        int32_t h = 0;
        SLM_CUDA(cudaMemcpyAsync(&h, lp, sizeof h, cudaMemcpyDeviceToHost, st));
        stream_sync(st);
        if (h == 0) break;
    }
    k_colour_take<<<grid_for(n, 256), 256, 0, st>>>(n, cr.as<long long>(), colour, key.as<uint32_t>(),
                                                    order, lp + 1);
    SLM_LAUNCH_CHECK();
    int32_t ncol = 0;
    SLM_CUDA(cudaMemcpyAsync(&ncol, lp + 1, sizeof ncol, cudaMemcpyDeviceToHost, st));
    stream_sync(st);
    int bits = 1;
    while ((1LL << bits) < ncol) bits++;
    radix_sort_u32(key.as<uint32_t>(), order, ktmp.as<uint32_t>(), vtmp.as<int32_t>(), n, bits, st);
    DevBuf cnt(4 * (size_t)(ncol + 1), st);
    SLM_CUDA(cudaMemsetAsync(cnt.get(), 0, 4 * (size_t)(ncol + 1), st));
    k_colour_count<<<grid_for(n, 256), 256, 0, st>>>(n, colour, cnt.as<int32_t>());
    SLM_LAUNCH_CHECK();
    std::vector<int32_t> h(ncol);
    SLM_CUDA(cudaMemcpyAsync(h.data(), cnt.get(), 4 * (size_t)ncol, cudaMemcpyDeviceToHost, st));
    stream_sync(st);
    for (int k = 0; k < ncol; k++) class_off.push_back(class_off.back() + h[k]);
    return class_off;
}

void louvain_init(int32_t n, const int32_t *s, int32_t *comm, int32_t *sigma, cudaStream_t st) {
    if (n <= 0) return;
    k_louvain_init<<<grid_for(n, 256), 256, 0, st>>>(n, s, comm, sigma);
    SLM_LAUNCH_CHECK();
}

void louvain_move(const int32_t *list, int32_t cnt, const int32_t *best, int32_t *comm,
                  const int32_t *s, int32_t *sigma, unsigned long long *moves, cudaStream_t st) {
    if (cnt <= 0) return;
    k_louvain_move<<<grid_for(cnt, 256), 256, 0, st>>>(list, cnt, best, comm, s, sigma, moves);
    SLM_LAUNCH_CHECK();
}

int32_t compact_names(int32_t n, const int32_t *comm, int32_t *id, int32_t *scratch_n,
                      cudaStream_t st) {
    if (n <= 0) return 0;
    DevBuf tot(sizeof(int32_t), st);
    SLM_CUDA(cudaMemsetAsync(scratch_n, 0, 4 * (size_t)n, st));
    k_name_used<<<grid_for(n, 256), 256, 0, st>>>(n, comm, scratch_n);
    SLM_LAUNCH_CHECK();
    exclusive_scan_i32(scratch_n, scratch_n, n, tot.as<int32_t>(), st);
    k_name_rank<<<grid_for(n, 256), 256, 0, st>>>(n, comm, scratch_n, id);
    SLM_LAUNCH_CHECK();
    int32_t K = 0;
    SLM_CUDA(cudaMemcpyAsync(&K, tot.get(), sizeof K, cudaMemcpyDeviceToHost, st));
    stream_sync(st);
    return K;
}

}  // namespace slm
