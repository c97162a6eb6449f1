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
#include <algorithm>
#include <climits>
#include <mutex>

#include "forest_dev.cuh"

namespace slm {
namespace {

__device__ __forceinline__ unsigned long long colour_key(unsigned long long seed, int t, int v) {
    return mix64(seed ^ mix64(((unsigned long long)(unsigned)t << 32) | (unsigned long long)(unsigned)v));
}

// cr[v] = -1 while v is uncoloured, then (round << 32) | colour.  A neighbour
// coloured in the current round counts as uncoloured, so a decision never
// depends on the order in which the round's writes land (64-bit stores are
// seen whole).  One warp per node; returns (to every lane) whether v stays
// uncoloured because an uncoloured neighbour comes first.
// bits per warp of the colour bitmaps: a node's first-fit colour is at most
// its row length, so rows shorter than this take the bitmap
constexpr int kColourBits = 8192;

// resume[v] (zeroed before the first round) is the offset in v's row of the
// first entry that may still hold a neighbour blocking v: the entries before
// it were found coloured in an earlier round or ordered after v, and neither
// ever changes, so each node's rows are checked O(row length) times in all.
// cmax holds the largest colour given so far.
__device__ __forceinline__ bool colour_node(long long v, const int32_t *rp, const int32_t *col,
                                            unsigned long long seed, int t, int round, long long *cr,
                                            unsigned *bm, int32_t *resume, int32_t *cmax) {
    const int lane = threadIdx.x & 31;
    const unsigned long long kv = colour_key(seed, t, (int)v);
    const int b = rp[v], e = rp[v + 1];
    // the whole warp stops at the first 32 entries that hold an uncoloured
    // neighbour coming first (on a dense row that is usually the first look)
    for (int p0 = b + resume[v]; p0 < e; p0 += 32) {
        const int p = p0 + lane;
        bool blocked = false;
        if (p < e) {
            const int u = col[p];
            const long long c = u != v ? cr[u] : 0;
            if (u != v && (c < 0 || (int)(c >> 32) == round)) {
                const unsigned long long ku = colour_key(seed, t, u);
                blocked = ku > kv || (ku == kv && u < (int)v);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, blocked);
        if (bal) {
            if (lane == 0) resume[v] = p0 - b + __ffs((int)bal) - 1;
            return true;
        }
    }
    int colour = 0;
    // The bitmap holds colours below kColourBits.  It decides exactly when
    // the row is shorter (a first-fit colour is at most the row length) or
    // when every colour given in earlier rounds is below kColourBits - 1 (the
    // neighbours then show at most kColourBits - 1 distinct colours, all in
    // the bitmap, so its first clear bit is the answer).
    const int words = e - b < kColourBits ? (e - b) / 32 + 1 : kColourBits / 32;
    if (e - b < kColourBits || *((volatile int32_t *)cmax) < kColourBits - 1) {
        // one look at the row: the colours of the neighbours coloured before
        // this round as bits of the warp's bitmap, then its first clear bit
        for (int q = lane; q < words; q += 32) bm[q] = 0u;
        __syncwarp();
        for (int p0 = b + lane; p0 < e; p0 += 128) {
            int u[4];
#pragma unroll
            for (int k = 0; k < 4; k++) u[k] = p0 + 32 * k < e ? col[p0 + 32 * k] : (int)v;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (u[k] == v) continue;
                const long long c = cr[u[k]];
                if (c >= 0 && (int)(c >> 32) != round) {
                    const int cu = (int)(c & 0xffffffffll);
                    if (cu < 32 * words) atomicOr(&bm[cu >> 5], 1u << (cu & 31));
                }
            }
        }
        __syncwarp();
        int first = INT_MAX;
        for (int q = lane; q < words && first == INT_MAX; q += 32)
            if (bm[q] != 0xffffffffu) first = 32 * q + __ffs((int)~bm[q]) - 1;
#pragma unroll
        for (int o = 16; o; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        __syncwarp();  // the bitmap is reused by the warp's next node
        if (lane == 0) {
            cr[v] = ((long long)round << 32) | (long long)first;
            atomicMax(cmax, first);
        }
        return false;
    }
    // a long row: 64 colours per look at the row, four entries per lane in flight
    for (int base = 0;; base += 64) {
        unsigned long long mask = 0;
        for (int p0 = b + lane; p0 < e; p0 += 128) {
            int u[4];
#pragma unroll
            for (int k = 0; k < 4; k++) u[k] = p0 + 32 * k < e ? col[p0 + 32 * k] : (int)v;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (u[k] == v) continue;
                const long long c = cr[u[k]];
                if (c >= 0 && (int)(c >> 32) != round) {
                    const int cu = (int)(c & 0xffffffffll);
                    if (cu >= base && cu < base + 64) mask |= 1ull << (cu - base);
                }
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
        if (mask != ~0ull) {
            colour = base + __ffsll((long long)~mask) - 1;
            break;
        }
    }
    if (lane == 0) {
        cr[v] = ((long long)round << 32) | (long long)colour;
        atomicMax(cmax, colour);
    }
    return false;
}

// Every round of the colouring in one cooperative launch (the rows of a dense
// aggregated graph can need one round per node): rounds are separated by grid
// barriers with a time limit, and a round visits only the nodes still
// uncoloured.  Round r reads its list from wl[r & 1] (lcnt[r % 3] entries)
// and appends the nodes it leaves uncoloured to wl[(r + 1) & 1], counting
// them in lcnt[(r + 1) % 3]; lcnt[(r + 2) % 3], last read in round r - 1, is
// cleared during round r.  Ends when a round leaves no node; *rounds_out gets
// the number of rounds (at most n + 1).
__global__ void __launch_bounds__(256) k_colour_rounds(int32_t n, const int32_t *rp, const int32_t *col,
                                                       unsigned long long seed, int t, long long *cr,
                                                       int32_t *wl0, int32_t *wl1, int32_t *resume,
                                                       GridBarrier *bar, int32_t *lcnt, long long limit_ns,
                                                       int32_t *rounds_out) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const bool rank0 = blockIdx.x == 0 && threadIdx.x == 0;
    __shared__ unsigned bitmaps[256 / 32][kColourBits / 32];
    __shared__ int keep[256 / 32][32];
    unsigned *bm = bitmaps[threadIdx.x >> 5];
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
    {
        wl0[v] = (int32_t)v;
        resume[v] = 0;
    }
    if (rank0) {
        lcnt[0] = n;
        lcnt[1] = 0;
        lcnt[2] = 0;
        lcnt[3] = -1;  // the largest colour given so far
    }
    if (!gbar(bar, limit_ns)) return;
    for (int round = 0; round <= n; round++) {
        const int32_t *in = (round & 1) ? wl1 : wl0;
        int32_t *out = (round & 1) ? wl0 : wl1;
        const int32_t cnt = *((volatile int32_t *)&lcnt[round % 3]);
        if (rank0) lcnt[(round + 2) % 3] = 0;
        // the nodes left uncoloured are gathered per warp and appended 32 at
        // a time, one atomic for each
        int nbuf = 0;
        int *buf = keep[threadIdx.x >> 5];
        for (long long k = warp; k < cnt; k += nw) {
            const int v = in[k];
            if (colour_node(v, rp, col, seed, t, round, cr, bm, resume, lcnt + 3)) {
                if (lane == 0) buf[nbuf] = v;
                if (++nbuf == 32) {
                    __syncwarp();
                    int at = 0;
                    if (lane == 0) at = atomicAdd(&lcnt[(round + 1) % 3], 32);
                    at = __shfl_sync(0xffffffffu, at, 0);
                    out[at + lane] = buf[lane];
                    __syncwarp();
                    nbuf = 0;
                }
            }
        }
        if (nbuf > 0) {
            __syncwarp();
            int at = 0;
            if (lane == 0) at = atomicAdd(&lcnt[(round + 1) % 3], nbuf);
            at = __shfl_sync(0xffffffffu, at, 0);
            if (lane < nbuf) out[at + lane] = buf[lane];
            __syncwarp();
        }
        if (!gbar(bar, limit_ns)) return;
        if (*((volatile int32_t *)&lcnt[(round + 1) % 3]) == 0) {
            if (rank0) *rounds_out = round + 1;
            return;
        }
    }
}

// Small graphs (at most kColourSeqMax nodes, so every row is shorter than
// kColourBits): the first-fit colouring itself, one node after the other in
// key order, by one block with a bitmap of the node's neighbours' colours.
// Dense aggregated levels would need about one Jones-Plassmann round per node.
constexpr int32_t kColourSeqMax = 4096;

__global__ void k_colour_keys(int32_t n, unsigned long long seed, int t, unsigned long long *key,
                              int32_t *node) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        key[v] = ~colour_key(seed, t, (int)v);  // ascending sort = descending key
        node[v] = (int32_t)v;
    }
}

__global__ void __launch_bounds__(512) k_colour_seq(int32_t n, const int32_t *order, const int32_t *rp,
                                                    const int32_t *col, long long *cr) {
    __shared__ unsigned bm[kColourBits / 32];
    __shared__ int first;
    for (int k = 0; k < n; k++) {
        const int v = order[k];
        const int b = rp[v], e = rp[v + 1];
        const int words = (e - b) / 32 + 1;  // covers colours 0 .. row length
        for (int q = threadIdx.x; q < words; q += blockDim.x) bm[q] = 0u;
        if (threadIdx.x == 0) first = INT_MAX;
        __syncthreads();
        for (int p = b + threadIdx.x; p < e; p += blockDim.x) {
            const int u = col[p];
            if (u == v) continue;
            const long long c = cr[u];
            if (c >= 0 && c < 32LL * words) atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        __syncthreads();
        for (int q = threadIdx.x; q < words; q += blockDim.x)
            if (bm[q] != 0xffffffffu) atomicMin(&first, 32 * q + __ffs((int)~bm[q]) - 1);
        __syncthreads();
        if (threadIdx.x == 0) cr[v] = first;
        __syncthreads();  // the colour is visible to the next node's look
    }
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

// The decision of one listed node by one block, for level graphs small
// enough that a colour class holds a few nodes: the MAXIMAL scan's decision
// (stay unless the best other neighbouring community, ties to the smallest
// name, beats the own one by a positive amount) from a shared-memory table of
// the neighbouring communities' weights, 2^lg slots (at least twice the
// row's length).  Self-loops are left out as the scan leaves them out.
__global__ void __launch_bounds__(256) k_louvain_decide(const int32_t *list, int32_t cnt, const int32_t *rp,
                                                        const int32_t *col, const int32_t *w,
                                                        const int32_t *s, long long m, const int32_t *comm,
                                                        const int32_t *sigma, int lg, int32_t *best) {
    extern __shared__ int tab[];
    __shared__ long long w_sc[8], w_own[8];
    __shared__ int w_c[8];
    const int T = 1 << lg;
    int *keys = tab, *vals = tab + T;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long k = blockIdx.x; k < cnt; k += gridDim.x) {
        const int i = list[k];
        const int ci = comm[i];
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            keys[t] = -1;
            vals[t] = 0;
        }
        __syncthreads();
        long long own = 0;
        const int b = rp[i], e = rp[i + 1];
        for (int p = b + threadIdx.x; p < e; p += blockDim.x) {
            const int j = col[p];
            if (j == i) continue;
            const int c = comm[j], wv = w[p];
            if (c == ci) {
                own += wv;
                continue;
            }
            unsigned h = ((unsigned)c * 2654435761u) >> (32 - lg);
            for (;;) {
                const int prev = atomicCAS(&keys[h], -1, c);
                if (prev == -1 || prev == c) {
                    atomicAdd(&vals[h], wv);
                    break;
                }
                h = (h + 1) & (unsigned)(T - 1);
            }
        }
        __syncthreads();
        const long long si = s[i];
        long long bsc = LLONG_MIN;
        int bc = INT_MAX;
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            const int c = keys[t];
            if (c < 0) continue;
            const long long sc = m * (long long)vals[t] - si * (long long)sigma[c];
            if (sc > bsc || (sc == bsc && c < bc)) {
                bsc = sc;
                bc = c;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            own += __shfl_xor_sync(0xffffffffu, own, o);
            const long long osc = __shfl_xor_sync(0xffffffffu, bsc, o);
            const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
            if (osc > bsc || (osc == bsc && oc < bc)) {
                bsc = osc;
                bc = oc;
            }
        }
        if (lane == 0) {
            w_sc[wid] = bsc;
            w_c[wid] = bc;
            w_own[wid] = own;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long tsc = LLONG_MIN, town = 0;
            int tc = INT_MAX;
            for (int q = 0; q < (int)(blockDim.x >> 5); q++) {
                town += w_own[q];
                if (w_sc[q] > tsc || (w_sc[q] == tsc && w_c[q] < tc)) {
                    tsc = w_sc[q];
                    tc = w_c[q];
                }
            }
            const long long g = m * town - si * ((long long)sigma[ci] - si);
            best[i] = (tc != INT_MAX && tsc - g > 0) ? tc : ci;
        }
        __syncthreads();  // the table is cleared for the next node
    }
}

__global__ void k_class_max_row(int32_t n, const int32_t *rp, const int32_t *colour, int32_t *mx) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int d = rp[v + 1] - rp[v];
        if (d > 0) atomicMax(&mx[colour[v]], d);
    }
}

__global__ void k_max_row(int32_t n, const int32_t *rp, int32_t *mx) {
    int d = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        d = max(d, rp[v + 1] - rp[v]);
#pragma unroll
    for (int o = 16; o; o >>= 1) d = max(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0 && d > 0) atomicMax(mx, d);
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
    if (n <= kColourSeqMax) {
        DevBuf key(8 * (size_t)n, st), ktmp(8 * (size_t)n, st), ord(4 * (size_t)n, st), otmp(4 * (size_t)n, st);
        k_colour_keys<<<grid_for(n, 256), 256, 0, st>>>(n, seed, level, key.as<unsigned long long>(),
                                                        ord.as<int32_t>());
        SLM_LAUNCH_CHECK();
        radix_sort_u64(key.as<unsigned long long>(), ord.as<int32_t>(), ktmp.as<unsigned long long>(),
                       otmp.as<int32_t>(), n, 64, st);
        k_colour_seq<<<1, 512, 0, st>>>(n, ord.as<int32_t>(), rp, col, cr.as<long long>());
        SLM_LAUNCH_CHECK();
        SLM_CUDA(cudaMemsetAsync(lp, 0, 8, st));
    } else {
        // the barrier word, the three list counters and the largest colour,
        // the two node lists and the resume offsets
        DevBuf barm(sizeof(GridBarrier) + 16, st), wl(12 * (size_t)n, st);
        SLM_CUDA(cudaMemsetAsync(barm.get(), 0, sizeof(GridBarrier) + 16, st));
        GridBarrier *bar = barm.as<GridBarrier>();
        int32_t *cnt3 = reinterpret_cast<int32_t *>(bar + 1);
        int32_t *wl0 = wl.as<int32_t>(), *wl1 = wl0 + n, *resume = wl0 + 2 * (size_t)n;
        int dev = 0, sms = 0, per_sm = 0;
        SLM_CUDA(cudaGetDevice(&dev));
        SLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        SLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_colour_rounds, 256, 0));
        if (per_sm < 1) fail(SLM_ERR_CUDA, "colouring kernel cannot be resident");
        // every resident block while the lists are long (a warp per node),
        // no more blocks than a warp per node needs
        const int nb = (int)std::min<long long>((long long)sms * per_sm, ((long long)n * 32 + 255) / 256);
        long long lim = kBarrierLimitNs;
        long long *cr_p = cr.as<long long>();
        int32_t *rounds = lp + 2;
        void *kargs[] = {&n, (void *)&rp, (void *)&col, &seed, &level, (void *)&cr_p, &wl0, &wl1, &resume,
                         &bar, &cnt3, &lim, &rounds};
        serialised_cooperative(st, [&] {
            SLM_CUDA(cudaLaunchCooperativeKernel((const void *)k_colour_rounds, dim3(nb), dim3(256), kargs,
                                                 0, st));
            SLM_LAUNCH_CHECK();
        });
        GridBarrier hb{};
        SLM_CUDA(cudaMemcpyAsync(&hb, bar, sizeof hb, cudaMemcpyDeviceToHost, st));
        stream_sync(st);
        if (hb.failed) fail(SLM_ERR_TIMEOUT, "a colouring grid barrier waited past its time limit");
        SLM_CUDA(cudaMemsetAsync(lp, 0, 8, st));
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

int32_t max_row_length(int32_t n, const int32_t *rp, cudaStream_t st) {
    if (n <= 0) return 0;
    DevBuf mx(16, st);
    SLM_CUDA(cudaMemsetAsync(mx.get(), 0, 16, st));
    k_max_row<<<grid_for(n, 256), 256, 0, st>>>(n, rp, mx.as<int32_t>());
    SLM_LAUNCH_CHECK();
    int32_t h = 0;
    SLM_CUDA(cudaMemcpyAsync(&h, mx.get(), sizeof h, cudaMemcpyDeviceToHost, st));
    stream_sync(st);
    return h;
}

std::vector<int32_t> class_max_rows(int32_t n, const int32_t *rp, const int32_t *colour, int32_t ncol,
                                    cudaStream_t st) {
    std::vector<int32_t> h((size_t)(ncol > 0 ? ncol : 0), 0);
    if (n <= 0 || ncol <= 0) return h;
    DevBuf mx(4 * (size_t)ncol, st);
    SLM_CUDA(cudaMemsetAsync(mx.get(), 0, 4 * (size_t)ncol, st));
    k_class_max_row<<<grid_for(n, 256), 256, 0, st>>>(n, rp, colour, mx.as<int32_t>());
    SLM_LAUNCH_CHECK();
    SLM_CUDA(cudaMemcpyAsync(h.data(), mx.get(), 4 * (size_t)ncol, cudaMemcpyDeviceToHost, st));
    stream_sync(st);
    return h;
}

void louvain_decide(const int32_t *list, int32_t cnt, const int32_t *rp, const int32_t *col,
                    const int32_t *w, const int32_t *s, long long m, const int32_t *comm,
                    const int32_t *sigma, int32_t max_row, int32_t *best, cudaStream_t st) {
    if (cnt <= 0) return;
    if (max_row > kLouvainDecideMaxRow) fail(SLM_ERR_INVALID_ARGUMENT, "row too long for the direct decision");
    int lg = 5;
    while ((1 << lg) < 2 * max_row) lg++;
    const size_t smem = (size_t)8 << lg;
    static std::mutex mu;
    static unsigned long long ready = 0;  // bit d: device d allows the largest table
    int dev = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 64 || !((ready >> dev) & 1ull)) {
            SLM_CUDA(cudaFuncSetAttribute(k_louvain_decide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)((size_t)8 << kLouvainDecideMaxLg)));
            if (dev < 64) ready |= 1ull << dev;
        }
    }
    k_louvain_decide<<<(int)std::min<long long>(cnt, (long long)kNumSMs * 8), 256, smem, st>>>(
        list, cnt, rp, col, w, s, m, comm, sigma, lg, best);
    SLM_LAUNCH_CHECK();
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
