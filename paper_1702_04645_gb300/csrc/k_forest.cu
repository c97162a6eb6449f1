// k_forest.cu -- kernels on the assignment graph a (one out-edge per node).
//
//  * forest_analyse: COMPONENTS (Section 3.2): communities are the weakly
//    connected components of a, each holding one cycle; a community is named
//    by the smallest node on its cycle.  Pointer jumping with a running
//    minimum gives the names in ceil(log2 n) rounds; a second jumping pass
//    gives every node's entry (first cycle node on its path), its depth, and
//    for cycle nodes the forward distance to the name.
//  * branch_gains: Algorithm MAXIMAL's Delta H(c_i -> b(i) -> c_i^*) for every
//    candidate i: the tail b(i) is every node whose path reaches i.  Leaves
//    reuse the single-node gain, cycle nodes move their whole community, and
//    inner tree nodes aggregate their subtree by ancestor walks, with the
//    weight inside the subtree credited at the lowest common ancestor of each
//    edge's endpoints.
#include <climits>

#include "forest_dev.cuh"

namespace slm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
#define GRID_STRIDE SLM_GRID_STRIDE

// ---------------------------------------------------------------------------
// Components
// ---------------------------------------------------------------------------
// Every kernel of COMPONENTS runs over all n nodes (list == nullptr) or over
// the n nodes listed, a set closed under a (their paths never leave it).
#define NODE_LOOP(v, n, list)            \
    GRID_STRIDE(_k, n)                   \
    for (long long v = list ? list[_k] : _k, _o = 1; _o; _o = 0)

// ---------------------------------------------------------------------------
// Branch gains of Algorithm MAXIMAL
// ---------------------------------------------------------------------------
__global__ void k_haschild(int32_t n, const int32_t *a, int32_t *haschild) {
    GRID_STRIDE(v, n) if (a[v] != v) haschild[a[v]] = 1;
}

// 0: not a candidate, 1: bg = single-node gain (leaf or singleton), 2: cycle node, 3: inner tree node
__device__ __forceinline__ int cand_kind(int i, const int32_t *a, const uint8_t *oncycle,
                                         const int32_t *haschild, const long long *gain) {
    if (gain[i] <= 0) return 0;
    if (oncycle[i]) return (a[i] == i && !haschild[i]) ? 1 : 2;
    return haschild[i] ? 3 : 1;
}

__global__ void k_classify(int32_t n, const int32_t *a, const uint8_t *oncycle,
                           const int32_t *entry, const int32_t *root, const int32_t *haschild,
                           const long long *gain, int32_t *active, int32_t *treeact,
                           int32_t *commcyc) {
    GRID_STRIDE(i, n) {
        int k = cand_kind((int)i, a, oncycle, haschild, gain);
        if (k == 3) { active[i] = 1; treeact[entry[i]] = 1; }
        else if (k == 2) commcyc[root[i]] = 1;
    }
}

// every node of a tree holding an inner candidate adds itself to the
// candidates among its ancestors (itself included)
// (strengths are summed as 64-bit values: for a directed graph the packed
// (out, in) pairs, whose components only grow)
template <class NM>
__global__ void k_walk_tree(int32_t n, const int32_t *a, const uint8_t *oncycle,
                            const int32_t *entry, const int32_t *depth, const int32_t *treeact,
                            const int32_t *active,
                            const typename NM::ST *s, const int32_t *kown, long long *subS,
                            long long *subWA, int32_t *covered) {
    GRID_STRIDE(x, n) {
        if (oncycle[x] || !treeact[entry[x]]) continue;
        int y = (int)x, cov = 0;
        long long sx = (long long)s[x], kx = kown[x];
        for (int d = depth[x]; d > 0; d--) {  // the non-cycle ancestors, x included
            if (active[y]) {
                add64(&subS[y], sx);
                add64(&subWA[y], kx);
                cov = 1;
            }
            y = a[y];
        }
        if (cov) covered[x] = 1;
    }
}

// weight from the subtree to the target community, and LCA credits for the
// weight inside the subtree; one warp per covered node
__global__ void k_edges_tree(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                             const int32_t *a, const uint8_t *oncycle, const int32_t *entry,
                             const int32_t *depth, const int32_t *root, const int32_t *best,
                             const int32_t *active, const int32_t *covered, long long *WB,
                             long long *credit) {
    __shared__ int lst[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // each warp tests 32 consecutive nodes at once and then serves the
    // covered ones with all its lanes
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
         base += (long long)gridDim.x * blockDim.x)
    for (unsigned sel = __ballot_sync(FULL, base + lane < n && covered[base + lane]); sel;
         sel &= sel - 1) {
        const int x = (int)(base + __ffs(sel) - 1);
        const int rx = root[x], ex = entry[x];
        int y = x, dleft = depth[x];
        bool first_pass = true;
        while (true) {
            // collect up to 32 inner candidates on the path, starting at y
            int k = 0;
            if (lane == 0) {
                while (dleft > 0 && k < 32) {
                    if (active[y]) lst[wib][k++] = y;
                    y = a[y];
                    dleft--;
                }
            }
            k = __shfl_sync(FULL, k, 0);
            dleft = __shfl_sync(FULL, dleft, 0);
            __syncwarp();
            for (int p = rp[x] + lane; p < rp[x + 1]; p += 32) {
                int j = col[p];
                if (j == x) continue;
                int rj = root[j], wv = w[p];
                for (int t = 0; t < k; t++) {
                    int c = lst[wib][t];
                    if (rj == best[c]) add64(&WB[c], wv);
                }
                if (first_pass && rj == rx && entry[j] == ex) {
                    int l = lca_walk(x, j, a, depth);
                    if (!oncycle[l] && covered[l]) add64(&credit[l], wv);
                }
            }
            first_pass = false;
            __syncwarp();
            if (dleft == 0) break;
        }
    }
}

__global__ void k_walk_credit(int32_t n, const int32_t *a, const int32_t *depth,
                              const int32_t *active, const long long *credit,
                              long long *subWin) {
    GRID_STRIDE(x, n) {
        long long c = credit[x];
        if (c == 0) continue;
        int y = (int)x;
        for (int d = depth[x]; d > 0; d--) {
            if (active == nullptr || active[y]) add64(&subWin[y], c);
            y = a[y];
        }
    }
}

// weight from a whole community to each of its cycle candidates' targets
__global__ void k_edges_cycle(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                              const int32_t *a, const int32_t *root, const int32_t *cdist,
                              const int32_t *best, const long long *gain, const int32_t *commcyc,
                              long long *WB) {
    __shared__ int lst[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
         base += (long long)gridDim.x * blockDim.x)
    for (unsigned sel = __ballot_sync(FULL, base + lane < n && commcyc[root[base + lane]]); sel;
         sel &= sel - 1) {
        const int x = (int)(base + __ffs(sel) - 1);
        const int r = root[x];
        int c = r;
        // cycle length: the name's successor is L-1 steps from the name
        int left = (a[r] == r) ? 1 : cdist[a[r]] + 1;
        while (true) {
            int k = 0;
            if (lane == 0) {
                // walk the cycle from its name, at most 32 candidates per pass
                while (k < 32 && left > 0) {
                    if (gain[c] > 0) lst[wib][k++] = c;
                    c = a[c];
                    left--;
                }
            }
            k = __shfl_sync(FULL, k, 0);
            left = __shfl_sync(FULL, left, 0);
            __syncwarp();
            for (int p = rp[x] + lane; p < rp[x + 1]; p += 32) {
                int j = col[p];
                if (j == x) continue;
                int rj = root[j], wv = w[p];
                for (int t = 0; t < k; t++) {
                    int cc = lst[wib][t];
                    if (rj == best[cc]) add64(&WB[cc], wv);
                }
            }
            __syncwarp();
            if (left == 0) break;
        }
    }
}

template <class NM>
__global__ void k_bg_final(int32_t n, const int32_t *a, const uint8_t *oncycle,
                           const int32_t *root, const int32_t *haschild,
                           const typename NM::ST *sigma,
                           const int32_t *best, const long long *gain, MParam mp,
                           const long long *subS, const long long *subWA, const long long *subWin,
                           const long long *WB, long long *bg) {
    GRID_STRIDE(i, n) {
        const long long m = mp.of((int)i);
        int k = cand_kind((int)i, a, oncycle, haschild, gain);
        long long r = 0;
        long long sA = (long long)sigma[root[i]], sB = (long long)sigma[best[i]];
        if (k == 1) r = gain[i];
        else if (k == 2) r = m * WB[i] - NM::cross(sA, sB);
        else if (k == 3) {
            long long sS = subS[i];
            long long wout = subWA[i] - subWin[i];
            // S (sB - sA + S) expanded, so that no packed difference can go negative
            r = m * (WB[i] - wout) - (NM::cross(sS, sB) - NM::cross(sS, sA) + NM::cross(sS, sS));
        }
        bg[i] = r;
    }
}

__global__ void k_accept(int32_t n, const long long *bg, RngParam rng, unsigned long long P,
                         int level, int sweep, int32_t *list, int32_t *cnt,
                         unsigned long long *npos, const int32_t *active, int32_t *per_graph) {
    // the accepted nodes are appended with one atomic per warp (the list's
    // order is free: every use of it is per node)
    const int lane = threadIdx.x & 31;
    unsigned loc = 0;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + lane;
        bool acc = false, cand = false;
        int g = 0;
        if (i < n && bg[i] > 0) {
            g = rng.gid ? rng.gid[i] : 0;
            if (!active || active[g]) {
                cand = true;
                loc++;
                acc = (unsigned long long)accept_draw(rng.seed_of((int)i), level, sweep, rng.local((int)i)) < P;
            }
        }
        if (per_graph) {  // uniform over the launch
            warp_count(per_graph, 2 * g, cand);
            warp_count(per_graph, 2 * g + 1, acc);
        }
        const unsigned bal = __ballot_sync(FULL, acc);
        int at = 0;
        if (lane == 0 && bal) at = atomicAdd(cnt, __popc(bal));
        at = __shfl_sync(FULL, at, 0);
        if (acc) list[at + __popc(bal & ((1u << lane) - 1u))] = (int)i;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) loc += __shfl_xor_sync(FULL, loc, o);
    if ((threadIdx.x & 31) == 0 && loc) atomicAdd(npos, (unsigned long long)loc);
}

__global__ void k_apply(const int32_t *list, const int32_t *cnt, const int32_t *tgt, int32_t *a) {
    GRID_STRIDE(idx, *cnt) {
        int i = list[idx];
        a[i] = tgt[i];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int jump_rounds(int32_t n) {
    int K = 0;
    while ((1LL << K) < (long long)n) K++;
    return K;
}

namespace {
// Every round of COMPONENTS in one launch, its phases separated by barriers
// (block barriers for a single block, the time-limited grid barrier for a
// cooperative grid): pointer jumping with a running minimum names every
// component by the smallest node on its cycle and marks the cycle nodes; a
// second jumping pass gives every node its entry (first cycle node on its
// path) and depth, and every cycle node its forward distance to the name.
constexpr int kForestThreads = 1024;
constexpr int kForestOneBlock = 4096;  // listed nodes up to which one block runs them all

__global__ void __launch_bounds__(kForestThreads) k_forest_rounds(
    int32_t cnt, const int32_t *list, const int32_t *a, int2 *JA, int2 *JB, int32_t *root,
    uint8_t *oncycle, int32_t *entry, int32_t *depth, int32_t *cdist, int K, GridBarrier *bar,
    long long limit_ns, int *changed) {
    NODE_LOOP(v, cnt, list) JA[v] = make_int2(a[v], (int)v);
    if (!gbar(bar, limit_ns)) return;
    int2 *cur = JA, *nxt = JB;
    for (int k = 0; k < K; k++) {
        NODE_LOOP(v, cnt, list) {
            const int2 x = cur[v];
            const int2 y = cur[x.x];
            nxt[v] = make_int2(y.x, min(x.y, y.y));
        }
        if (!gbar(bar, limit_ns)) return;
        int2 *t = cur;
        cur = nxt;
        nxt = t;
    }
    NODE_LOOP(v, cnt, list) oncycle[v] = 0;
    if (!gbar(bar, limit_ns)) return;
    NODE_LOOP(v, cnt, list) {
        const int c = cur[v].x;  // a^(2^K)(v): on the cycle
        root[v] = cur[c].y;      // minimum over 2^K >= L consecutive cycle nodes
        oncycle[c] = 1;
    }
    if (!gbar(bar, limit_ns)) return;
    // the tree nodes walk to their entry, the cycle nodes to their name; the
    // buffer that does not hold the names' jumps takes the distances
    int2 *D0 = (cur == JA) ? JB : JA, *D1 = cur;
    NODE_LOOP(v, cnt, list) {
        if (oncycle[v] && root[v] == v) D0[v] = make_int2((int)v, 0);
        else D0[v] = make_int2(a[v], 1);
    }
    if (!gbar(bar, limit_ns)) return;
    cur = D0;
    nxt = D1;
    // this pass reaches a fixed point (tree nodes stop at their entry, cycle
    // nodes at the name): once a round changes nothing, the later rounds
    // would not either; changed[k] (zeroed by the host) records round k
    __shared__ int any;
    for (int k = 0; k < K; k++) {
        if (threadIdx.x == 0) any = 0;
        __syncthreads();
        int mine = 0;
        NODE_LOOP(v, cnt, list) {
            const int2 x = cur[v];
            int2 z = x;
            if (oncycle[v] || !oncycle[x.x]) {
                const int2 y = cur[x.x];
                z = make_int2(y.x, x.y + y.y);
            }
            nxt[v] = z;
            mine |= (z.x != x.x || z.y != x.y) ? 1 : 0;
        }
        if (mine) any = 1;
        __syncthreads();
        if (threadIdx.x == 0 && any) atomicOr(&changed[k], 1);
        if (!gbar(bar, limit_ns)) return;
        int2 *t = cur;
        cur = nxt;
        nxt = t;
        if (*((volatile int *)&changed[k]) == 0) break;  // the same in every block
    }
    NODE_LOOP(v, cnt, list) {
        const int2 d = cur[v];
        if (oncycle[v]) {
            entry[v] = (int)v;
            depth[v] = 0;
            cdist[v] = d.y;
        } else {
            entry[v] = d.x;
            depth[v] = d.y;
            cdist[v] = 0;
        }
    }
}
}  // namespace

static void forest_pass(int32_t cnt, const int32_t *list, const int32_t *a, Forest &f,
                        cudaStream_t st) {
    // 2^K >= cnt jumps reach the cycle from any listed node and cover its cycle
    int K = jump_rounds(cnt);
    // the barrier word, then one "changed" word per round of the second pass
    DevBuf barm(sizeof(GridBarrier) + sizeof(int) * 64, st);
    SLM_CUDA(cudaMemsetAsync(barm.get(), 0, sizeof(GridBarrier) + sizeof(int) * 64, st));
    GridBarrier *bar = barm.as<GridBarrier>();
    int *changed = reinterpret_cast<int *>(bar + 1);
    long long lim = kBarrierLimitNs;
    if (cnt <= kForestOneBlock) {
        // one block: block barriers only, an ordinary launch
        k_forest_rounds<<<1, kForestThreads, 0, st>>>(cnt, list, a, f.jmpA, f.jmpB, f.root, f.oncycle,
                                                      f.entry, f.depth, f.cdist, K, bar, lim, changed);
        SLM_LAUNCH_CHECK();
        return;
    }
    int dev = 0, sms = 0, per_sm = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    SLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forest_rounds, kForestThreads, 0));
    if (per_sm < 1) fail(SLM_ERR_CUDA, "COMPONENTS kernel cannot be resident");
    int nb = (int)std::min<long long>((long long)sms, (cnt + kForestThreads - 1) / kForestThreads);
    void *kargs[] = {&cnt, (void *)&list, (void *)&a, &f.jmpA, &f.jmpB, &f.root, &f.oncycle,
                     &f.entry, &f.depth, &f.cdist, &K, &bar, &lim, &changed};
    serialised_cooperative(st, [&] {
        SLM_CUDA(cudaLaunchCooperativeKernel((const void *)k_forest_rounds, dim3(nb),
                                             dim3(kForestThreads), kargs, 0, st));
        SLM_LAUNCH_CHECK();
    });
    GridBarrier hb{};
    SLM_CUDA(cudaMemcpyAsync(&hb, bar, sizeof hb, cudaMemcpyDeviceToHost, st));
    stream_sync(st);
    if (hb.failed) fail(SLM_ERR_TIMEOUT, "a COMPONENTS grid barrier waited past its time limit");
}

void forest_analyse(int32_t n, const int32_t *a, Forest &f, cudaStream_t st) {
    if (n <= 0) return;
    forest_pass(n, nullptr, a, f, st);
}

void forest_analyse_subset(int32_t cnt, const int32_t *list, const int32_t *a, Forest &f,
                           cudaStream_t st) {
    if (cnt <= 0) return;
    forest_pass(cnt, list, a, f, st);
}

template <class NM>
void branch_gains(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                  const typename NM::ST *s, MParam m, const int32_t *a, const Forest &f,
                  const typename NM::ST *sigma, const int32_t *best, const long long *gain,
                  const int32_t *kown, BranchScratch &bs, long long *bg, cudaStream_t st) {
    if (n <= 0) return;
    const int g = grid_for(n, 256);
    const int gw = grid_for((long long)n * 32, 256, kNumSMs * 16);
    // the five int32 and five int64 arrays, one memset each when they lie
    // back to back (as the per-level workspace lays them out)
    if (bs.active == bs.haschild + n && bs.covered == bs.active + n && bs.treeact == bs.covered + n &&
        bs.commcyc == bs.treeact + n)
        SLM_CUDA(cudaMemsetAsync(bs.haschild, 0, sizeof(int32_t) * 5 * (size_t)n, st));
    else
        for (int32_t *p : {bs.haschild, bs.active, bs.covered, bs.treeact, bs.commcyc})
            SLM_CUDA(cudaMemsetAsync(p, 0, sizeof(int32_t) * n, st));
    if (bs.subWA == bs.subS + n && bs.subWin == bs.subWA + n && bs.credit == bs.subWin + n &&
        bs.WB == bs.credit + n)
        SLM_CUDA(cudaMemsetAsync(bs.subS, 0, sizeof(long long) * 5 * (size_t)n, st));
    else
        for (long long *p : {bs.subS, bs.subWA, bs.subWin, bs.credit, bs.WB})
            SLM_CUDA(cudaMemsetAsync(p, 0, sizeof(long long) * n, st));
    k_haschild<<<g, 256, 0, st>>>(n, a, bs.haschild);
    SLM_LAUNCH_CHECK();
    k_classify<<<g, 256, 0, st>>>(n, a, f.oncycle, f.entry, f.root, bs.haschild, gain, bs.active,
                                  bs.treeact, bs.commcyc);
    SLM_LAUNCH_CHECK();
    k_walk_tree<NM><<<g, 256, 0, st>>>(n, a, f.oncycle, f.entry, f.depth, bs.treeact, bs.active, s, kown,
                                   bs.subS, bs.subWA, bs.covered);
    SLM_LAUNCH_CHECK();
    k_edges_tree<<<gw, 256, 0, st>>>(n, rp, col, w, a, f.oncycle, f.entry, f.depth, f.root, best,
                                     bs.active, bs.covered, bs.WB, bs.credit);
    SLM_LAUNCH_CHECK();
    k_walk_credit<<<g, 256, 0, st>>>(n, a, f.depth, bs.active, bs.credit, bs.subWin);
    SLM_LAUNCH_CHECK();
    k_edges_cycle<<<gw, 256, 0, st>>>(n, rp, col, w, a, f.root, f.cdist, best, gain, bs.commcyc, bs.WB);
    SLM_LAUNCH_CHECK();
    k_bg_final<NM><<<g, 256, 0, st>>>(n, a, f.oncycle, f.root, bs.haschild, sigma, best, gain, m,
                                  bs.subS, bs.subWA, bs.subWin, bs.WB, bg);
    SLM_LAUNCH_CHECK();
}

void accept_moves(int32_t n, const long long *bg, RngParam rng, unsigned long long P,
                  int32_t level, int32_t sweep, int32_t *acc_list, int32_t *acc_cnt_dev,
                  unsigned long long *npos_dev, cudaStream_t st, const int32_t *active,
                  int32_t *per_graph) {
    if (n <= 0) return;
    k_accept<<<grid_for(n, 256), 256, 0, st>>>(n, bg, rng, P, level, sweep, acc_list, acc_cnt_dev,
                                               npos_dev, active, per_graph);
    SLM_LAUNCH_CHECK();
}

void apply_moves(const int32_t *list, const int32_t *cnt_dev, int32_t max_cnt, const int32_t *tgt,
                 int32_t *a, cudaStream_t st) {
    if (max_cnt <= 0) return;
    k_apply<<<grid_for(max_cnt, 256), 256, 0, st>>>(list, cnt_dev, tgt, a);
    SLM_LAUNCH_CHECK();
}

template void branch_gains<NMSym>(int32_t, const int32_t *, const int32_t *, const int32_t *,
                                 const int32_t *, MParam, const int32_t *, const Forest &,
                                 const int32_t *, const int32_t *, const long long *,
                                 const int32_t *, BranchScratch &, long long *, cudaStream_t);
template void branch_gains<NMDir>(int32_t, const int32_t *, const int32_t *, const int32_t *,
                                 const unsigned long long *, MParam, const int32_t *,
                                 const Forest &, const unsigned long long *, const int32_t *,
                                 const long long *, const int32_t *, BranchScratch &,
                                 long long *, cudaStream_t);

}  // namespace slm
