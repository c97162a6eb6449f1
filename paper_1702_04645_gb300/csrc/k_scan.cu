// k_scan.cu -- neighbourhood scans of the Synchronised Louvain Method.
//
//  * scan_nodes: the per-node half of MAXIMAL (Section 3.4, Algorithm
//    MAXIMAL's c_i^* = argmax_c Delta H(c_i -> i -> c)): accumulate the weight
//    k_{i,C} from node i to every neighbouring community C and pick the best
//    by the exact score m_w k_{i,C} - s_i Sigma_C (Section 2.4).  Rows of up
//    to 4096 entries are scanned by the kernels of k_scan_fine.cu; hubs by
//    the global-table kernels here.
//  * assign_nodes: ASSIGN (Section 3.1): best neighbour by m_w W_ij - s_i s_j.
//  * target_nodes: the new assignment a(i) = argmax_{j in c_i^*} of the same
//    pair score (Algorithm MAXIMAL).
//  * own_weight_nodes: k_{i,c_i} and the local gain g(i) of POSITIVE
//    (Section 3.3, Algorithm POSITIVE).
//
// Degree buckets pick the shape of ASSIGN, the own weights and the scan: lane
// groups or warps for short rows, blocks for long ones, and for hubs (more
// than 4096 entries) a global-memory table shared by the blocks of a row.
// Every reduction compares (score desc, name asc), so the result does not
// depend on the order in which lanes or blocks finish.
#include <algorithm>
#include <climits>
#include <initializer_list>
#include <mutex>

#include "slm_internal.cuh"

namespace slm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kHubSlice = 2048;  // hub table slots read by one block
constexpr int kBlockThreads = 256;

__device__ __forceinline__ int fine_of(int d) {
    if (d == 0) return kFineEmpty;
    if (d <= 4) return kFine4;
    if (d <= 8) return kFine8;
    if (d <= 16) return kFine16;
    if (d <= 32) return kFine32;
    if (d <= 64) return kFine64;
    if (d <= 128) return kFine128;
    if (d <= 256) return kFine256;
    if (d <= 512) return kFine512;
    if (d <= 1024) return kFine1024;
    if (d <= 2048) return kFine2048;
    if (d <= kBlockSmemMaxDeg) return kFine4096;
    return kFineHub;
}

// coarse bucket of every fine class
constexpr int kCoarseOf[kNumFine] = {kBucketEmpty, kBucketG4, kBucketG8, kBucketG16, kBucketG32,
                                     kBucketWarpHash, kBucketWarpHash, kBucketWarpHash,
                                     kBucketBlockS, kBucketBlockS, kBucketBlockM, kBucketBlockL,
                                     kBucketHub};
static_assert(kWarpHashMaxDeg == 256 && kBlockSmallMaxDeg == 1024 && kBlockMidMaxDeg == 2048,
              "coarse buckets must be unions of fine classes");

__device__ __forceinline__ bool better(long long sc, int c, long long bsc, int bc) {
    return sc > bsc || (sc == bsc && c < bc);
}

__device__ __forceinline__ unsigned hash_slot(int c, int lg) {
    return ((unsigned)c * 2654435761u) >> (32 - lg);
}


// Decision shared by every scan shape.
template <class NM>
__device__ __forceinline__ void scan_emit(int i, int ci, long long si, long long m,
                                          const typename NM::ST *sigma, long long own,
                                          long long bsc, int bc, int32_t *best,
                                          long long *gain, int32_t *kown, unsigned &cand) {
    long long g = m * own - NM::cross(si, (long long)sigma[ci] - si);
    long long gn = (bc != INT_MAX) ? bsc - g : 0;
    if (bc != INT_MAX && gn > 0) {
        best[i] = bc;
        gain[i] = gn;
        cand++;
    } else {
        best[i] = ci;
        gain[i] = 0;
    }
    kown[i] = (int32_t)own;
}

__device__ __forceinline__ void count_add(unsigned long long *ctr, unsigned v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, (unsigned long long)v);
}

// ---------------------------------------------------------------------------
// Buckets
// ---------------------------------------------------------------------------
// bucket keys of all n nodes (list == nullptr) or of the n listed nodes
__global__ void k_bucket_keys(int32_t n, const int32_t *list, const int32_t *rp, uint32_t *keys,
                              int32_t *vals, int32_t *counts) {
    __shared__ int loc[kNumFine];
    if (threadIdx.x < kNumFine) loc[threadIdx.x] = 0;
    __syncthreads();
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int v = list ? list[k] : (int)k;
        int b = fine_of(rp[v + 1] - rp[v]);
        keys[k] = (uint32_t)b;
        vals[k] = v;
        atomicAdd(&loc[b], 1);
    }
    __syncthreads();
    if (threadIdx.x < kNumFine && loc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], loc[threadIdx.x]);
}

// Block-wide argmax + sum; result valid in thread 0.
__device__ void block_reduce_best(long long &own, long long &sc, int &cc) {
    __shared__ long long r_own[32], r_sc[32];
    __shared__ int r_cc[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        own += __shfl_xor_sync(FULL, own, o);
        long long osc = __shfl_xor_sync(FULL, sc, o);
        int occ = __shfl_xor_sync(FULL, cc, o);
        if (better(osc, occ, sc, cc)) { sc = osc; cc = occ; }
    }
    if (lane == 0) { r_own[wid] = own; r_sc[wid] = sc; r_cc[wid] = cc; }
    __syncthreads();
    if (wid == 0) {
        own = lane < nw ? r_own[lane] : 0;
        sc = lane < nw ? r_sc[lane] : LLONG_MIN;
        cc = lane < nw ? r_cc[lane] : INT_MAX;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            own += __shfl_xor_sync(FULL, own, o);
            long long osc = __shfl_xor_sync(FULL, sc, o);
            int occ = __shfl_xor_sync(FULL, cc, o);
            if (better(osc, occ, sc, cc)) { sc = osc; cc = occ; }
        }
    }
    __syncthreads();
}

__global__ void k_scan_empty(const int32_t *order, int32_t cnt, const int32_t *root,
                             int32_t *best, long long *gain, int32_t *kown) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < cnt;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = order[idx];
        best[i] = root[i];
        gain[i] = 0;
        kown[i] = 0;
    }
}

// ---------------------------------------------------------------------------
// MAXIMAL scan, hub shape: a hub's row is split into chunks of kHubChunk
// edges, one block each, all inserting into the hub's global table; a second
// kernel, one block per hub, reads the table, resets it for the next sweep,
// and picks the best community.
// ---------------------------------------------------------------------------
// A chunk's entries are first summed per community in a shared-memory table
// (the entries of a hub often concentrate on a few large communities, whose
// global slots would otherwise take thousands of atomics each); then every
// community of the chunk goes into the hub's global table with one atomic.
__global__ void __launch_bounds__(kBlockThreads) k_hub_insert(const int4 *chunks, int nchunk, const int32_t *hubs,
                             const long long *hoff, const int32_t *hlg, const long long *uoff,
                             const int32_t *col, const int32_t *w, const int32_t *root,
                             unsigned long long *tslot, int *ulist, int *ucnt,
                             unsigned long long *own_acc) {
    // a chunk is at most kHubChunk = 8 * kBlockThreads entries: eight per
    // thread, loaded and inserted together so that their atomics overlap
    constexpr int B = kHubChunk / kBlockThreads;
    constexpr int SLG = 12;  // 4096 shared slots: twice a chunk
    static_assert((1 << SLG) == 2 * kHubChunk, "shared table of twice a chunk");
    __shared__ unsigned long long stab[1 << SLG];
    __shared__ unsigned long long red[kBlockThreads / 32];
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < (1 << SLG); k += kBlockThreads) stab[k] = 0ull;
    __syncthreads();
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const int4 ch = chunks[c];  // (hub index, first edge, end edge, unused)
        const int i = hubs[ch.x];
        const int ci = root[i];
        const int lg = hlg[ch.x];
        const unsigned mask = (1u << lg) - 1u;
        unsigned long long *T = tslot + hoff[ch.x];
        int *ul = ulist + uoff[ch.x];
        int cc[B], wv[B];
#pragma unroll
        for (int t = 0; t < B; t++) {
            const int p = ch.y + threadIdx.x + t * kBlockThreads;
            const int j = p < ch.z ? col[p] : i;
            wv[t] = p < ch.z ? w[p] : 0;
            cc[t] = j;
        }
#pragma unroll
        for (int t = 0; t < B; t++) cc[t] = cc[t] != i ? root[cc[t]] : -1;
        // the own community never enters a table (all of a star's leaves
        // would hit its one slot): summed per block, one atomic per chunk
        unsigned long long own = 0;
        int cl[B];
#pragma unroll
        for (int t = 0; t < B; t++) {
            if (cc[t] == ci) own += (unsigned long long)wv[t];
            cl[t] = -1;
            if (cc[t] < 0 || cc[t] == ci) continue;
            const unsigned long long key = (unsigned long long)(unsigned)(cc[t] + 1) << 32;
            unsigned h = ((unsigned)cc[t] * 2654435761u) >> (32 - SLG);
            for (;;) {
                const unsigned long long o = atomicCAS(&stab[h], 0ull, key | (unsigned)wv[t]);
                if (o == 0ull) { cl[t] = (int)h; break; }
                if ((o & 0xffffffff00000000ull) == key) {
                    atomicAdd(&stab[h], (unsigned long long)(unsigned)wv[t]);
                    break;
                }
                h = (h + 1) & ((1u << SLG) - 1u);
            }
        }
        __syncthreads();
        // every community of the chunk into the hub's table: the home-slot
        // CASes are issued before any result is looked at
        unsigned long long gv[B], gold[B];
        unsigned gh[B];
#pragma unroll
        for (int t = 0; t < B; t++) {
            gv[t] = 0ull;
            gold[t] = 1ull;
            gh[t] = 0u;
            if (cl[t] < 0) continue;
            gv[t] = stab[cl[t]];
            stab[cl[t]] = 0ull;  // empty again for the next chunk
            const unsigned cm = (unsigned)(gv[t] >> 32) - 1u;
            gh[t] = (cm * 2654435761u) >> (32 - lg);
            gold[t] = atomicCAS(&T[gh[t]], 0ull, gv[t]);
        }
        int claimed[B];
        unsigned bal[B];
        int nclaim = 0;
#pragma unroll
        for (int t = 0; t < B; t++) {
            claimed[t] = -1;
            if (cl[t] >= 0) {
                const unsigned long long key = gv[t] & 0xffffffff00000000ull;
                unsigned long long o = gold[t];
                unsigned hh = gh[t];
                for (;;) {
                    if (o == 0ull) { claimed[t] = (int)hh; break; }
                    if ((o & 0xffffffff00000000ull) == key) {
                        atomicAdd(&T[hh], gv[t] & 0xffffffffull);
                        break;
                    }
                    hh = (hh + 1) & mask;
                    o = atomicCAS(&T[hh], 0ull, gv[t]);
                }
            }
            bal[t] = __ballot_sync(FULL, claimed[t] >= 0);
            nclaim += __popc(bal[t]);
        }
        // the slots a warp claimed are listed with one atomic on the hub's count
        if (nclaim) {
            int at = 0;
            if (lane == 0) at = atomicAdd(&ucnt[ch.x], nclaim);
            at = __shfl_sync(FULL, at, 0);
            const unsigned below = (1u << lane) - 1u;
#pragma unroll
            for (int t = 0; t < B; t++) {
                if (claimed[t] >= 0) ul[at + __popc(bal[t] & below)] = claimed[t];
                at += __popc(bal[t]);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) own += __shfl_xor_sync(FULL, own, o);
        if (lane == 0) red[threadIdx.x >> 5] = own;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int k = 0; k < kBlockThreads / 32; k++) t += red[k];
            if (t) atomicAdd(&own_acc[ch.x], t);
        }
        __syncthreads();  // the shared table is empty and red is free
    }
}

// one block per slice of kHubSlice entries of a hub's list of occupied
// table slots: partial (own weight, best score, best community), and the
// slots are reset for the next scan
template <class NM>
__global__ void __launch_bounds__(kBlockThreads) k_hub_slices(const int2 *tchunks, int ntchunk, const int32_t *hubs,
                             const long long *hoff, const long long *uoff, const int *ulist,
                             const int *ucnt, const typename NM::ST *s, MParam mp, const int32_t *root,
                             const typename NM::ST *sigma, unsigned long long *tslot,
                             long long *part_sc, int32_t *part_cc) {
    constexpr int B = kHubSlice / kBlockThreads;
    for (int tc = blockIdx.x; tc < ntchunk; tc += gridDim.x) {
        const int2 d = tchunks[tc];  // (hub index, first list entry)
        const int i = hubs[d.x];
        const long long m = mp.of(i);
        const long long si = (long long)s[i];
        const int nu = ucnt[d.x];
        unsigned long long *T = tslot + hoff[d.x];
        const int *ul = ulist + uoff[d.x];
        int hh[B], kk[B], vv[B];
        long long sg[B];
#pragma unroll
        for (int t = 0; t < B; t++) {
            int k = d.y + threadIdx.x + t * kBlockThreads;
            hh[t] = k < nu ? ul[k] : -1;
        }
#pragma unroll
        for (int t = 0; t < B; t++) {
            const unsigned long long v = hh[t] >= 0 ? T[hh[t]] : 0ull;
            kk[t] = (int)(v >> 32) - 1;  // -1: no slot
            vv[t] = (int)(unsigned)v;
        }
#pragma unroll
        for (int t = 0; t < B; t++) sg[t] = kk[t] >= 0 ? (long long)sigma[kk[t]] : 0;
        long long own = 0, sc = LLONG_MIN;
        int cc = INT_MAX;
#pragma unroll
        for (int t = 0; t < B; t++) {
            int c = kk[t];
            if (c < 0) continue;
            T[hh[t]] = 0ull;  // leave the table empty for the next sweep
            long long x = m * (long long)vv[t] - NM::cross(si, sg[t]);
            if (better(x, c, sc, cc)) { sc = x; cc = c; }
        }
        block_reduce_best(own, sc, cc);
        if (threadIdx.x == 0) {
            part_sc[tc] = sc;
            part_cc[tc] = cc;
        }
    }
}
template <class NM>
__global__ void k_hub_finish(int nhub, const int32_t *hubs, const int32_t *tc_off,
                             const typename NM::ST *s, MParam mp, const int32_t *root,
                             const typename NM::ST *sigma,
                             unsigned long long *own_acc, const long long *part_sc,
                             const int32_t *part_cc, int *ucnt, int32_t *best, long long *gain,
                             int32_t *kown, unsigned long long *ncand) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned cand = 0;
    for (long long h = warp; h < nhub; h += nwarps) {
        const int i = hubs[h];
        const long long m = mp.of(i);
        long long sc = LLONG_MIN;
        int cc = INT_MAX;
        for (int t = tc_off[h] + lane; t < tc_off[h + 1]; t += 32)
            if (better(part_sc[t], part_cc[t], sc, cc)) { sc = part_sc[t]; cc = part_cc[t]; }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            long long osc = __shfl_xor_sync(FULL, sc, o);
            int occ = __shfl_xor_sync(FULL, cc, o);
            if (better(osc, occ, sc, cc)) { sc = osc; cc = occ; }
        }
        if (lane == 0) {
            const long long own = (long long)own_acc[h];
            scan_emit<NM>(i, root[i], (long long)s[i], m, sigma, own, sc, cc, best, gain, kown, cand);
            ucnt[h] = 0;     // the hub's slot list starts empty at the next scan
            own_acc[h] = 0;  // and so does its own-community sum
        }
    }
    count_add(ncand, cand);
}

// own-community weight of hubs: chunk partial sums, then the local gain
__global__ void __launch_bounds__(kBlockThreads) k_own_hub_chunk(const int4 *chunks, int nchunk, const int32_t *hubs,
                                const int32_t *col, const int32_t *w, const int32_t *root,
                                unsigned long long *acc) {
    __shared__ unsigned long long red[kBlockThreads / 32];
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        int4 ch = chunks[c];
        const int i = hubs[ch.x];
        const int ci = root[i];
        unsigned long long own = 0;
        for (int p = ch.y + threadIdx.x; p < ch.z; p += blockDim.x) {
            int j = col[p];
            if (j != i && root[j] == ci) own += (unsigned long long)w[p];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) own += __shfl_xor_sync(FULL, own, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = own;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int k = 0; k < kBlockThreads / 32; k++) t += red[k];
            if (t) atomicAdd(&acc[ch.x], t);
        }
        __syncthreads();
    }
}

template <class NM>
__global__ void k_own_hub_finish(int nhub, const int32_t *hubs, const typename NM::ST *s,
                                 MParam mp, const int32_t *root, const typename NM::ST *sigma,
                                 const unsigned long long *acc, int32_t *kown, int32_t *flag) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nhub; h += gridDim.x * blockDim.x) {
        int i = hubs[h];
        const long long m = mp.of(i);
        int ci = root[i];
        long long own = (long long)acc[h];
        kown[i] = (int32_t)own;
        long long si = (long long)s[i];
        if (m * own - NM::cross(si, (long long)sigma[ci] - si) < 0) flag[ci] = 1;
    }
}

__global__ void k_hub_rows(int nhub, const int32_t *hubs, const int32_t *rp, int2 *rows) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nhub; h += gridDim.x * blockDim.x)
        rows[h] = make_int2(rp[hubs[h]], rp[hubs[h] + 1]);
}

// ---------------------------------------------------------------------------
// Pair argmax (ASSIGN and target): argmax over neighbours j != i, optionally
// restricted to root[j] == want, of m_w W_ij - s_i s_j; ties smallest j.
// ---------------------------------------------------------------------------
struct PairBest {
    long long sc;
    int j;
};
__device__ __forceinline__ void pair_consider(PairBest &b, long long sc, int j) {
    if (better(sc, j, b.sc, b.j)) { b.sc = sc; b.j = j; }
}

template <class NM, int G>
__global__ void __launch_bounds__(256) k_assign_group(const int32_t *order, int32_t cnt, const int32_t *rp,
                               const int32_t *col, const int32_t *w, const typename NM::ST *s,
                               MParam mp, int32_t *a) {
    constexpr int NPW = 32 / G;
    const int lane = threadIdx.x & 31, gl = lane % G;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * NPW; base < cnt; base += nwarps * NPW) {
        long long idx = base + lane / G;
        bool vn = idx < cnt;
        int i = vn ? order[idx] : 0;
        const long long m = mp.of(i);
        int start = vn ? rp[i] : 0, end = vn ? rp[i + 1] : 0;
        long long si = vn ? (long long)s[i] : 0;
        PairBest b{LLONG_MIN, INT_MAX};
        for (int p = start + gl; p < end; p += G) {
            int j = col[p];
            if (j == i) continue;
            pair_consider(b, m * (long long)w[p] - NM::cross(si, (long long)s[j]), j);
        }
#pragma unroll
        for (int o = G / 2; o; o >>= 1) {
            long long osc = __shfl_xor_sync(FULL, b.sc, o);
            int oj = __shfl_xor_sync(FULL, b.j, o);
            pair_consider(b, osc, oj);
        }
        if (gl == 0 && vn) a[i] = (b.j != INT_MAX && b.sc > 0) ? b.j : i;
    }
}

template <class NM>
__global__ void __launch_bounds__(kBlockThreads) k_assign_block(const int32_t *order, int32_t cnt, const int32_t *rp,
                               const int32_t *col, const int32_t *w, const typename NM::ST *s,
                               MParam mp, int32_t *a) {
    for (long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
        int i = order[idx];
        const long long m = mp.of(i);
        long long si = (long long)s[i];
        PairBest b{LLONG_MIN, INT_MAX};
        for (int p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) {
            int j = col[p];
            if (j == i) continue;
            pair_consider(b, m * (long long)w[p] - NM::cross(si, (long long)s[j]), j);
        }
        long long dummy = 0;
        block_reduce_best(dummy, b.sc, b.j);
        if (threadIdx.x == 0) a[i] = (b.j != INT_MAX && b.sc > 0) ? b.j : i;
    }
}

__global__ void k_assign_empty(const int32_t *order, int32_t cnt, int32_t *a) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < cnt;
         idx += (long long)gridDim.x * blockDim.x)
        a[order[idx]] = order[idx];
}

// Target of every accepted node: one warp per node.
template <class NM>
__global__ void k_target(const int32_t *list, const int32_t *cnt_dev, const int32_t *rp,
                         const int32_t *col, const int32_t *w, const typename NM::ST *s, MParam mp,
                         const int32_t *root, const int32_t *best, int32_t *tgt) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int cnt = *cnt_dev;
    for (long long idx = warp; idx < cnt; idx += nwarps) {
        int i = list[idx];
        const long long m = mp.of(i);
        int want = best[i];
        long long si = (long long)s[i];
        PairBest b{LLONG_MIN, INT_MAX};
        for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
            int j = col[p];
            if (j == i || root[j] != want) continue;
            pair_consider(b, m * (long long)w[p] - NM::cross(si, (long long)s[j]), j);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            long long osc = __shfl_xor_sync(FULL, b.sc, o);
            int oj = __shfl_xor_sync(FULL, b.j, o);
            pair_consider(b, osc, oj);
        }
        // never empty: best_i is a neighbouring community; a self-assignment
        // keeps the array valid should that ever fail
        if (lane == 0) tgt[i] = (b.j != INT_MAX) ? b.j : i;
    }
}

// ---------------------------------------------------------------------------
// Own-community weight and POSITIVE's flags.
// ---------------------------------------------------------------------------
template <class NM>
__device__ __forceinline__ void own_emit(int i, int ci, long long si, long long m,
                                         const typename NM::ST *sigma, long long own,
                                         int32_t *kown, int32_t *flag) {
    kown[i] = (int32_t)own;
    long long g = m * own - NM::cross(si, (long long)sigma[ci] - si);
    if (g < 0) flag[ci] = 1;
}

template <class NM, int G>
__global__ void __launch_bounds__(256) k_own_group(const int32_t *order, int32_t cnt, const int32_t *rp,
                            const int32_t *col, const int32_t *w, const typename NM::ST *s, MParam mp,
                            const int32_t *root, const typename NM::ST *sigma, int32_t *kown,
                            int32_t *flag) {
    constexpr int NPW = 32 / G;
    const int lane = threadIdx.x & 31, gl = lane % G;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * NPW; base < cnt; base += nwarps * NPW) {
        long long idx = base + lane / G;
        bool vn = idx < cnt;
        int i = vn ? order[idx] : 0;
        const long long m = mp.of(i);
        int ci = vn ? root[i] : -1;
        long long own = 0;
        if (vn)
            for (int p = rp[i] + gl; p < rp[i + 1]; p += G) {
                int j = col[p];
                if (j != i && root[j] == ci) own += w[p];
            }
#pragma unroll
        for (int o = G / 2; o; o >>= 1) own += __shfl_xor_sync(FULL, own, o);
        if (gl == 0 && vn) own_emit<NM>(i, ci, (long long)s[i], m, sigma, own, kown, flag);
    }
}

template <class NM>
__global__ void __launch_bounds__(kBlockThreads) k_own_block(const int32_t *order, int32_t cnt, const int32_t *rp,
                            const int32_t *col, const int32_t *w, const typename NM::ST *s, MParam mp,
                            const int32_t *root, const typename NM::ST *sigma, int32_t *kown,
                            int32_t *flag) {
    for (long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
        int i = order[idx];
        const long long m = mp.of(i);
        int ci = root[i];
        long long own = 0;
        const int e = rp[i + 1];
        // eight entries per thread in flight
        for (int p0 = rp[i] + threadIdx.x; p0 < e; p0 += 8 * blockDim.x) {
            int j[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const int p = p0 + t * (int)blockDim.x;
                j[t] = p < e ? col[p] : -1;
            }
#pragma unroll
            for (int t = 0; t < 8; t++)
                if (j[t] >= 0 && j[t] != i && root[j[t]] == ci) own += w[p0 + t * (int)blockDim.x];
        }
        long long sc = LLONG_MIN;
        int cc = INT_MAX;
        block_reduce_best(own, sc, cc);
        if (threadIdx.x == 0) own_emit<NM>(i, ci, (long long)s[i], m, sigma, own, kown, flag);
    }
}

template <class NM>
__global__ void k_local_gain(int32_t n, const typename NM::ST *s, MParam mp, const int32_t *root,
                             const typename NM::ST *sigma, const int32_t *kown, long long *g) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long m = mp.of((int)i);
        long long si = (long long)s[i];
        g[i] = m * (long long)kown[i] - NM::cross(si, (long long)sigma[root[i]] - si);
    }
}

}  // namespace

template <class NM>
void local_gain_nodes(int32_t n, const typename NM::ST *s, MParam m, const int32_t *root,
                      const typename NM::ST *sigma, const int32_t *kown, long long *g,
                      cudaStream_t st) {
    if (n <= 0) return;
    k_local_gain<NM><<<grid_for(n, 256), 256, 0, st>>>(n, s, m, root, sigma, kown, g);
    SLM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
Buckets::~Buckets() {
    if (cs_tex) cudaDestroyTextureObject(cs_tex);
    for (int k = 0; k < kSide; k++) {
        if (side[k]) cudaStreamDestroy(side[k]);
        if (join[k]) cudaEventDestroy(join[k]);
    }
    if (fork) cudaEventDestroy(fork);
    for (auto &pe : pev)
        for (cudaEvent_t e : pe)
            if (e) cudaEventDestroy(e);
}

void Buckets::build(int32_t n, const int32_t *rp, cudaStream_t s) { build_list(n, nullptr, rp, s); }

void Buckets::build_list(int32_t n, const int32_t *list, const int32_t *rp, cudaStream_t s) {
    if (!fork && !one_stream) {
        for (int k = 0; k < kSide; k++) {
            SLM_CUDA(cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking));
            SLM_CUDA(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
        }
        SLM_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    }
    for (int b = 0; b <= kNumBuckets; b++) off[b] = 0;
    for (int b = 0; b <= kNumFine; b++) foff[b] = 0;
    lay_ready = false;
    order.ensure(sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s);
    if (n <= 0) return;
    DevBuf keys(sizeof(uint32_t) * n, s), keys_tmp(sizeof(uint32_t) * n, s),
        vals_tmp(sizeof(int32_t) * n, s), counts(sizeof(int32_t) * kNumFine, s);
    SLM_CUDA(cudaMemsetAsync(counts.get(), 0, counts.bytes(), s));
    k_bucket_keys<<<grid_for(n, 256), 256, 0, s>>>(n, list, rp, keys.as<uint32_t>(), order.as<int32_t>(),
                                                   counts.as<int32_t>());
    SLM_LAUNCH_CHECK();
    radix_sort_u32(keys.as<uint32_t>(), order.as<int32_t>(), keys_tmp.as<uint32_t>(),
                   vals_tmp.as<int32_t>(), n, 4, s);
    int32_t h[kNumFine];
    SLM_CUDA(cudaMemcpyAsync(h, counts.get(), sizeof h, cudaMemcpyDeviceToHost, s));
    slm::stream_sync(s);
    int32_t hc[kNumBuckets] = {0};
    for (int b = 0; b < kNumFine; b++) {
        foff[b + 1] = foff[b] + h[b];
        hc[kCoarseOf[b]] += h[b];
    }
    for (int b = 0; b < kNumBuckets; b++) off[b + 1] = off[b] + hc[b];
    // hubs: table offsets and chunk list, built on the host (hubs are few)
    nhub = off[kBucketHub + 1] - off[kBucketHub];
    nchunk = 0;
    if (nhub > 0) {
        DevBuf rows(sizeof(int2) * nhub, s);
        const int32_t *hubs = order.as<int32_t>() + off[kBucketHub];
        k_hub_rows<<<grid_for(nhub, 256), 256, 0, s>>>(nhub, hubs, rp, rows.as<int2>());
        SLM_LAUNCH_CHECK();
        std::vector<int2> hr(nhub);
        SLM_CUDA(cudaMemcpyAsync(hr.data(), rows.get(), sizeof(int2) * nhub, cudaMemcpyDeviceToHost, s));
        slm::stream_sync(s);
        std::vector<long long> hoff(nhub);
        std::vector<int32_t> hlg(nhub), tcoff(nhub + 1);
        std::vector<int4> ch;
        std::vector<int2> tch;
        long long tot = 0;
        std::vector<long long> uoff(nhub);
        long long utot = 0;
        for (int k = 0; k < nhub; k++) {
            int deg = hr[k].y - hr[k].x;
            int lg = 0;
            while ((1LL << lg) < 2LL * deg) lg++;
            hoff[k] = tot;
            hlg[k] = lg;
            tot += 1LL << lg;
            uoff[k] = utot;  // the hub's list of occupied slots holds at most deg entries
            utot += deg;
            for (int p0 = hr[k].x; p0 < hr[k].y; p0 += kHubChunk)
                ch.push_back(make_int4(k, p0, std::min(p0 + kHubChunk, hr[k].y), 0));
            tcoff[k] = (int32_t)tch.size();
            for (long long s0 = 0; s0 < deg; s0 += kHubSlice) tch.push_back(make_int2(k, (int)s0));
        }
        hub_uoff.alloc(sizeof(long long) * nhub, s);
        hub_ucnt.alloc(sizeof(int) * nhub, s);
        ulist.alloc(sizeof(int) * (utot > 0 ? utot : 1), s);
        SLM_CUDA(cudaMemcpyAsync(hub_uoff.get(), uoff.data(), sizeof(long long) * nhub, cudaMemcpyHostToDevice, s));
        SLM_CUDA(cudaMemsetAsync(hub_ucnt.get(), 0, sizeof(int) * nhub, s));
        tcoff[nhub] = (int32_t)tch.size();
        ntchunk = (int32_t)tch.size();
        tchunks.alloc(sizeof(int2) * tch.size(), s);
        tc_off.alloc(sizeof(int32_t) * (nhub + 1), s);
        part_sc.alloc(sizeof(long long) * tch.size(), s);
        part_cc.alloc(sizeof(int32_t) * tch.size(), s);
        SLM_CUDA(cudaMemcpyAsync(tchunks.get(), tch.data(), sizeof(int2) * tch.size(), cudaMemcpyHostToDevice, s));
        SLM_CUDA(cudaMemcpyAsync(tc_off.get(), tcoff.data(), sizeof(int32_t) * (nhub + 1), cudaMemcpyHostToDevice, s));
        nchunk = (int32_t)ch.size();
        hub_off.alloc(sizeof(long long) * nhub, s);
        hub_lg.alloc(sizeof(int32_t) * nhub, s);
        chunks.alloc(sizeof(int4) * ch.size(), s);
        hub_acc.alloc(sizeof(unsigned long long) * nhub, s);
        hub_own.alloc(sizeof(unsigned long long) * nhub, s);
        tslot.alloc(sizeof(unsigned long long) * tot, s);
        SLM_CUDA(cudaMemcpyAsync(hub_off.get(), hoff.data(), sizeof(long long) * nhub, cudaMemcpyHostToDevice, s));
        SLM_CUDA(cudaMemcpyAsync(hub_lg.get(), hlg.data(), sizeof(int32_t) * nhub, cudaMemcpyHostToDevice, s));
        SLM_CUDA(cudaMemcpyAsync(chunks.get(), ch.data(), sizeof(int4) * ch.size(), cudaMemcpyHostToDevice, s));
        // the tables start empty and every scan leaves them empty
        SLM_CUDA(cudaMemsetAsync(tslot.get(), 0, sizeof(unsigned long long) * tot, s));
        SLM_CUDA(cudaMemsetAsync(hub_own.get(), 0, sizeof(unsigned long long) * nhub, s));
        slm::stream_sync(s);  // host vectors go out of scope
    }
}

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per device.
template <class K> static void allow_smem(K kernel, size_t bytes, int which) {
    static std::mutex mu;
    static unsigned long long done[2] = {0, 0};  // bit d: device d set up
    int dev = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && (done[which] >> dev) & 1ull) return;
    SLM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (dev < 64) done[which] |= 1ull << dev;
}

static std::mutex g_tuning_mu;
static ScanTuning g_tuning;

ScanTuning scan_tuning() {
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    return g_tuning;
}
void set_scan_tuning(const ScanTuning &t) {
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    g_tuning = t;
}

static int blocks_for_groups(long long cnt, int nodes_per_warp, int threads = 256,
                             int per_sm = 16) {
    long long warps = (cnt + nodes_per_warp - 1) / nodes_per_warp;
    return grid_for(warps * 32, threads, kNumSMs * per_sm);
}

template <class NM>
void assign_nodes(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                  const typename NM::ST *s, MParam m, const Buckets &bk, int32_t *a, cudaStream_t st) {
    if (n <= 0) return;
    const int32_t *ord = bk.order.as<int32_t>();
    auto seg = [&](int b) { return std::make_pair(ord + bk.off[b], bk.off[b + 1] - bk.off[b]); };
    {
        auto [o, c] = seg(kBucketEmpty);
        if (c) { k_assign_empty<<<grid_for(c, 256), 256, 0, st>>>(o, c, a); SLM_LAUNCH_CHECK(); }
    }
    {
        auto [o, c] = seg(kBucketG4);
        if (c) { k_assign_group<NM, 4><<<blocks_for_groups(c, 8), 256, 0, st>>>(o, c, rp, col, w, s, m, a); SLM_LAUNCH_CHECK(); }
    }
    {
        auto [o, c] = seg(kBucketG8);
        if (c) { k_assign_group<NM, 8><<<blocks_for_groups(c, 4), 256, 0, st>>>(o, c, rp, col, w, s, m, a); SLM_LAUNCH_CHECK(); }
    }
    {
        auto [o, c] = seg(kBucketG16);
        if (c) { k_assign_group<NM, 16><<<blocks_for_groups(c, 2), 256, 0, st>>>(o, c, rp, col, w, s, m, a); SLM_LAUNCH_CHECK(); }
    }
    {
        // 17..256 edges: one warp per node, lanes stride over the row
        int c = bk.off[kBucketWarpHash + 1] - bk.off[kBucketG32];
        if (c) { k_assign_group<NM, 32><<<blocks_for_groups(c, 1), 256, 0, st>>>(ord + bk.off[kBucketG32], c, rp, col, w, s, m, a); SLM_LAUNCH_CHECK(); }
    }
    {
        int c = bk.off[kBucketHub + 1] - bk.off[kBucketBlockS];
        if (c) { k_assign_block<NM><<<grid_for(c, 1, kNumSMs * 8), kBlockThreads, 0, st>>>(ord + bk.off[kBucketBlockS], c, rp, col, w, s, m, a); SLM_LAUNCH_CHECK(); }
    }
}

template <class NM>
void scan_nodes(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                const typename NM::ST *s, MParam m, const int32_t *root,
                const typename NM::ST *sigma, const Buckets &bk, int32_t *best,
                long long *gain, int32_t *kown, unsigned long long *ncand, cudaStream_t st) {
    if (n <= 0) return;
    const int32_t *ord = bk.order.as<int32_t>();
    auto cnt = [&](int b) { return bk.off[b + 1] - bk.off[b]; };
    const ScanTuning tu = scan_tuning();
    const bool side = tu.streams > 1 && bk.fork != nullptr;
    Buckets &bl = const_cast<Buckets &>(bk);
    build_scan_layout<NM>(bl, n, rp, col, w, s, st);
    pack_community_totals<NM>(n, root, sigma, bl, st);
    // the buckets write disjoint nodes: run them side by side
    if (side) {
        SLM_CUDA(cudaEventRecord(bk.fork, st));
        for (int k = 0; k < Buckets::kSide; k++) SLM_CUDA(cudaStreamWaitEvent(bk.side[k], bk.fork, 0));
    }
    cudaStream_t s0 = st, s1 = side ? bk.side[0] : st, s2 = side ? bk.side[1] : st,
                 s3 = side ? bk.side[2] : st;
    Buckets &bt = const_cast<Buckets &>(bk);
    if (bt.prof_ms)
        for (int b = 0; b < kNumBuckets; b++)
            for (int e = 0; e < 2; e++)
                if (!bt.pev[b][e]) SLM_CUDA(cudaEventCreate(&bt.pev[b][e]));
    auto mark = [&](int b, int e, cudaStream_t so) {
        if (bt.prof_ms) SLM_CUDA(cudaEventRecord(bt.pev[b][e], so));
    };
    // the hub chain (insert, slices, decisions) is the longest: start it first
    if (bk.nhub > 0) {
        mark(kBucketHub, 0, s3);
        const int32_t *hubs = ord + bk.off[kBucketHub];
        k_hub_insert<<<grid_for(bk.nchunk, 1, kNumSMs * tu.blocks_hub), kBlockThreads, 0, s3>>>(
            bk.chunks.as<int4>(), bk.nchunk, hubs, bk.hub_off.as<long long>(), bk.hub_lg.as<int32_t>(),
            bk.hub_uoff.as<long long>(), col, w, root, bk.tslot.as<unsigned long long>(),
            bk.ulist.as<int>(), bk.hub_ucnt.as<int>(), bk.hub_own.as<unsigned long long>());
        SLM_LAUNCH_CHECK();
        k_hub_slices<NM><<<grid_for(bk.ntchunk, 1, kNumSMs * tu.blocks_hub), kBlockThreads, 0, s3>>>(
            bk.tchunks.as<int2>(), bk.ntchunk, hubs, bk.hub_off.as<long long>(),
            bk.hub_uoff.as<long long>(), bk.ulist.as<int>(), bk.hub_ucnt.as<int>(), s, m, root, sigma,
            bk.tslot.as<unsigned long long>(),
            bk.part_sc.as<long long>(), bk.part_cc.as<int32_t>());
        SLM_LAUNCH_CHECK();
        k_hub_finish<NM><<<grid_for((long long)bk.nhub * 32, 256), 256, 0, s3>>>(
            bk.nhub, hubs, bk.tc_off.as<int32_t>(), s, m, root, sigma, bk.hub_own.as<unsigned long long>(),
            bk.part_sc.as<long long>(), bk.part_cc.as<int32_t>(), bk.hub_ucnt.as<int>(), best, gain,
            kown, ncand);
        SLM_LAUNCH_CHECK();
        mark(kBucketHub, 1, s3);
    }
    // every other fine class on the layout of k_scan_fine.cu: the long
    // blocks first on their stream, the lane groups and small blocks beside
    auto run_classes = [&](int coarse, std::initializer_list<int> fines, cudaStream_t so) {
        bool any = false;
        for (int f : fines) any = any || bk.foff[f + 1] > bk.foff[f];
        if (!any) return;
        mark(coarse, 0, so);
        for (int f : fines)
            scan_fine_class<NM>(f, bk, s, m, best, gain, kown, ncand, tu, so);
        mark(coarse, 1, so);
    };
    run_classes(kBucketBlockL, {kFine4096}, s0);
    run_classes(kBucketBlockM, {kFine2048}, s0);
    run_classes(kBucketWarpHash, {kFine256, kFine128, kFine64}, s1);
    run_classes(kBucketBlockS, {kFine1024, kFine512}, s2);
    run_classes(kBucketG16, {kFine16}, s2);
    run_classes(kBucketG32, {kFine32}, s2);
    run_classes(kBucketG4, {kFine4}, s3);
    run_classes(kBucketG8, {kFine8}, s3);
    if (int c = cnt(kBucketEmpty)) {
        mark(kBucketEmpty, 0, s1);
        k_scan_empty<<<grid_for(c, 256), 256, 0, s1>>>(ord + bk.off[kBucketEmpty], c, root, best, gain, kown);
        SLM_LAUNCH_CHECK();
        mark(kBucketEmpty, 1, s1);
    }
    if (side)
        for (int k = 0; k < Buckets::kSide; k++) {
            SLM_CUDA(cudaEventRecord(bk.join[k], bk.side[k]));
            SLM_CUDA(cudaStreamWaitEvent(st, bk.join[k], 0));
        }
    if (bt.prof_ms) {
        stream_sync(st);
        for (int b = 0; b < kNumBuckets; b++) {
            if (b != kBucketHub && bk.off[b + 1] == bk.off[b]) continue;
            if (b == kBucketHub && bk.nhub == 0) continue;
            float t = 0;
            SLM_CUDA(cudaEventElapsedTime(&t, bt.pev[b][0], bt.pev[b][1]));
            bt.prof_ms[b] += t;
        }
    }
}

template <class NM>
void own_weight_nodes(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                      const typename NM::ST *s, MParam m, const int32_t *root,
                      const typename NM::ST *sigma, const Buckets &bk, int32_t *kown,
                      int32_t *flag, cudaStream_t st) {
    if (n <= 0) return;
    const int32_t *ord = bk.order.as<int32_t>();
    // the classes write disjoint nodes: run them side by side, as the scan's
    const bool side = scan_tuning().streams > 1 && bk.fork != nullptr;
    if (side) {
        SLM_CUDA(cudaEventRecord(bk.fork, st));
        for (int k = 0; k < Buckets::kSide; k++) SLM_CUDA(cudaStreamWaitEvent(bk.side[k], bk.fork, 0));
    }
    cudaStream_t s1 = side ? bk.side[0] : st, s2 = side ? bk.side[1] : st, s3 = side ? bk.side[2] : st;
    // isolated nodes: own weight 0, local gain 0 (never flagged)
    int c0 = bk.off[kBucketEmpty + 1] - bk.off[kBucketEmpty];
    if (c0) {
        k_own_group<NM, 4><<<blocks_for_groups(c0, 8), 256, 0, s3>>>(ord, c0, rp, col, w, s, m, root, sigma, kown, flag);
        SLM_LAUNCH_CHECK();
    }
    if (int c = bk.off[kBucketG4 + 1] - bk.off[kBucketG4]) {
        k_own_group<NM, 4><<<blocks_for_groups(c, 8), 256, 0, s3>>>(ord + bk.off[kBucketG4], c, rp, col, w, s, m, root, sigma, kown, flag);
        SLM_LAUNCH_CHECK();
    }
    if (int c = bk.off[kBucketG8 + 1] - bk.off[kBucketG8]) {
        k_own_group<NM, 8><<<blocks_for_groups(c, 4), 256, 0, s3>>>(ord + bk.off[kBucketG8], c, rp, col, w, s, m, root, sigma, kown, flag);
        SLM_LAUNCH_CHECK();
    }
    if (int c = bk.off[kBucketG16 + 1] - bk.off[kBucketG16]) {
        k_own_group<NM, 16><<<blocks_for_groups(c, 2), 256, 0, s2>>>(ord + bk.off[kBucketG16], c, rp, col, w, s, m, root, sigma, kown, flag);
        SLM_LAUNCH_CHECK();
    }
    if (int c = bk.off[kBucketWarpHash + 1] - bk.off[kBucketG32]) {
        k_own_group<NM, 32><<<blocks_for_groups(c, 1), 256, 0, s2>>>(ord + bk.off[kBucketG32], c, rp, col, w, s, m, root, sigma, kown, flag);
        SLM_LAUNCH_CHECK();
    }
    if (int c = bk.off[kBucketBlockL + 1] - bk.off[kBucketBlockS]) {
        k_own_block<NM><<<grid_for(c, 1, kNumSMs * 8), kBlockThreads, 0, st>>>(ord + bk.off[kBucketBlockS], c, rp, col, w, s, m, root, sigma, kown, flag);
        SLM_LAUNCH_CHECK();
    }
    if (bk.nhub > 0) {
        const int32_t *hubs = ord + bk.off[kBucketHub];
        SLM_CUDA(cudaMemsetAsync(bk.hub_acc.get(), 0, sizeof(unsigned long long) * bk.nhub, s1));
        k_own_hub_chunk<<<grid_for(bk.nchunk, 1, kNumSMs * 8), kBlockThreads, 0, s1>>>(
            bk.chunks.as<int4>(), bk.nchunk, hubs, col, w, root, bk.hub_acc.as<unsigned long long>());
        SLM_LAUNCH_CHECK();
        k_own_hub_finish<NM><<<grid_for(bk.nhub, 256), 256, 0, s1>>>(bk.nhub, hubs, s, m, root, sigma,
                                                               bk.hub_acc.as<unsigned long long>(), kown, flag);
        SLM_LAUNCH_CHECK();
    }
    if (side)
        for (int k = 0; k < Buckets::kSide; k++) {
            SLM_CUDA(cudaEventRecord(bk.join[k], bk.side[k]));
            SLM_CUDA(cudaStreamWaitEvent(st, bk.join[k], 0));
        }
}

template <class NM>
void target_nodes(const int32_t *list, const int32_t *cnt_dev, int32_t max_cnt, const int32_t *rp,
                  const int32_t *col, const int32_t *w, const typename NM::ST *s, MParam m,
                  const int32_t *root, const int32_t *best, int32_t *tgt, cudaStream_t st) {
    if (max_cnt <= 0) return;
    k_target<NM><<<grid_for((long long)max_cnt * 32, 256, kNumSMs * 16), 256, 0, st>>>(
        list, cnt_dev, rp, col, w, s, m, root, best, tgt);
    SLM_LAUNCH_CHECK();
}

// the two null models (undirected and directed graphs)
#define SLM_SCAN_INSTANTIATE(NM)                                                                   \
    template void assign_nodes<NM>(int32_t, const int32_t *, const int32_t *, const int32_t *,    \
                                   const NM::ST *, MParam, const Buckets &, int32_t *,            \
                                   cudaStream_t);                                                 \
    template void scan_nodes<NM>(int32_t, const int32_t *, const int32_t *, const int32_t *,      \
                                 const NM::ST *, MParam, const int32_t *, const NM::ST *,         \
                                 const Buckets &, int32_t *, long long *, int32_t *,              \
                                 unsigned long long *, cudaStream_t);                             \
    template void own_weight_nodes<NM>(int32_t, const int32_t *, const int32_t *, const int32_t *, \
                                       const NM::ST *, MParam, const int32_t *, const NM::ST *,   \
                                       const Buckets &, int32_t *, int32_t *, cudaStream_t);      \
    template void local_gain_nodes<NM>(int32_t, const NM::ST *, MParam, const int32_t *,          \
                                       const NM::ST *, const int32_t *, long long *, cudaStream_t); \
    template void target_nodes<NM>(const int32_t *, const int32_t *, int32_t, const int32_t *,    \
                                   const int32_t *, const int32_t *, const NM::ST *, MParam,      \
                                   const int32_t *, const int32_t *, int32_t *, cudaStream_t);
SLM_SCAN_INSTANTIATE(NMSym)
SLM_SCAN_INSTANTIATE(NMDir)
#undef SLM_SCAN_INSTANTIATE

}  // namespace slm
