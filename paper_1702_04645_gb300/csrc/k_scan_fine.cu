// k_scan_fine.cu -- the MAXIMAL scan (Section 3.4, Algorithm MAXIMAL: for
// every node i the weight k_{i,C} to each neighbouring community C, and the
// best C != c_i by the exact score m_w k_{i,C} - s_i Sigma_C of Section 2.4,
// ties to the smallest name) for every node of degree 1..4096; rows above
// 4096 entries (hubs) go through the global-table kernels of k_scan.cu.
//
// Layout (built once per level, on the first scan after Buckets::build):
//   ent[e]  int2 (column, weight) -- the rows of the bucketed nodes, copied in
//           bucket order, so every fine class reads one contiguous stream
//           with one 8-byte load per entry;
//   nrec[k] int4 (node, first entry in ent, degree, s_i) per bucketed node.
// Per scan:
//   cs[j]   int2 (root_j, Sigma_{root_j}) -- one 8-byte gather per entry gives
//           a neighbour's community and that community's total.
//
// Shapes, one per fine degree class: one thread per node (1..8 entries:
// communities grouped in registers), 4/8/16/32 lanes per node (9..256), one
// block per node (257..4096), each lane holding at most EPL entries.  Both
// table shapes accumulate in a shared-memory open-addressing table with at
// least twice as many slots as the row has entries, and the lane that claims
// a slot keeps the slot, the community and its total in registers and decides
// it after the inserts, so nothing scans the table or lists its slots:
//   * lane groups: 64-bit slots (C + 1) << 32 | k_{i,C} (0 = empty); a new
//     community costs one CAS, a repeated one a CAS and an add, and the
//     claimer empties its slot after deciding it;
//   * blocks: 32-bit keys C + 1 and a separate weight word; every lane's
//     home-slot CASes are issued before any result is looked at, the claimer
//     keeps the first weight in a register, a repeated community adds to the
//     weight word without a return value, and the used part of the table is
//     cleared with 16-byte stores.
// (Measured per class on the R-MAT scale-20 graph, each form is the faster
// one for its shape.)  The weight to the node's own community is summed in
// registers instead (often most of a row: every lane would hit one slot).
// The (community, total) gathers go through the texture path (a separate data
// pipe from the shared-memory table's), with plain loads when the array
// exceeds a 1D texture's width.
// Every comparison is (score desc, name asc) and every sum an integer
// atomic: the result does not depend on scheduling.
#include <atomic>
#include <climits>

#include "slm_internal.cuh"

namespace slm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ bool better(long long sc, int c, long long bsc, int bc) {
    return sc > bsc || (sc == bsc && c < bc);
}

// ---------------------------------------------------------------------------
// Layout
// ---------------------------------------------------------------------------
// degree of every bucketed node that gets a copied row (hubs keep the CSR)
__global__ void k_lay_deg(int32_t cnt, int32_t copy_end, const int32_t *order, const int32_t *rp,
                          int32_t *deg) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < cnt;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = order[k];
        deg[k] = k < copy_end ? rp[i + 1] - rp[i] : 0;
    }
}

// one warp per bucketed node: its record, and its row copied into ent
template <class NM>
__global__ void k_lay_fill(int32_t cnt, int32_t copy_end, const int32_t *order, const int32_t *rp,
                           const int32_t *col, const int32_t *w, const typename NM::ST *s,
                           const int32_t *est, int4 *nrec, int2 *ent) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < cnt; k += nwarps) {
        const int i = order[k];
        const int start = rp[i], d = rp[i + 1] - start;
        const int e0 = est[k];
        // a directed graph's packed strength does not fit: the scan reads it from s
        if (lane == 0) nrec[k] = make_int4(i, e0, d, NM::kDirected ? 0 : (int)s[i]);
        if (k < copy_end)
            for (int p = lane; p < d; p += 32) ent[e0 + p] = make_int2(col[start + p], w[start + p]);
    }
}

// cs[v] = (root_v, Sigma_{root_v}) for every node of the graph: int2 for an
// undirected graph; int4 (root, packed total low and high words, 0) for a
// directed one
__global__ void k_pack_cs(int32_t n, const int32_t *root, const int32_t *sigma, int2 *cs) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int c = root[v];
        cs[v] = make_int2(c, sigma[c]);
    }
}
__global__ void k_pack_cs(int32_t n, const int32_t *root, const unsigned long long *sigma,
                          int4 *cs) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int c = root[v];
        const unsigned long long t = sigma[c];
        cs[v] = make_int4(c, (int)(unsigned)(t & 0xffffffffull), (int)(unsigned)(t >> 32), 0);
    }
}

template <class NM> struct CsOf { using T = int2; };
template <> struct CsOf<NMDir> { using T = int4; };

}  // namespace

template <class NM>
void build_scan_layout(Buckets &bk, int32_t n, const int32_t *rp, const int32_t *col,
                       const int32_t *w, const typename NM::ST *s, cudaStream_t st) {
    using CS = typename CsOf<NM>::T;
    const void *src[4] = {rp, col, w, s};
    bool same = bk.lay_ready;
    for (int k = 0; k < 4; k++) same = same && bk.lay_src[k] == src[k];
    const void *cs_before = bk.csbuf().get();
    bk.csbuf().ensure(sizeof(CS) * (size_t)(n > 0 ? n : 1), st);
    if (bk.csbuf().get() != cs_before || !bk.cs_tex || bk.cs_elem != (int)sizeof(CS)) {
        if (bk.cs_tex) cudaDestroyTextureObject(bk.cs_tex);
        bk.cs_tex = 0;
        int dev = 0, maxw = 0;
        SLM_CUDA(cudaGetDevice(&dev));
        SLM_CUDA(cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, dev));
        const size_t elems = bk.csbuf().bytes() / sizeof(CS);
        if (elems <= (size_t)maxw) {
            cudaResourceDesc rd{};
            rd.resType = cudaResourceTypeLinear;
            rd.res.linear.devPtr = bk.csbuf().get();
            rd.res.linear.desc = cudaCreateChannelDesc<CS>();
            rd.res.linear.sizeInBytes = elems * sizeof(CS);
            cudaTextureDesc td{};
            td.readMode = cudaReadModeElementType;
            SLM_CUDA(cudaCreateTextureObject(&bk.cs_tex, &rd, &td, nullptr));
            bk.cs_elem = (int)sizeof(CS);
        }
    }
    if (same) return;
    const int32_t cnt = bk.off[kNumBuckets];
    const int32_t copy_end = bk.foff[kFineHub];  // hubs sit at the end of the order
    bk.nrec.ensure(sizeof(int4) * (size_t)(cnt > 0 ? cnt : 1), st);
    if (cnt > 0) {
        DevBuf deg(sizeof(int32_t) * (size_t)cnt, st), est(sizeof(int32_t) * (size_t)cnt, st),
            tot(sizeof(int32_t), st);
        const int32_t *ord = bk.order.as<int32_t>();
        k_lay_deg<<<grid_for(cnt, 256), 256, 0, st>>>(cnt, copy_end, ord, rp, deg.as<int32_t>());
        SLM_LAUNCH_CHECK();
        exclusive_scan_i32(deg.as<int32_t>(), est.as<int32_t>(), cnt, tot.as<int32_t>(), st);
        int32_t ne = 0;
        SLM_CUDA(cudaMemcpyAsync(&ne, tot.get(), sizeof ne, cudaMemcpyDeviceToHost, st));
        stream_sync(st);
        bk.ent.ensure(sizeof(int2) * (size_t)(ne > 0 ? ne : 1), st);
        k_lay_fill<NM><<<grid_for((long long)cnt * 32, 256), 256, 0, st>>>(
            cnt, copy_end, ord, rp, col, w, s, est.as<int32_t>(), bk.nrec.as<int4>(), bk.ent.as<int2>());
        SLM_LAUNCH_CHECK();
    }
    for (int k = 0; k < 4; k++) bk.lay_src[k] = src[k];
    bk.lay_ready = true;
}

template <class NM>
void pack_community_totals(int32_t n, const int32_t *root, const typename NM::ST *sigma,
                           Buckets &bk, cudaStream_t st) {
    if (n <= 0) return;
    k_pack_cs<<<grid_for(n, 256), 256, 0, st>>>(n, root, sigma,
                                                 bk.csbuf().as<typename CsOf<NM>::T>());
    SLM_LAUNCH_CHECK();
}

namespace {

template <class NM>
struct FsArgs {
    const int4 *nrec;  // records of this fine class (offset into the bucket order)
    int32_t cnt;       // nodes of this fine class
    const int2 *ent;
    const typename CsOf<NM>::T *cs;
    cudaTextureObject_t cs_tex;  // the same array through the texture path (0: none)
    const typename NM::ST *s;    // node strengths (read only for a directed graph)
    MParam mp;
    int32_t *best;
    long long *gain;
    int32_t *kown;
    unsigned long long *ncand;
};

// The decision of one node (Algorithm MAXIMAL): stay unless the best other
// community beats the own one by a positive amount.
template <class NM>
__device__ __forceinline__ void fs_emit(const FsArgs<NM> &A, int i, int ci, long long sig_ci,
                                        long long si, long long m, long long own, long long bsc,
                                        int bc, unsigned &cand) {
    const long long g = m * own - NM::cross(si, sig_ci - si);
    const long long gn = bc != INT_MAX ? bsc - g : 0;
    if (bc != INT_MAX && gn > 0) {
        A.best[i] = bc;
        A.gain[i] = gn;
        cand++;
    } else {
        A.best[i] = ci;
        A.gain[i] = 0;
    }
    A.kown[i] = (int32_t)own;
}

__device__ __forceinline__ void fs_count(unsigned long long *ctr, unsigned v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, (unsigned long long)v);
}

// (community, total) of node j: through the texture pipe when the array has a
// texture object (the random gathers then leave the load/store pipe to the
// shared-memory table), else a plain load
__device__ __forceinline__ void cs_at(const FsArgs<NMSym> &A, int j, int &c, int &sig) {
    const int2 q = A.cs_tex ? tex1Dfetch<int2>(A.cs_tex, j) : A.cs[j];
    c = q.x;
    sig = q.y;
}
__device__ __forceinline__ void cs_at(const FsArgs<NMDir> &A, int j, int &c, long long &sig) {
    const int4 q = A.cs_tex ? tex1Dfetch<int4>(A.cs_tex, j) : A.cs[j];
    c = q.x;
    sig = (long long)(((unsigned long long)(unsigned)q.z << 32) | (unsigned long long)(unsigned)q.y);
}

// strength of the node of record r
__device__ __forceinline__ int node_s(const FsArgs<NMSym> &, const int4 &r) { return r.w; }
__device__ __forceinline__ long long node_s(const FsArgs<NMDir> &A, const int4 &r) {
    return (long long)A.s[r.x];
}

__device__ __forceinline__ unsigned slot_of(int c, int lg) {
    return ((unsigned)c * 2654435761u) >> (32 - lg);
}

// Insert the E entries (c[t] >= 0: community, wv[t]: weight) of one lane into
// a table of 2^lg slots: K[h] holds C + 1 (0 = empty), W[h] the weight added
// by lanes that found C already there.  Every home-slot CAS is issued before
// any result is looked at, so their latencies overlap.  On return cl[t] is
// the slot this lane claimed for entry t (it keeps wv[t] as that slot's first
// weight), or -1.
template <int E>
__device__ __forceinline__ void table_insert(unsigned *K, unsigned *W, int lg, const int (&c)[E],
                                             const int (&wv)[E], int (&cl)[E]) {
    const unsigned mask = (1u << lg) - 1u;
    unsigned h[E], old[E];
#pragma unroll
    for (int t = 0; t < E; t++) {
        h[t] = c[t] >= 0 ? slot_of(c[t], lg) : 0u;
        old[t] = c[t] >= 0 ? atomicCAS(&K[h[t]], 0u, (unsigned)c[t] + 1u) : 1u;
    }
#pragma unroll
    for (int t = 0; t < E; t++) {
        cl[t] = -1;
        if (c[t] < 0) continue;
        const unsigned key = (unsigned)c[t] + 1u;
        unsigned o = old[t], hh = h[t];
        for (;;) {
            if (o == 0u) { cl[t] = (int)hh; break; }
            if (o == key) { atomicAdd(&W[hh], (unsigned)wv[t]); break; }
            hh = (hh + 1) & mask;
            o = atomicCAS(&K[hh], 0u, key);
        }
    }
}

// Add weight wv to community c in a table of 2^lg 64-bit slots; returns the
// slot when this call claimed it, -1 when the community was already there.
__device__ __forceinline__ int table_add(unsigned long long *T, int lg, int c, int wv) {
    const unsigned long long key = (unsigned long long)(unsigned)(c + 1) << 32;
    unsigned h = slot_of(c, lg);
    const unsigned mask = (1u << lg) - 1u;
    for (;;) {
        const unsigned long long old = atomicCAS(&T[h], 0ull, key | (unsigned)wv);
        if (old == 0ull) return (int)h;
        if ((old >> 32) == (unsigned long long)(unsigned)(c + 1)) {
            atomicAdd(&T[h], (unsigned long long)(unsigned)wv);
            return -1;
        }
        h = (h + 1) & mask;
    }
}

// Zero slots [0, 2^lg) of K and W with 16-byte stores by `nthr` threads
// (rank `r`); 2^lg is a multiple of 4.
__device__ __forceinline__ void table_clear(unsigned *K, unsigned *W, int lg, int r, int nthr) {
    const int q = (1 << lg) >> 2;
    uint4 *K4 = reinterpret_cast<uint4 *>(K), *W4 = reinterpret_cast<uint4 *>(W);
    for (int k = r; k < q; k += nthr) {
        K4[k] = make_uint4(0u, 0u, 0u, 0u);
        W4[k] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// log2 of the table a row of d entries uses: at least 2 d slots, at least 4
__device__ __forceinline__ int table_lg(int d) {
    int lg = 2;
    while ((1 << lg) < 2 * d) lg++;
    return lg;
}

// ---------------------------------------------------------------------------
// One thread per node, at most D entries: communities grouped in registers.
// ---------------------------------------------------------------------------
template <class NM, int D>
__global__ void __launch_bounds__(256) k_fs_thread(FsArgs<NM> A) {
    unsigned cand = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < A.cnt;
         k += (long long)gridDim.x * blockDim.x) {
        const int4 r = A.nrec[k];
        const int i = r.x, e0 = r.y, d = r.z;
        const typename NM::V si = node_s(A, r);
        int me_c;
        typename NM::V me_s;
        cs_at(A, i, me_c, me_s);
        const long long m = A.mp.of(i);
        int c[D], wv[D];
        typename NM::V sg[D];
#pragma unroll
        for (int t = 0; t < D; t++) {
            const int2 e = t < d ? A.ent[e0 + t] : make_int2(i, 0);
            c[t] = e.x;
            wv[t] = e.y;
        }
#pragma unroll
        for (int t = 0; t < D; t++) {
            if (c[t] != i) {
                cs_at(A, c[t], c[t], sg[t]);
            } else {
                c[t] = -1;  // the node's own self-loop, or a slot past the row
                sg[t] = 0;
            }
        }
        long long own = 0, bsc = LLONG_MIN;
        int bc = INT_MAX;
#pragma unroll
        for (int t = 0; t < D; t++) {
            if (c[t] < 0) continue;
            bool first = true;
#pragma unroll
            for (int u = 0; u < t; u++) first = first && c[u] != c[t];
            if (!first) continue;
            long long k_ic = 0;
#pragma unroll
            for (int u = t; u < D; u++) k_ic += c[u] == c[t] ? wv[u] : 0;
            if (c[t] == me_c) {
                own = k_ic;
            } else {
                const long long x = m * k_ic - NM::cross(si, sg[t]);
                if (better(x, c[t], bsc, bc)) { bsc = x; bc = c[t]; }
            }
        }
        fs_emit<NM>(A, i, me_c, me_s, si, m, own, bsc, bc, cand);
    }
    fs_count(A.ncand, cand);
}

// ---------------------------------------------------------------------------
// L lanes per node (32 / L nodes per warp), at most EPL entries per lane, one
// table of 2 L EPL slots per node in shared memory.
// ---------------------------------------------------------------------------
constexpr int kFsWarps = 8;  // warps per block of the lane-group shape
template <class NM, int L, int EPL>
__device__ __forceinline__ void fs_lanes_body(const FsArgs<NM> &A) {
    constexpr int NPW = 32 / L;
    constexpr int CAP = 2 * L * EPL;
    constexpr int LG = __builtin_ctz(CAP);
    static_assert((CAP & (CAP - 1)) == 0, "table size must be a power of two");
    __shared__ unsigned long long tab[kFsWarps][NPW * CAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / L, gl = lane % L;
    unsigned long long *T = tab[wib] + grp * CAP;
    for (int k = lane; k < NPW * CAP; k += 32) tab[wib][k] = 0ull;
    __syncwarp();
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned cand = 0;
    for (long long base = warp * NPW; base < A.cnt; base += nwarps * NPW) {
        const long long k = base + grp;
        const bool valid = k < A.cnt;
        const int4 r = valid ? A.nrec[k] : make_int4(0, 0, 0, 0);
        const int i = r.x, e0 = r.y, d = r.z;
        const typename NM::V si = valid ? node_s(A, r) : 0;
        int c[EPL], wv[EPL], cl[EPL];
        typename NM::V sg[EPL];
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            const int p = gl + t * L;
            const int2 e = p < d ? A.ent[e0 + p] : make_int2(i, 0);
            c[t] = e.x;
            wv[t] = e.y;
        }
        int me_c = -1;
        typename NM::V me_s = 0;
        if (valid) cs_at(A, i, me_c, me_s);
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            if (c[t] != i) cs_at(A, c[t], c[t], sg[t]);
            else c[t] = -1;
        }
        // weight to the own community is summed in registers: it never
        // enters the table, where all its entries would hit one slot
        long long own = 0;
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            if (c[t] == me_c) own += wv[t];
            cl[t] = (c[t] >= 0 && c[t] != me_c) ? table_add(T, LG, c[t], wv[t]) : -1;
        }
        __syncwarp();
        const long long m = A.mp.of(i);
        long long bsc = LLONG_MIN;
        int bc = INT_MAX;
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            if (cl[t] < 0) continue;
            const long long k_ic = (long long)(unsigned)T[cl[t]];
            T[cl[t]] = 0ull;  // empty again for the next node
            const long long x = m * k_ic - NM::cross(si, sg[t]);
            if (better(x, c[t], bsc, bc)) { bsc = x; bc = c[t]; }
        }
#pragma unroll
        for (int o = L / 2; o; o >>= 1) {
            own += __shfl_xor_sync(FULL, own, o);
            const long long osc = __shfl_xor_sync(FULL, bsc, o);
            const int occ = __shfl_xor_sync(FULL, bc, o);
            if (better(osc, occ, bsc, bc)) { bsc = osc; bc = occ; }
        }
        if (gl == 0 && valid) fs_emit<NM>(A, i, me_c, me_s, si, m, own, bsc, bc, cand);
        __syncwarp();
    }
    fs_count(A.ncand, cand);
}

// The undirected kernels are compiled for SLM_FS_LANES_MIN_BLOCKS resident
// blocks per SM: 4 holds the 8-entry shape (32 lanes) at 64 registers without
// spills, where it would take 74 and fit three blocks.  The directed records
// are twice as wide and would spill at 64 registers, so the directed kernels
// keep the compiler's own choice (no minimum).
#ifndef SLM_FS_LANES_MIN_BLOCKS
#define SLM_FS_LANES_MIN_BLOCKS 4
#endif
template <class NM, int L, int EPL>
__global__ void __launch_bounds__(kFsWarps * 32, SLM_FS_LANES_MIN_BLOCKS) k_fs_lanes(FsArgs<NM> A) {
    fs_lanes_body<NM, L, EPL>(A);
}
template <class NM, int L, int EPL>
__global__ void __launch_bounds__(kFsWarps * 32) k_fs_lanes_wide(FsArgs<NM> A) {
    fs_lanes_body<NM, L, EPL>(A);
}
template <class NM, int L, int EPL>
constexpr auto lanes_kernel() {
    if constexpr (NM::kDirected) return &k_fs_lanes_wide<NM, L, EPL>;
    else return &k_fs_lanes<NM, L, EPL>;
}

// ---------------------------------------------------------------------------
// One block of T threads per node, at most EPL entries per thread, one table
// of 2 T EPL slots in dynamic shared memory.  The next node's record and
// entries are loaded while the current one is decided.
// ---------------------------------------------------------------------------
template <int T, int EPL>
constexpr size_t fs_block_smem() {
    return 2 * sizeof(unsigned) * 2 * T * EPL;
}

template <class NM, int T, int EPL>
__global__ void __launch_bounds__(T) k_fs_block(FsArgs<NM> A) {
    constexpr int CAP = 2 * T * EPL;
    constexpr int NW = T / 32;
    extern __shared__ __align__(16) unsigned tabd[];
    unsigned *K = tabd, *W = tabd + CAP;
    __shared__ long long r_own[NW], r_sc[NW];
    __shared__ int r_cc[NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = tid; k < 2 * CAP; k += T) tabd[k] = 0u;
    __syncthreads();
    unsigned cand = 0;
    long long k = blockIdx.x;
    int4 r = k < A.cnt ? A.nrec[k] : make_int4(0, 0, 0, 0);
    int2 pe[EPL];
#pragma unroll
    for (int t = 0; t < EPL; t++) {
        const int p = tid + t * T;
        pe[t] = p < r.z ? A.ent[r.y + p] : make_int2(r.x, 0);
    }
    for (; k < A.cnt; k += gridDim.x) {
        const int i = r.x;
        const typename NM::V si = node_s(A, r);
        const int lg = table_lg(r.z);
        int me_c;
        typename NM::V me_s;
        cs_at(A, i, me_c, me_s);
        int c[EPL], wv[EPL], cl[EPL], ck[EPL];
        typename NM::V sg[EPL];
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            wv[t] = pe[t].y;
            if (pe[t].x != i) cs_at(A, pe[t].x, c[t], sg[t]);
            else c[t] = -1;
        }
        long long own = 0;  // the own community stays out of the table, as above
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            if (c[t] == me_c) own += wv[t];
            ck[t] = (c[t] >= 0 && c[t] != me_c) ? c[t] : -1;
        }
        table_insert<EPL>(K, W, lg, ck, wv, cl);
        // the next node's entries are in flight while this one is decided
        const long long kn = k + gridDim.x;
        const int4 rn = kn < A.cnt ? A.nrec[kn] : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            const int p = tid + t * T;
            pe[t] = p < rn.z ? A.ent[rn.y + p] : make_int2(rn.x, 0);
        }
        __syncthreads();
        const long long m = A.mp.of(i);
        long long bsc = LLONG_MIN;
        int bc = INT_MAX;
#pragma unroll
        for (int t = 0; t < EPL; t++) {
            if (cl[t] < 0) continue;
            const long long k_ic = (long long)wv[t] + (long long)W[cl[t]];
            const long long x = m * k_ic - NM::cross(si, sg[t]);
            if (better(x, c[t], bsc, bc)) { bsc = x; bc = c[t]; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            own += __shfl_xor_sync(FULL, own, o);
            const long long osc = __shfl_xor_sync(FULL, bsc, o);
            const int occ = __shfl_xor_sync(FULL, bc, o);
            if (better(osc, occ, bsc, bc)) { bsc = osc; bc = occ; }
        }
        if (lane == 0) { r_own[wid] = own; r_sc[wid] = bsc; r_cc[wid] = bc; }
        __syncthreads();                 // every thread has read its slots
        table_clear(K, W, lg, tid, T);   // empty again for the next node
        if (wid == 0) {
            own = lane < NW ? r_own[lane] : 0;
            bsc = lane < NW ? r_sc[lane] : LLONG_MIN;
            bc = lane < NW ? r_cc[lane] : INT_MAX;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                own += __shfl_xor_sync(FULL, own, o);
                const long long osc = __shfl_xor_sync(FULL, bsc, o);
                const int occ = __shfl_xor_sync(FULL, bc, o);
                if (better(osc, occ, bsc, bc)) { bsc = osc; bc = occ; }
            }
            if (lane == 0) fs_emit<NM>(A, i, me_c, me_s, si, m, own, bsc, bc, cand);
        }
        __syncthreads();  // the table is empty and r_* are free for the next node
        r = rn;
    }
    if (tid == 0 && cand) atomicAdd(A.ncand, (unsigned long long)cand);
}

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per device.
template <class K> void allow_smem(K kernel, size_t bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load() & bit)) return;
    SLM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (bit) done.fetch_or(bit);
}

int fs_grid(long long units, int per_block, int per_sm) {
    return grid_for((units + per_block - 1) / per_block, 1, kNumSMs * per_sm);
}

}  // namespace

// Launch the scan of fine class f on stream so.
template <class NM>
void scan_fine_class(int f, const Buckets &bk, const typename NM::ST *s, MParam mp, int32_t *best,
                     long long *gain, int32_t *kown, unsigned long long *ncand,
                     const ScanTuning &tu, cudaStream_t so) {
    FsArgs<NM> A;
    A.nrec = bk.nrec.as<int4>() + bk.foff[f];
    A.cnt = bk.foff[f + 1] - bk.foff[f];
    A.ent = bk.ent.as<int2>();
    A.cs = bk.csbuf().as<typename CsOf<NM>::T>();
    A.cs_tex = bk.cs_tex;
    A.s = s;
    A.mp = mp;
    A.best = best;
    A.gain = gain;
    A.kown = kown;
    A.ncand = ncand;
    if (A.cnt <= 0) return;
    const bool alt = (tu.shape_alt >> (f - 1)) & 1;
    // lane groups of L lanes, EPL entries per lane: 32 / L nodes per warp
    auto lanes = [&](auto kernel, int L, int per_sm) {
        kernel<<<fs_grid(A.cnt, kFsWarps * (32 / L), per_sm), kFsWarps * 32, 0, so>>>(A);
    };
    // one block of T threads per node; tables above 48 KB are opted in once per device
    auto block = [&](auto kernel, int T, size_t smem, std::atomic<unsigned long long> &done,
                     int per_sm) {
        if (smem > 48 * 1024) allow_smem(kernel, smem, done);
        kernel<<<fs_grid(A.cnt, 1, per_sm), T, smem, so>>>(A);
    };
    static std::atomic<unsigned long long> d1{0}, d2{0};
    switch (f) {
    case kFine4:
        if (alt) lanes(lanes_kernel<NM, 4, 1>(), 4, tu.blocks_group);
        else k_fs_thread<NM, 4><<<fs_grid(A.cnt, 256, tu.blocks_group), 256, 0, so>>>(A);
        break;
    case kFine8:
        if (alt) lanes(lanes_kernel<NM, 8, 1>(), 8, tu.blocks_group);
        else k_fs_thread<NM, 8><<<fs_grid(A.cnt, 256, tu.blocks_group), 256, 0, so>>>(A);
        break;
    case kFine16:
        if (alt) lanes(lanes_kernel<NM, 8, 2>(), 8, tu.blocks_group);
        else lanes(lanes_kernel<NM, 4, 4>(), 4, tu.blocks_group);
        break;
    case kFine32:
        if (alt) lanes(lanes_kernel<NM, 16, 2>(), 16, tu.blocks_group);
        else lanes(lanes_kernel<NM, 8, 4>(), 8, tu.blocks_group);
        break;
    case kFine64:
        if (alt) lanes(lanes_kernel<NM, 32, 2>(), 32, tu.blocks_warp);
        else lanes(lanes_kernel<NM, 16, 4>(), 16, tu.blocks_warp);
        break;
    case kFine128:
        if (alt) block(k_fs_block<NM, 64, 2>, 64, fs_block_smem<64, 2>(), d1, 4 * tu.blocks_warp);
        else lanes(lanes_kernel<NM, 32, 4>(), 32, tu.blocks_warp);
        break;
    case kFine256:
        if (alt) block(k_fs_block<NM, 64, 4>, 64, fs_block_smem<64, 4>(), d1, 4 * tu.blocks_warp);
        else lanes(lanes_kernel<NM, 32, 8>(), 32, tu.blocks_warp);
        break;
    case kFine512:
        if (alt) block(k_fs_block<NM, 256, 2>, 256, fs_block_smem<256, 2>(), d1, tu.blocks_small);
        else block(k_fs_block<NM, 128, 4>, 128, fs_block_smem<128, 4>(), d1, 2 * tu.blocks_small);
        break;
    case kFine1024:
        if (alt) block(k_fs_block<NM, 512, 2>, 512, fs_block_smem<512, 2>(), d1, tu.blocks_small);
        else block(k_fs_block<NM, 256, 4>, 256, fs_block_smem<256, 4>(), d1, tu.blocks_small);
        break;
    case kFine2048:
        if (alt) block(k_fs_block<NM, 512, 4>, 512, fs_block_smem<512, 4>(), d1, tu.blocks_mid);
        else block(k_fs_block<NM, 256, 8>, 256, fs_block_smem<256, 8>(), d1, tu.blocks_mid);
        break;
    case kFine4096:
        if (alt) block(k_fs_block<NM, 1024, 4>, 1024, fs_block_smem<1024, 4>(), d2, tu.blocks_large);
        else block(k_fs_block<NM, 512, 8>, 512, fs_block_smem<512, 8>(), d1, tu.blocks_large);
        break;
    default:
        return;
    }
    SLM_LAUNCH_CHECK();
}

#define SLM_FINE_INSTANTIATE(NM)                                                                \
    template void build_scan_layout<NM>(Buckets &, int32_t, const int32_t *, const int32_t *,    \
                                        const int32_t *, const NM::ST *, cudaStream_t);          \
    template void pack_community_totals<NM>(int32_t, const int32_t *, const NM::ST *, Buckets &, \
                                            cudaStream_t);                                       \
    template void scan_fine_class<NM>(int, const Buckets &, const NM::ST *, MParam, int32_t *,   \
                                      long long *, int32_t *, unsigned long long *,              \
                                      const ScanTuning &, cudaStream_t);
SLM_FINE_INSTANTIATE(NMSym)
SLM_FINE_INSTANTIATE(NMDir)
#undef SLM_FINE_INSTANTIATE

}  // namespace slm
