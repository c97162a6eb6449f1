// k_positive.cu -- Algorithm POSITIVE (Section 3.3) on the GPU.
//
// The local gain of node i is g(i) = m_w k_{i,c_i} - s_i (Sigma_{c_i} - s_i)
// (Section 2.4 specialised to a symmetric W).  Every community holding a node
// with g < 0 is bisected optimally and its parts are examined again, until no
// node has a negative local gain.  The candidate bisections of a community A
// are
//   * a branch cut at a non-cycle node u: a(u) <- u, parts tail(u) and A\tail(u);
//   * a cycle cut at two distinct cycle nodes u, v: a(u) <- u, a(v) <- v, each
//     part being the nodes whose forward path reaches u (resp. v) first;
// and splitting A into S and R changes the modularity numerator by twice
// Sigma_S Sigma_R - m_w W(S,R).  The best value wins even when it is not
// positive; ties prefer a branch cut, then the smaller u, then the smaller v.
//
// Communities are independent (Section 4.2), so every flagged community is
// split in the same round.  A round touches only the members of the flagged
// communities: their subtree sums (ancestor walks, with the weight inside a
// subtree credited at the lowest common ancestor of each edge), the L x L
// weights between the trees hanging from a cycle of length L >= 2, the best
// split, and afterwards the members' components, totals and local gains.
#include <algorithm>
#include <climits>


#include "forest_dev.cuh"


namespace slm {

namespace {

#define GRID_STRIDE SLM_GRID_STRIDE

// Warp loops over the members that need work: each warp tests 32 consecutive
// members at once and then serves the selected ones one after the other with
// all its lanes (an entry of the member's row per lane).
#define WARP_SELECTED(k, cnt, pred)                                                           \
    for (long long _b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; _b < (cnt); \
         _b += (long long)gridDim.x * blockDim.x)                                             \
        for (unsigned _sel = __ballot_sync(0xffffffffu, _b + (threadIdx.x & 31) < (cnt) &&    \
                                                         (pred)(_b + (threadIdx.x & 31)));     \
             _sel; _sel &= _sel - 1)                                                          \
            for (long long k = _b + __ffs(_sel) - 1, _once = 1; _once; _once = 0)


__device__ __forceinline__ unsigned long long split_key(int type, int u, int v) {
    return ((unsigned long long)type << 62) | ((unsigned long long)(unsigned)u << 31) |
           (unsigned long long)(unsigned)v;
}

__device__ __forceinline__ int cyc_index(int v, int r, int l, const int32_t *cdist) {
    return v == r ? 0 : l - cdist[v];
}

// ---------------------------------------------------------------------------
// member lists
// ---------------------------------------------------------------------------
// the listed (or all) nodes of flagged communities, one atomic per warp
__global__ void k_compact_atomic(long long cnt, const int32_t *list, const int32_t *root,
                                 const int32_t *flag, int32_t *out, int32_t *count) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < cnt;
         base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + lane;
        int v = -1;
        bool keep = false;
        if (k < cnt) {
            v = list ? list[k] : (int)k;
            keep = flag[root[v]] != 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        int at = 0;
        if (lane == 0 && bal) at = atomicAdd(count, __popc(bal));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (keep) out[at + __popc(bal & ((1u << lane) - 1u))] = v;
    }
}

// ---------------------------------------------------------------------------
// one round (phases of the persistent kernel below)
// ---------------------------------------------------------------------------
// The set-up of member v at position k of a round's list: new parts (every
// part in the first round) start their sums from zero, and each community
// root is listed once with its cycle length and an empty best cut.
struct RoundInit {
    const int32_t *ideg, *root, *freshN, *a, *cdist;
    long long *subS, *subWA, *subWin, *credit, *TS;
    int32_t *rlist, *posr, *L, *degm;
    long long *kacc, *bestsc;
    unsigned long long *bestkey;
};
__device__ __forceinline__ void init_member(const RoundInit &I, long long k, int v, bool first, int32_t *rcnt) {
    const int r = I.root[v];
    const bool fr = first || I.freshN[r];
    I.degm[k] = fr ? I.ideg[v] : 0;  // only new parts rescan their entries
    I.kacc[k] = 0;
    if (fr) {
        I.subS[v] = 0;
        I.subWA[v] = 0;
        I.subWin[v] = 0;
        I.credit[v] = 0;
        I.TS[v] = 0;
    }
    if (r == v) {
        const int q = atomicAdd(rcnt, 1);
        I.rlist[q] = v;
        I.posr[v] = q;
        I.L[q] = (I.a[v] == v) ? 1 : I.cdist[I.a[v]] + 1;  // cycle length of v's community
        I.bestsc[q] = LLONG_MIN;
        I.bestkey[q] = ~0ull;
    }
}

__device__ __forceinline__ void k_round_init(int cnt, const int32_t *M, const RoundInit &I, bool first,
                                             int32_t *rcnt) {
    GRID_STRIDE(k, cnt) init_member(I, k, M[k], first, rcnt);
}

// The list of the next round from the members of the still-flagged
// communities (in any order: every reduction of a round is order-free), each
// kept member set up for that round at its new position as k_round_init
// would, with its root listed in *rnext.
__device__ __forceinline__ void d_compact_init(int cnt, const int32_t *list, const int32_t *root,
                                               const int32_t *flag, int32_t *out, int32_t *count,
                                               const RoundInit &I, int32_t *rnext) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < cnt;
         base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + lane;
        int v = -1;
        bool keep = false;
        if (k < cnt) {
            v = list[k];
            keep = flag[root[v]] != 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        int at = 0;
        if (lane == 0 && bal) at = atomicAdd(count, __popc(bal));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (keep) {
            const int q = at + __popc(bal & ((1u << lane) - 1u));
            out[q] = v;
            init_member(I, q, v, false, rnext);
        }
    }
}


// pool sizes of the first round, padded with zeros to cnt entries so that
// the offsets can be scanned over the member list's length
__device__ __forceinline__ void k_root_pools(int cnt, const int32_t *Rdev, const int32_t *L,
                                             long long *msz, int32_t *csz) {
    const int R = *Rdev;
    GRID_STRIDE(q, cnt) {
        const int l = q < R ? L[q] : 0;
        msz[q] = l >= 2 ? (long long)l * l : 0;
        csz[q] = l >= 2 ? l : 0;
    }
}

// every member adds itself to its non-cycle ancestors (itself included) and to
// the total of the tree hanging from its entry
template <class NM>
__device__ __forceinline__ void k_walk(int cnt, const int32_t *M, const int32_t *a, const int32_t *depth,
                       const typename NM::ST *s, const int32_t *kown, const int32_t *root,
                       const int32_t *freshN, bool first, long long *subS, long long *subWA,
                       long long *TS) {
    GRID_STRIDE(k, cnt) {
        int x = M[k];
        if (!first && !freshN[root[x]]) continue;
        long long sx = (long long)s[x], kx = kown[x];
        int y = x;
        for (int d = depth[x]; d > 0; d--) {
            add64(&subS[y], sx);
            add64(&subWA[y], kx);
            y = a[y];
        }
        add64(&TS[y], sx);
    }
}

__device__ __forceinline__ void k_cycle_order(int cnt, const int32_t *M, const uint8_t *oncycle,
                              const int32_t *root, const int32_t *posr, const int32_t *L,
                              const int32_t *cdist, const int32_t *coffN, int32_t *cyc) {
    GRID_STRIDE(k, cnt) {
        int v = M[k];
        if (!oncycle[v]) continue;
        int r = root[v];
        int q = posr[r];
        int l = L[q];
        if (l < 2) continue;
        int c = cyc_index(v, r, l, cdist);
        if (c >= 0 && c < l) cyc[coffN[r] + c] = v;
    }
}

// member owning edge slot e of the members' concatenated rows: the last k
// in [lo, hi] with epref[k] <= e
__device__ __forceinline__ int owner_in(long long e, const int32_t *epref, int lo, int hi) {
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if ((long long)epref[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The 32 lanes of a warp hold the consecutive slots base .. base+31: lanes 0
// and 31 search the whole list for the owners of the first and last slot,
// then every lane searches only between those two owners.  Every lane of
// the warp must call this (shuffles); e is clamped to the last slot E-1.
__device__ __forceinline__ int warp_owner(long long base, long long E, const int32_t *epref,
                                          int cnt, long long &e) {
    const int lane = threadIdx.x & 31;
    const long long last = min(base + 31, E - 1);
    e = min(base + lane, last);
    int k = 0;
    if (lane == 0 || lane == 31) k = owner_in(lane == 0 ? base : last, epref, 0, cnt - 1);
    const int lo = __shfl_sync(0xffffffffu, k, 0), hi = __shfl_sync(0xffffffffu, k, 31);
    return owner_in(e, epref, lo, hi);
}

// loop over the slots [0, E) in warp-sized runs of consecutive slots
#define WARP_SLOTS(base, E)                                                               \
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;     \
         base < (E); base += (long long)gridDim.x * blockDim.x)

// one thread per internal edge of a member: LCA credits inside a tree,
// tree-to-tree weights of the cycle
__device__ __forceinline__ void k_edges(int cnt, const int32_t *M, const int32_t *epref, const int32_t *Edev,
                        const int32_t *istart, const int32_t *col, const int32_t *w, const int32_t *a,
                        const uint8_t *oncycle, const int32_t *entry, const int32_t *depth,
                        const int32_t *root, const int32_t *posr, const int32_t *L,
                        const int32_t *cdist, const long long *moffN, long long *Mw,
                        long long *credit) {
    const long long E = *Edev;
    WARP_SLOTS(base, E) {
        long long e;
        const int k = warp_owner(base, E, epref, cnt, e);
        if (e != base + (threadIdx.x & 31)) continue;  // past the last slot
        const int x = M[k];
        const int p = istart[x] + (int)(e - epref[k]);
        const int j = col[p];
        const int r = root[x];
        if (root[j] != r) continue;  // joined by a cut of an earlier round
        const int ex = entry[x], ej = entry[j], wv = w[p];
        if (ej == ex) {
            int l = lca_walk(x, j, a, depth);
            if (!oncycle[l]) add64(&credit[l], wv);
        } else {
            const int q = posr[r];
            int l = L[q];
            int kx = cyc_index(ex, r, l, cdist), kj = cyc_index(ej, r, l, cdist);
            if (l >= 2 && kx >= 0 && kx < l && kj >= 0 && kj < l)
                add64(&Mw[moffN[r] + (long long)kx * l + kj], wv);
        }
    }
}

// credits of the entries of new parts after the first round: every new part
// hangs from a self-loop, so all its entries join nodes of one tree (one warp
// per member of a new part)
__device__ __forceinline__ void k_edges_members(int cnt, const int32_t *M, const int32_t *root,
                                                const int32_t *freshN, const int32_t *istart,
                                                const int32_t *ideg, const int32_t *col,
                                                const int32_t *w, const int32_t *a,
                                                const uint8_t *oncycle, const int32_t *depth,
                                                long long *credit) {
    const int lane = threadIdx.x & 31;
    auto sel = [&](long long k) { return freshN[root[M[k]]] != 0; };
    WARP_SELECTED(k, cnt, sel) {
        const int x = M[k], r = root[x];
        const int b = istart[x], end = b + ideg[x];
        for (int t = b + lane; t < end; t += 32) {
            const int j = col[t];
            if (root[j] != r) continue;
            const int l = lca_walk(x, j, a, depth);
            if (!oncycle[l]) add64(&credit[l], w[t]);
        }
    }
}

__device__ __forceinline__ void k_credit(int cnt, const int32_t *M, const int32_t *a, const int32_t *depth,
                         const int32_t *root, const int32_t *freshN, bool first,
                         const long long *credit, long long *subWin) {
    GRID_STRIDE(k, cnt) {
        int x = M[k];
        if (!first && !freshN[root[x]]) continue;
        long long c = credit[x];
        if (c == 0) continue;
        int y = x;
        for (int d = depth[x]; d > 0; d--) {
            add64(&subWin[y], c);
            y = a[y];
        }
    }
}

template <class NM>
__device__ __forceinline__ void k_branch(int cnt, const int32_t *M, const uint8_t *oncycle, const int32_t *root,
                         const int32_t *posr, const typename NM::ST *sigma, MParam mp,
                         const long long *subS, const long long *subWA, const long long *subWin,
                         long long *bestsc, unsigned long long *bestkey, long long *msc,
                         int32_t *mq, int pass) {
    const int lane = threadIdx.x & 31;
    for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < cnt;
         base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + lane;
        int u = -1, q = -1;
        long long sc = LLONG_MIN;
        if (k < cnt) {
            u = M[k];
            if (pass == 0) {
                if (!oncycle[u]) {
                    const int r = root[u];
                    q = posr[r];
                    const long long m = mp.of(u), sS = subS[u], sA = (long long)sigma[r];
                    sc = NM::cross(sS, sA - sS) - m * (subWA[u] - subWin[u]);
                }
                msc[k] = sc;  // the tie pass reads the member's value back
                mq[k] = q;
            } else {
                sc = msc[k];
                q = mq[k];
            }
        }
        if (pass == 0) {
            // a warp whose branch cuts all belong to one community (the common
            // case when one large community is split again and again) sends
            // one atomic instead of 32
            const int q0 = __shfl_sync(0xffffffffu, q, 0);
            if (__all_sync(0xffffffffu, q == q0 || q < 0) && q0 >= 0) {
#pragma unroll
                for (int o = 16; o; o >>= 1) sc = max(sc, __shfl_xor_sync(0xffffffffu, sc, o));
                if (lane == 0) atomicMax(&bestsc[q0], sc);
            } else if (q >= 0) {
                atomicMax(&bestsc[q], sc);
            }
        } else if (q >= 0 && sc == bestsc[q]) {
            atomicMin(&bestkey[q], split_key(0, u, 0));
        }
    }
}

// one block per community with a cycle of length >= 2; one thread per p, the
// part V = trees (p, q] grows with q: W(V+q, U-q) = W(V,U) + row(q) - 2 W(V,q).
// The row total row(q) and the weight W(V,q) from the trees (p, q) to tree q
// are read from a 2D prefix table of the tree-to-tree weights Mr, built by
// the block in the first pass of each round (P[a][b] = sum of Mr[k][k'] over
// k < a, k' < b), so every cut costs O(1) and a community O(l^2) instead of
// O(l^3).  The sums are those of Mr itself: the values are unchanged.
template <class NM>
__device__ __forceinline__ void k_cycle(const int32_t *Rdev, const int32_t *rlist, const int32_t *L, const int32_t *coffN,
                        const int32_t *cyc, const long long *moffN, const long long *Mw, long long *Mp,
                        const long long *TS, const typename NM::ST *sigma, MParam mp, int32_t n,
                        long long *bestsc, unsigned long long *bestkey, int pass) {
    const int R = *Rdev;
    for (int q0 = blockIdx.x; q0 < R; q0 += gridDim.x) {
        const int l = L[q0];
        if (l < 2) continue;
        const int r = rlist[q0];
        const long long m = mp.of(r);
        const int32_t *cy = cyc + coffN[r];
        const long long *Mr = Mw + moffN[r];
        const long long l1 = l + 1;
        // (l + 1)^2 <= l^2 + 3 l entries: the region of this community in Mp
        long long *P = Mp + moffN[r] + 3LL * coffN[r];
        if (pass == 0) {
            for (int b = threadIdx.x; b <= l; b += blockDim.x) P[b] = 0;
            for (int k = threadIdx.x; k < l; k += blockDim.x) {  // prefixes along each row
                long long acc = 0;
                long long *row = P + (long long)(k + 1) * l1;
                row[0] = 0;
                for (int t = 0; t < l; t++) {
                    acc += Mr[(long long)k * l + t];
                    row[t + 1] = acc;
                }
            }
            __syncthreads();
            for (int bcol = threadIdx.x; bcol <= l; bcol += blockDim.x) {  // then down each column
                long long acc = 0;
                for (int a = 1; a <= l; a++) {
                    acc += P[(long long)a * l1 + bcol];
                    P[(long long)a * l1 + bcol] = acc;
                }
            }
            __syncthreads();
        }
        const long long sA = (long long)sigma[r];
        for (int p = threadIdx.x; p < l; p += blockDim.x) {
            const int cp = cy[p];
            if (cp < 0 || cp >= n) continue;  // unfilled slot (cannot happen): no cut at p
            const long long *Pp1 = P + (long long)(p + 1) * l1;
            long long cut = 0, sV = 0;
            for (int q = p + 1; q < l; q++) {
                const int cq = cy[q];
                if (cq < 0 || cq >= n) break;
                const long long *Pq = P + (long long)q * l1, *Pq1 = P + (long long)(q + 1) * l1;
                const long long rowq = Pq1[l] - Pq[l];
                const long long inV = (Pq[q + 1] - Pq[q]) - (Pp1[q + 1] - Pp1[q]);
                cut += rowq - 2 * inV;
                sV += TS[cq];
                long long sc = NM::cross(sV, sA - sV) - m * cut;
                int u = min(cp, cq), v = max(cp, cq);
                if (pass == 0) atomicMax(&bestsc[q0], sc);
                else if (sc == bestsc[q0]) atomicMin(&bestkey[q0], split_key(1, u, v));
            }
        }
    }
}

// per split community: record the cut, set the totals of the two parts from
// the subtree sums, and remove the cut assignments (a(u) <- u, a(v) <- v).
// A branch cut keeps the remainder's sums (they are corrected in place after
// the cut), so it records what the corrections need: the cut subtree's sums,
// u's old parent and entry.  The part cut off, and both parts of a cycle
// cut, are new (their sums are recomputed in the next round).
template <class NM>
__device__ __forceinline__ void k_cut_info(const int32_t *Rdev, const int32_t *rlist,
                           const unsigned long long *bestkey, int32_t n, const int32_t *L,
                           const int32_t *coffN, const int32_t *cyc, const long long *TS,
                           const int32_t *depth, const int32_t *entry, const int32_t *cdist,
                           const long long *subS, const long long *subWA,
                           const long long *subWin, typename NM::ST *sigma, int4 *cut, long long *cutsum,
                           int32_t *cutpar, int32_t *freshN, int32_t *a, const int32_t *gid,
                           int32_t *splits_per_graph) {
    const int R = *Rdev;
    GRID_STRIDE(q, R) {
        const int r = rlist[q];
        if (splits_per_graph) atomicAdd(&splits_per_graph[gid ? gid[r] : 0], 1);
        const unsigned long long key = bestkey[q];
        if (key == ~0ull) {  // no option recorded (cannot happen for size >= 2)
            cut[q] = make_int4(-1, 0, 0, 0);
            freshN[r] = 1;
            continue;
        }
        const int type = (int)(key >> 62);
        const int u = (int)((key >> 31) & 0x7fffffffu);
        const int v = (int)(key & 0x7fffffffu);
        if (u >= n || (type == 1 && v >= n)) {
            cut[q] = make_int4(-1, 0, 0, 0);
            freshN[r] = 1;
            continue;
        }
        if (type == 0) {
            const long long sS = subS[u];
            cut[q] = make_int4(0, u, depth[u], entry[u]);
            cutsum[3 * q] = sS;
            cutsum[3 * q + 1] = subWA[u];
            cutsum[3 * q + 2] = subWin[u];
            cutpar[q] = a[u];
            using ST = typename NM::ST;
            sigma[r] = (ST)((long long)sigma[r] - sS);  // S is part of A: no component goes negative
            sigma[u] = (ST)sS;
            a[u] = u;
            freshN[r] = 0;
            freshN[u] = 1;
        } else {
            const int l = L[q];
            const int iu = cyc_index(u, r, l, cdist), iv = cyc_index(v, r, l, cdist);
            const int p = min(iu, iv), pq = max(iu, iv);
            const int32_t *cy = cyc + coffN[r];
            long long sV = 0;
            for (int k = p + 1; k <= pq; k++) sV += TS[cy[k]];
            const long long sA = (long long)sigma[r];
            const int cp = cy[p], cq = cy[pq];
            cut[q] = make_int4(1, p, pq, l);
            sigma[cq] = (typename NM::ST)sV;
            sigma[cp] = (typename NM::ST)(sA - sV);
            a[cp] = cp;
            a[cq] = cq;
            freshN[cp] = 1;
            freshN[cq] = 1;
        }
    }
}

// components of the members after the cuts, in closed form from the old
// forest: a branch cut at u roots tail(u) at u (depths shift by depth(u)); a
// cycle cut at positions p < q of the cycle roots the trees of (p, q] at
// c_q and the others at c_p, each tree's depth growing by its distance along
// the cycle.  Read-only phase: the new values go to per-member scratch.
__device__ __forceinline__ void k_forest_new(int cnt, const int32_t *M, const int32_t *a, const int32_t *root,
                             const int32_t *entry, const int32_t *depth, const int32_t *cdist,
                             const uint8_t *oncycle, const int32_t *posr, const int4 *cut,
                             const int32_t *coffN, const int32_t *cyc, int4 *nf, uint8_t *noc,
                             int32_t *oldroot, uint8_t *recomp) {
    GRID_STRIDE(k, cnt) {
        const int x = M[k];
        const int r = root[x];
        const int4 ct = cut[posr[r]];
        int4 v = make_int4(r, entry[x], depth[x], cdist[x]);
        uint8_t oc = oncycle[x];
        uint8_t rc = 0;  // 1: x's new part is new (its local gain is recomputed)
        if (ct.x == 0) {
            const int u = ct.y, du = ct.z;
            int dx = depth[x];
            if (dx >= du) {
                int y = x;
                for (int t = dx - du; t > 0; t--) y = a[y];
                if (y == u) {
                    v = make_int4(u, u, dx - du, 0);
                    oc = (x == u);
                    rc = 1;
                }
            }
        } else if (ct.x == 1) {
            rc = 1;
            const int p = ct.y, pq = ct.z, l = ct.w;
            const int e = entry[x];
            const int ie = cyc_index(e, r, l, cdist);
            const int32_t *cy = cyc + coffN[r];
            if (ie > p && ie <= pq) {
                const int cq = cy[pq];
                v = make_int4(cq, cq, depth[x] + (pq - ie), 0);
                oc = (x == cq);
            } else {
                const int cp = cy[p];
                v = make_int4(cp, cp, depth[x] + ((p - ie + l) % l), 0);
                oc = (x == cp);
            }
        }
        nf[k] = v;
        noc[k] = oc;
        oldroot[k] = r;
        recomp[k] = rc;
    }
}

// Corrections of a branch cut's remainder R = A \ S (S = tail(u)), with the
// values before the cut: every non-cycle ancestor of u loses S's strength
// total, S's own-weight total and S's internal weight, and the tree total of
// u's entry loses S's strength total (one thread per cut).  Then every entry
// (x, y) with x in S and y in R removes w from y's own weight and from the
// own-weight totals of y's non-cycle ancestors, 2w from the internal weight
// of the common non-cycle ancestors of u and y (both directions of the
// pair), or, when y hangs from another tree of the cycle, w from both
// directions of the tree-to-tree weight (one warp per member of S).
__device__ __forceinline__ void k_cut_fix(int cnt, const int32_t *M, const int32_t *Rdev,
                                          const int4 *cut, const long long *cutsum,
                                          const int32_t *cutpar, const int32_t *oldroot,
                                          const uint8_t *recomp, const int32_t *posr,
                                          const int32_t *root, const int32_t *a,
                                          const int32_t *depth, const int32_t *entry,
                                          const int32_t *cdist, const int32_t *istart,
                                          const int32_t *ideg, const int32_t *icol,
                                          const int32_t *iw, const long long *moffN,
                                          int32_t *kown, long long *subS, long long *subWA,
                                          long long *subWin, long long *TS, long long *Mw) {
    const int R = *Rdev;
    GRID_STRIDE(q, R) {
        const int4 ct = cut[q];
        if (ct.x != 0) continue;
        const long long cS = cutsum[3 * q], cWA = cutsum[3 * q + 1], cWin = cutsum[3 * q + 2];
        int y = cutpar[q];
        for (int d = depth[y]; d > 0; d--) {
            add64(&subS[y], -cS);
            add64(&subWA[y], -cWA);
            add64(&subWin[y], -cWin);
            y = a[y];
        }
        add64(&TS[y], -cS);
    }
    const int lane = threadIdx.x & 31;
    // x is in a cut subtree: its part is new, its old community had a branch
    // cut, and x no longer carries the old name
    auto sel = [&](long long k) {
        if (!recomp[k]) return false;
        const int r = oldroot[k];
        return cut[posr[r]].x == 0 && root[M[k]] != r;
    };
    WARP_SELECTED(k, cnt, sel) {
        const int r = oldroot[k];
        const int q = posr[r];
        const int4 ct = cut[q];
        const int x = M[k];
        const int e = ct.w, p = cutpar[q];
        const int l = (a[r] == r) ? 1 : cdist[a[r]] + 1;  // R keeps A's cycle
        const int ke = cyc_index(e, r, l, cdist);
        const int b = istart[x], end = b + ideg[x];
        for (int t = b + lane; t < end; t += 32) {
            const int yv = icol[t];
            if (root[yv] != r) continue;  // inside S, or left A in an earlier round
            const int wv = iw[t];
            atomicSub(&kown[yv], wv);
            int z = yv;
            for (int d = depth[yv]; d > 0; d--) {
                add64(&subWA[z], -(long long)wv);
                z = a[z];
            }
            if (entry[yv] == e) {
                z = lca_walk(p, yv, a, depth);
                for (int d = depth[z]; d > 0; d--) {
                    add64(&subWin[z], -2 * (long long)wv);
                    z = a[z];
                }
            } else if (l >= 2) {
                const int ky = cyc_index(entry[yv], r, l, cdist);
                if (ke >= 0 && ke < l && ky >= 0 && ky < l) {
                    add64(&Mw[moffN[r] + (long long)ke * l + ky], -(long long)wv);
                    add64(&Mw[moffN[r] + (long long)ky * l + ke], -(long long)wv);
                }
            }
        }
    }
}

__device__ __forceinline__ void k_forest_write(int cnt, const int32_t *M, const int4 *nf, const uint8_t *noc,
                               const uint8_t *recomp, int32_t *root, int32_t *entry, int32_t *depth,
                               int32_t *cdist, uint8_t *oncycle, int32_t *flag) {
    GRID_STRIDE(k, cnt) {
        const int x = M[k];
        flag[x] = 0;  // the names in use inside the member set are members
        if (!recomp[k]) continue;  // a remainder keeps its components
        const int4 v = nf[k];
        root[x] = v.x;
        entry[x] = v.y;
        depth[x] = v.z;
        cdist[x] = v.w;
        oncycle[x] = noc[k];
    }
}

// own-community weight of the members of new parts (one warp per member)
__device__ __forceinline__ void k_own_members(int cnt, const int32_t *M, const uint8_t *recomp,
                                              const int32_t *istart, const int32_t *ideg,
                                              const int32_t *col, const int32_t *w,
                                              const int32_t *root, long long *kacc) {
    const int lane = threadIdx.x & 31;
    auto sel = [&](long long k) { return recomp[k] != 0; };
    WARP_SELECTED(k, cnt, sel) {
        const int x = M[k], rx = root[x];
        const int b = istart[x], end = b + ideg[x];
        long long acc = 0;
        // four entries per lane in flight: a row's loads do not wait on one another
        for (int t0 = b + lane; t0 < end; t0 += 128) {
            int c[4];
#pragma unroll
            for (int u = 0; u < 4; u++) c[u] = (t0 + 32 * u < end) ? col[t0 + 32 * u] : -1;
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (c[u] >= 0 && root[c[u]] == rx) acc += w[t0 + 32 * u];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) kacc[k] = acc;
    }
}
// ---------------------------------------------------------------------------
// Internal edges of the members: POSITIVE only splits communities, so an
// entry (x, j) with root[j] != root[x] at the start never becomes internal
// again.  The rounds read a compacted copy of the members' internal entries
// (j != x, same community) instead of their whole rows: hubs whose rows
// mostly leave the community cost their internal degree only.
// ---------------------------------------------------------------------------
// members with longer rows are served by whole blocks (k_int_*_big)
constexpr int kIntWarpMaxDeg = 1024;

// The listed members k < cnt whose row is longer than `thr`, each handed to
// body(k) by a whole block: the first warp tests 32 members at once and the
// block walks the long ones in the tile, so finding the few long rows costs
// one load step per tile instead of one per member.  Members of a tile are
// taken in list order; the body may use __syncthreads.
template <class F>
__device__ __forceinline__ void for_long_rows(long long cnt, const int32_t *list, const int32_t *rp, int thr,
                                              unsigned *sbal, F &&body) {
    for (long long t0 = (long long)blockIdx.x * 32; t0 < cnt; t0 += (long long)gridDim.x * 32) {
        if (threadIdx.x < 32) {
            const long long k = t0 + threadIdx.x;
            bool lng = false;
            if (k < cnt) {
                const int x = list[k];
                lng = rp[x + 1] - rp[x] > thr;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, lng);
            if (threadIdx.x == 0) *sbal = bal;
        }
        __syncthreads();
        unsigned b = *sbal;
        while (b) {
            const int q = __ffs(b) - 1;
            b &= b - 1;
            body(t0 + q);
        }
        __syncthreads();
    }
}
// blocks for for_long_rows over cnt members
inline int long_row_blocks(long long cnt) { return grid_for((cnt + 31) / 32, 1, kNumSMs * 4); }

__global__ void k_int_fill(int cnt, const int32_t *M, const int32_t *rp, const int32_t *col,
                           const int32_t *w, const int32_t *root, const int32_t *ioff,
                           int32_t *istart, int32_t *ideg, int32_t *icol, int32_t *iw) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < cnt; k += nw) {
        const int x = M[k], r = root[x];
        const int b = rp[x], e = rp[x + 1];
        if (e - b > kIntWarpMaxDeg) continue;
        const int first = ioff[k];
        int out = first;
        for (int p0 = b; p0 < e; p0 += 32) {
            const int p = p0 + lane;
            int j = -1;
            if (p < e) j = col[p];
            const bool in = p < e && j != x && root[j] == r;
            const unsigned bal = __ballot_sync(0xffffffffu, in);
            if (in) {
                const int q = out + __popc(bal & ((1u << lane) - 1u));
                icol[q] = j;
                iw[q] = w[p];
            }
            out += __popc(bal);
        }
        if (lane == 0) {
            istart[x] = first;
            ideg[x] = out - first;
        }
    }
}

// a long row filled by a whole block: the order of a member's internal
// entries does not matter (every use of them is a sum or a test), so each
// warp claims its slots with one atomic on the member's cursor
__global__ void k_int_fill_big(int cnt, const int32_t *M, const int32_t *rp, const int32_t *col,
                               const int32_t *w, const int32_t *root, const int32_t *ioff,
                               int32_t *istart, int32_t *ideg, int32_t *icol, int32_t *iw) {
    __shared__ int cursor;
    __shared__ unsigned sbal;
    const int lane = threadIdx.x & 31;
    for_long_rows(cnt, M, rp, kIntWarpMaxDeg, &sbal, [&](long long k) {
        const int x = M[k];
        const int b = rp[x], e = rp[x + 1];
        const int r = root[x];
        if (threadIdx.x == 0) cursor = ioff[k];
        __syncthreads();
        // eight entries per lane in flight; one cursor claim per warp and batch
        const unsigned below = (1u << lane) - 1u;
        for (int p0 = b + (threadIdx.x & ~31); p0 < e; p0 += 8 * blockDim.x) {
            int j[8];
            bool in[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const int p = p0 + t * (int)blockDim.x + lane;
                j[t] = p < e ? col[p] : -1;
            }
#pragma unroll
            for (int t = 0; t < 8; t++) in[t] = j[t] >= 0 && j[t] != x && root[j[t]] == r;
            unsigned bal[8];
            int tot = 0;
#pragma unroll
            for (int t = 0; t < 8; t++) {
                bal[t] = __ballot_sync(0xffffffffu, in[t]);
                tot += __popc(bal[t]);
            }
            int at = 0;
            if (lane == 0 && tot) at = atomicAdd(&cursor, tot);
            at = __shfl_sync(0xffffffffu, at, 0);
#pragma unroll
            for (int t = 0; t < 8; t++) {
                if (in[t]) {
                    const int q = at + __popc(bal[t] & below);
                    icol[q] = j[t];
                    iw[q] = w[p0 + t * (int)blockDim.x + lane];
                }
                at += __popc(bal[t]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            istart[x] = ioff[k];
            ideg[x] = cursor - ioff[k];
        }
        __syncthreads();
    });
}
template <class NM>
__device__ __forceinline__ void k_own_finish(int cnt, const int32_t *M, const typename NM::ST *s, MParam mp,
                             const int32_t *root, const typename NM::ST *sigma, const long long *kacc,
                             const uint8_t *recomp, int32_t *kown, int32_t *flag) {
    GRID_STRIDE(k, cnt) {
        int i = M[k];
        const long long m = mp.of(i);
        int ci = root[i];
        long long own = kown[i];  // a remainder's own weights were corrected in place
        if (recomp[k]) {
            own = kacc[k];
            kown[i] = (int32_t)own;
        }
        long long si = (long long)s[i];
        if (m * own - NM::cross(si, (long long)sigma[ci] - si) < 0) flag[ci] = 1;
    }
}

// ---------------------------------------------------------------------------
// Grid-wide exclusive prefix sums inside the persistent kernel: block t owns a
// contiguous chunk; block sums are scanned by block 0.  Up to three arrays of
// the same length are scanned together.  Ends after a grid barrier.
// ---------------------------------------------------------------------------
// the own weights are recomputed by the bucketed pass over every node when
// the communities to re-examine hold more than n / kOwnFullDiv nodes, and
// node by node from their list otherwise (measured on R-MAT and LFR graphs:
// 16 is best on R-MAT, 2 and 4 save up to 2% on LFR graphs at high mixing)
#ifndef SLM_OWN_FULL_DIV
#define SLM_OWN_FULL_DIV 16
#endif
constexpr int kOwnFullDiv = SLM_OWN_FULL_DIV;
#ifndef SLM_POS_FULL_THREADS
#define SLM_POS_FULL_THREADS 256
#endif
// threads per block of the full grid (one block per SM); measured on R-MAT
// scale 20, 512 and 1,024 threads per block make the run 3% and 11% slower
// (the block barrier inside every grid barrier waits for more warps)
constexpr int kPosThreads = SLM_POS_FULL_THREADS;
// threads of a one-block tail: every member of a small round gets its own thread
constexpr int kPosTailThreads = 1024;
// a POSITIVE call continues on a grid of kPosTailBlocks blocks (by default
// one block, whose grid barriers are block barriers) once a round has at most
// kPosTailMembers members and kPosTailEntries internal entries: measured on
// R-MAT and weighted LFR graphs, one block with a 2,048-member handoff is the
// fastest of 1, 4 and 16 blocks with 2,048, 8,192 or 32,768 members
#ifndef SLM_POS_TAIL_BLOCKS
#define SLM_POS_TAIL_BLOCKS 1
#endif
constexpr int kPosTailBlocks = SLM_POS_TAIL_BLOCKS;
// blocks per SM of the full grid: rounds hold tens of thousands of members at
// most, and a grid barrier costs one atomic per block, so one block per SM
// is enough
#ifndef SLM_POS_BLOCKS_PER_SM
#define SLM_POS_BLOCKS_PER_SM 1
#endif
constexpr int kPosBlocksPerSM = SLM_POS_BLOCKS_PER_SM;
#ifndef SLM_POS_TAIL_MEMBERS
#define SLM_POS_TAIL_MEMBERS 2048
#endif
constexpr int kPosTailMembers = SLM_POS_TAIL_MEMBERS;
constexpr long long kPosTailEntries = 8LL * SLM_POS_TAIL_MEMBERS;

template <class T> __device__ T block_sum(T v, T *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
    __syncthreads();
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

// exclusive scan of one tile (one value per thread); returns the tile total
template <class T> __device__ T tile_scan(T v, T &excl, T *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) red[wid] = x;
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    if (threadIdx.x == 0) {
        T acc = 0;
        for (int k = 0; k < nw; k++) {
            T c = red[k];
            red[k] = acc;
            acc += c;
        }
        red[nw] = acc;
    }
    __syncthreads();
    excl = red[wid] + x - v;
    T tot = red[nw];
    __syncthreads();
    return tot;
}

struct ScanSlots {
    long long *a;
    int32_t *b, *c;  // arrays (c may be null)
    long long *tot_a;
    int32_t *tot_b, *tot_c;
    long long *bs_a;  // block sums, gridDim.x entries each
    int32_t *bs_b, *bs_c;
};

#define GBAR_OR_RETURN(r)                        \
    do {                                         \
        if (!gbar(A.bar, A.barrier_ns)) return r; \
    } while (0)

__device__ bool grid_scan(const ScanSlots &S, int n, GridBarrier *bar, long long barrier_ns) {
    __shared__ long long red64[33];  // one slot per warp (up to 32) and a total
    __shared__ int32_t red32[33];
    const int nb = gridDim.x;
    const int chunk = (n + nb - 1) / nb;
    const int lo = min(n, (int)blockIdx.x * chunk), hi = min(n, lo + chunk);
    long long sa = 0;
    int32_t sb = 0, sc = 0;
    for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        if (S.a) sa += S.a[k];
        sb += S.b[k];
        if (S.c) sc += S.c[k];
    }
    if (S.a) sa = block_sum<long long>(sa, red64);
    sb = block_sum<int32_t>(sb, red32);
    if (S.c) sc = block_sum<int32_t>(sc, red32);
    if (threadIdx.x == 0) {
        if (S.a) S.bs_a[blockIdx.x] = sa;
        S.bs_b[blockIdx.x] = sb;
        if (S.c) S.bs_c[blockIdx.x] = sc;
    }
    if (!gbar(bar, barrier_ns)) return false;
    if (blockIdx.x == 0) {
        long long ca = 0;
        int32_t cb = 0, cc = 0;
        for (int t0 = 0; t0 < nb; t0 += blockDim.x) {
            const int t = t0 + threadIdx.x;
            long long va = (S.a && t < nb) ? S.bs_a[t] : 0, ea = 0;
            int32_t vb = t < nb ? S.bs_b[t] : 0, eb = 0;
            int32_t vc = (S.c && t < nb) ? S.bs_c[t] : 0, ec = 0;
            long long ta = S.a ? tile_scan<long long>(va, ea, red64) : 0;
            int32_t tb = tile_scan<int32_t>(vb, eb, red32);
            int32_t tc = S.c ? tile_scan<int32_t>(vc, ec, red32) : 0;
            if (t < nb) {
                if (S.a) S.bs_a[t] = ca + ea;
                S.bs_b[t] = cb + eb;
                if (S.c) S.bs_c[t] = cc + ec;
            }
            ca += ta;
            cb += tb;
            cc += tc;
        }
        if (threadIdx.x == 0) {
            if (S.a) *S.tot_a = ca;
            *S.tot_b = cb;
            if (S.c) *S.tot_c = cc;
        }
    }
    if (!gbar(bar, barrier_ns)) return false;
    long long ca = S.a ? S.bs_a[blockIdx.x] : 0;
    int32_t cb = S.bs_b[blockIdx.x], cc = S.c ? S.bs_c[blockIdx.x] : 0;
    for (int k0 = lo; k0 < hi; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        long long va = (S.a && k < hi) ? S.a[k] : 0, ea = 0;
        int32_t vb = k < hi ? S.b[k] : 0, eb = 0;
        int32_t vc = (S.c && k < hi) ? S.c[k] : 0, ec = 0;
        long long ta = S.a ? tile_scan<long long>(va, ea, red64) : 0;
        int32_t tb = tile_scan<int32_t>(vb, eb, red32);
        int32_t tc = S.c ? tile_scan<int32_t>(vc, ec, red32) : 0;
        if (k < hi) {
            if (S.a) S.a[k] = ca + ea;
            S.b[k] = cb + eb;
            if (S.c) S.c[k] = cc + ec;
        }
        ca += ta;
        cb += tb;
        cc += tc;
    }
    return gbar(bar, barrier_ns);
}

// Control block shared by the host and the persistent kernel.
struct PosCtrl {
    int32_t cnt;     // members of the current round
    int32_t R[2];    // roots listed for the rounds of parity 0 and 1
    int32_t E;       // member edges of the current round
    int32_t ctot;    // cycle-order pool entries in use
    long long mtot;  // tree-weight pool entries in use
    int32_t nextc[2];// members kept, counted by atomics; round r uses nextc[r & 1]
    int32_t error;   // 1: round limit, 2: pool too small
    int32_t handoff; // 1: the grid stopped so that a smaller one continues
    int32_t list_b;  // 1: the current member list is listB
    GridBarrier bar; // zeroed by the host before every launch
    long long rounds, visits, splits;
    long long ph[kPosPhases];  // nanoseconds per phase, summed over rounds (when profiling)
};


template <class NM>
struct PosArgs {
    int32_t n;
    const int32_t *istart, *ideg, *icol, *iw;  // internal entries of the members
    const typename NM::ST *s;
    MParam m;
    int32_t *a, *root, *entry, *depth, *cdist;
    uint8_t *oncycle;
    typename NM::ST *sigma;
    int32_t *flag, *kown, *listA, *listB, *rlist, *posr, *L, *coff, *epref, *mark, *cyc;
    long long *msz, *subS, *subWA, *subWin, *credit, *TS, *bestsc, *kacc, *Mw;
    long long *Mp;  // 2D prefix tables of the cycles' tree-to-tree weights
    unsigned long long *bestkey;
    int4 *cut, *nf;
    uint8_t *noc, *recomp;
    long long *moffN, *cutsum;
    int32_t *coffN, *freshN, *cutpar, *oldroot;
    int first_round;  // 1 in the first launch of a call: every community is new
    int32_t *splits_per_graph;
    long long *bs64;
    int32_t *bs32a, *bs32b;
    long long pool_cap, cyc_cap, max_rounds;
    PosCtrl *ctrl;
    int profile;       // stamp the phases with the global timer
    GridBarrier *bar;  // zeroed before each launch
    long long barrier_ns;  // time limit of one barrier wait
    int handoff_cnt;   // > 0: stop (handoff = 1) once a round has at most this many members
    long long handoff_edges;  // ... and at most this many internal entries
};

// All rounds of POSITIVE in one cooperative launch: the phases of a round are
// separated by grid barriers and the loop ends on the device when no member
// is left.
template <class NM, int THREADS>
__global__ void __launch_bounds__(THREADS) k_positive_rounds(PosArgs<NM> A) {
    const bool rank0 = blockIdx.x == 0 && threadIdx.x == 0;
    PosCtrl *C = A.ctrl;
    int32_t *M = A.listA, *M2 = A.listB;
    const int32_t n = A.n;
    // phase stamps, taken by one thread right after a grid barrier
    const bool stamp = A.profile && rank0;
    long long t0 = stamp ? global_ns() : 0;
    auto mark_phase = [&](int k) {
        if (stamp) {
            const long long t = global_ns();
            C->ph[k] += t - t0;
            t0 = t;
        }
    };
    int cnt = C->cnt;  // members of the first round
    int parity = 0;
    bool first = A.first_round != 0;
    // the first round of a launch is set up here; every later one by the
    // compaction that ends the round before it
    bool need_init = true;
    const RoundInit RI{A.ideg, A.root, A.freshN, A.a, A.cdist, A.subS, A.subWA, A.subWin, A.credit, A.TS,
                       A.rlist, A.posr, A.L, A.epref, A.kacc, A.bestsc, A.bestkey};
    for (;;) {
        if (rank0) C->cnt = cnt;
        if (cnt == 0) break;
        if (A.handoff_cnt > 0 && cnt <= A.handoff_cnt && (!first || C->E <= A.handoff_edges)) {
            if (rank0) {
                C->handoff = 1;
                C->list_b = (M == A.listB) ? 1 : 0;
            }
            break;
        }
        if (C->rounds >= A.max_rounds) {
            if (rank0) C->error = 1;
            break;
        }
        // this round's roots are counted in R[parity]; R[parity ^ 1], last
        // read before the previous barrier, takes the next round's
        int32_t *rcnt = &C->R[parity];
        if (rank0) {
            C->nextc[parity] = 0;
            C->R[parity ^ 1] = 0;
        }
        if (need_init) {
            k_round_init(cnt, M, RI, first, rcnt);
            GBAR_OR_RETURN();
        }
        mark_phase(0);
        if (first) {
            // the cycles of every community are laid out once per call: cuts
            // never make a cycle longer, and a part that loses its cycle gets
            // a self-loop, so the layout stays valid for the remainders
            k_root_pools(cnt, rcnt, A.L, A.msz, A.coff);
            GBAR_OR_RETURN();
            ScanSlots S{A.msz, A.coff, A.epref, &C->mtot, &C->ctot, &C->E, A.bs64, A.bs32a, A.bs32b};
            if (!grid_scan(S, cnt, A.bar, A.barrier_ns)) return;
            mark_phase(1);
            if (C->mtot > A.pool_cap || C->ctot > A.cyc_cap) {
                if (rank0) C->error = 2;
                break;
            }
            const long long mtot = C->mtot, ctot = C->ctot;
            const int R = *rcnt;
            GRID_STRIDE(q, R) {
                const int r = A.rlist[q];
                A.moffN[r] = A.msz[q];
                A.coffN[r] = A.coff[q];
            }
            GRID_STRIDE(k, mtot) A.Mw[k] = 0;
            GRID_STRIDE(k, ctot) A.cyc[k] = -1;
            GBAR_OR_RETURN();
            k_walk<NM>(cnt, M, A.a, A.depth, A.s, A.kown, A.root, A.freshN, true, A.subS, A.subWA, A.TS);
            if (ctot > 0)
                k_cycle_order(cnt, M, A.oncycle, A.root, A.posr, A.L, A.cdist, A.coffN, A.cyc);
            k_edges(cnt, M, A.epref, &C->E, A.istart, A.icol, A.iw, A.a, A.oncycle, A.entry, A.depth,
                    A.root, A.posr, A.L, A.cdist, A.moffN, A.Mw, A.credit);
        } else {
            // later rounds: only the parts cut off in the last round are new
            k_walk<NM>(cnt, M, A.a, A.depth, A.s, A.kown, A.root, A.freshN, false, A.subS, A.subWA, A.TS);
            k_edges_members(cnt, M, A.root, A.freshN, A.istart, A.ideg, A.icol, A.iw, A.a, A.oncycle,
                            A.depth, A.credit);
        }
        const bool cycles = C->ctot > 0;
        GBAR_OR_RETURN();
        mark_phase(2);
        k_credit(cnt, M, A.a, A.depth, A.root, A.freshN, first, A.credit, A.subWin);
        GBAR_OR_RETURN();
        mark_phase(3);
        // the members' branch scores and community slots of the first pass are
        // kept for the tie pass in two per-member arrays that are free here:
        // kacc (rewritten by k_own_members before it is read) and epref (read
        // only by the first round's k_edges, which has finished)
        for (int pass = 0; pass < 2; pass++) {
            k_branch<NM>(cnt, M, A.oncycle, A.root, A.posr, A.sigma, A.m, A.subS, A.subWA, A.subWin,
                     A.bestsc, A.bestkey, A.kacc, A.epref, pass);
            if (cycles)
                k_cycle<NM>(rcnt, A.rlist, A.L, A.coffN, A.cyc, A.moffN, A.Mw, A.Mp, A.TS, A.sigma, A.m, n,
                        A.bestsc, A.bestkey, pass);
            GBAR_OR_RETURN();
        }
        mark_phase(4);
        k_cut_info<NM>(rcnt, A.rlist, A.bestkey, n, A.L, A.coffN, A.cyc, A.TS, A.depth, A.entry, A.cdist,
                   A.subS, A.subWA, A.subWin, A.sigma, A.cut, A.cutsum, A.cutpar, A.freshN, A.a,
                   A.m.gid, A.splits_per_graph);
        GBAR_OR_RETURN();
        mark_phase(5);
        k_forest_new(cnt, M, A.a, A.root, A.entry, A.depth, A.cdist, A.oncycle, A.posr, A.cut,
                     A.coffN, A.cyc, A.nf, A.noc, A.oldroot, A.recomp);
        GBAR_OR_RETURN();
        k_forest_write(cnt, M, A.nf, A.noc, A.recomp, A.root, A.entry, A.depth, A.cdist, A.oncycle,
                       A.flag);
        GBAR_OR_RETURN();
        mark_phase(6);
        k_cut_fix(cnt, M, rcnt, A.cut, A.cutsum, A.cutpar, A.oldroot, A.recomp, A.posr, A.root, A.a,
                  A.depth, A.entry, A.cdist, A.istart, A.ideg, A.icol, A.iw, A.moffN, A.kown, A.subS,
                  A.subWA, A.subWin, A.TS, A.Mw);
        k_own_members(cnt, M, A.recomp, A.istart, A.ideg, A.icol, A.iw, A.root, A.kacc);
        GBAR_OR_RETURN();
        k_own_finish<NM>(cnt, M, A.s, A.m, A.root, A.sigma, A.kacc, A.recomp, A.kown, A.flag);
        GBAR_OR_RETURN();
        mark_phase(7);
        // members of the still-flagged communities form the next list, set up
        // for the next round as they are written
        d_compact_init(cnt, M, A.root, A.flag, M2, &C->nextc[parity], RI, &C->R[parity ^ 1]);
        if (rank0) {
            C->rounds += 1;
            C->visits += cnt;
            C->splits += *rcnt;
            if (stamp && gridDim.x > kPosTailBlocks) {
                C->ph[9] += 1;
                C->ph[10] += cnt;
            }
        }
        GBAR_OR_RETURN();
        cnt = *((volatile int32_t *)&C->nextc[parity]);
        mark_phase(8);
        int32_t *tmp = M;
        M = M2;
        M2 = tmp;
        parity ^= 1;
        first = false;
        need_init = false;
    }
}

// Communities a synchronous write touched: the old community and the target
// community of every accepted node.
__global__ void k_mark_moved(const int32_t *acc, const int32_t *acc_cnt, const int32_t *root,
                             const int32_t *best, int32_t *mark) {
    const int c = *acc_cnt;
    GRID_STRIDE(k, c) {
        const int i = acc[k];
        mark[root[i]] = 1;
        mark[best[i]] = 1;
    }
}

// Communities whose membership changed since the last POSITIVE: a node whose
// name changed marks its new and its old name (the old name, when it is
// still in use, is the community that lost it).
__global__ void k_dirty(int32_t n, const int32_t *root, const int32_t *prev_root, int32_t *dirty) {
    GRID_STRIDE(v, n) {
        const int r = root[v], p = prev_root[v];
        if (r != p) {
            dirty[r] = 1;
            dirty[p] = 1;
        }
    }
}

// Own weight and local gain of listed nodes (one warp per node; rows longer
// than kOwnWarpMaxDeg are left to k_own_listed_big): flag[root] = 1 when the
// local gain is negative.
constexpr int kOwnWarpMaxDeg = 1024;
template <class NM>
__global__ void k_own_listed(int cnt, const int32_t *list, const int32_t *rp, const int32_t *col,
                             const int32_t *w, const typename NM::ST *s, MParam mp,
                             const int32_t *root, const typename NM::ST *sigma, int32_t *kown,
                             int32_t *flag) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < cnt; k += nw) {
        const int x = list[k];
        const int b = rp[x], e = rp[x + 1];
        if (e - b > kOwnWarpMaxDeg) continue;
        const int rx = root[x];
        long long acc = 0;
        for (int t = b + lane; t < e; t += 32) {
            const int j = col[t];
            if (j != x && root[j] == rx) acc += w[t];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            kown[x] = (int32_t)acc;
            const long long m = mp.of(x), si = (long long)s[x];
            if (m * acc - NM::cross(si, (long long)sigma[rx] - si) < 0) flag[rx] = 1;
        }
    }
}
template <class NM>
__global__ void k_own_listed_big(int cnt, const int32_t *list, const int32_t *rp, const int32_t *col,
                                 const int32_t *w, const typename NM::ST *s, MParam mp,
                                 const int32_t *root, const typename NM::ST *sigma, int32_t *kown,
                                 int32_t *flag) {
    __shared__ long long red[32];
    __shared__ unsigned sbal;
    for_long_rows(cnt, list, rp, kOwnWarpMaxDeg, &sbal, [&](long long k) {
        const int x = list[k];
        const int b = rp[x], e = rp[x + 1];
        const int rx = root[x];
        long long acc = 0;
        // eight entries per thread in flight: a hub's row takes few dependent steps
        for (int p0 = b + threadIdx.x; p0 < e; p0 += 8 * blockDim.x) {
            int j[8];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const int p = p0 + t * (int)blockDim.x;
                j[t] = p < e ? col[p] : -1;
            }
#pragma unroll
            for (int t = 0; t < 8; t++)
                if (j[t] >= 0 && j[t] != x && root[j[t]] == rx) acc += w[p0 + t * (int)blockDim.x];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += red[q];
            kown[x] = (int32_t)t;
            const long long m = mp.of(x), si = (long long)s[x];
            if (m * t - NM::cross(si, (long long)sigma[rx] - si) < 0) flag[rx] = 1;
        }
        __syncthreads();
    });
}

// bound of the pools: cycle lengths never grow during POSITIVE
__global__ void k_pool_bound(int cnt, const int32_t *M, const int32_t *root, const int32_t *a,
                             const int32_t *cdist, const int32_t *rp, int32_t *rowlen,
                             unsigned long long *msum, unsigned long long *csum) {
    GRID_STRIDE(k, cnt) {
        int r = M[k];
        rowlen[k] = rp[r + 1] - rp[r];  // room for the member's internal entries
        if (root[r] != r) continue;
        long long l = (a[r] == r) ? 1 : cdist[a[r]] + 1;
        if (l >= 2) {
            atomicAdd(msum, (unsigned long long)(l * l));
            atomicAdd(csum, (unsigned long long)l);
        }
    }
}

}  // namespace

// Member list of the flagged communities: from all nodes (list == nullptr) or
// from a previous list; returns its length (host-synchronous).  The list's
// order is that of the warps' atomics: everything that reads a member list
// (the own weights, COMPONENTS, the rounds of POSITIVE, whose roots are
// listed by atomics too) is independent of it.
int32_t compact_members(long long cnt, const int32_t *list, const int32_t *root,
                        const int32_t *flag, int32_t *out, DevBuf &mark, DevBuf &tot,
                        cudaStream_t st) {
    (void)mark;
    if (cnt <= 0) return 0;
    SLM_CUDA(cudaMemsetAsync(tot.get(), 0, sizeof(int32_t), st));
    k_compact_atomic<<<grid_for(cnt, 256, kNumSMs * 16), 256, 0, st>>>(cnt, list, root, flag, out,
                                                                       tot.as<int32_t>());
    SLM_LAUNCH_CHECK();
    int32_t h = 0;
    SLM_CUDA(cudaMemcpyAsync(&h, tot.get(), sizeof h, cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    return h;
}

int32_t moved_members(int32_t n, const int32_t *acc, const int32_t *acc_cnt, int32_t max_acc,
                      const int32_t *root, const int32_t *best, int32_t *out, DevBuf &mark,
                      DevBuf &scratch, DevBuf &tot, cudaStream_t st) {
    if (n <= 0) return 0;
    mark.ensure(4 * ((size_t)n + 1), st);
    tot.ensure(16, st);
    SLM_CUDA(cudaMemsetAsync(mark.get(), 0, 4 * (size_t)n, st));
    k_mark_moved<<<grid_for(max_acc > 0 ? max_acc : 1, 256), 256, 0, st>>>(acc, acc_cnt, root, best,
                                                                         mark.as<int32_t>());
    SLM_LAUNCH_CHECK();
    return compact_members(n, nullptr, root, mark.as<int32_t>(), out, scratch, tot, st);
}

template <class NM>
long long positive_correct(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                           const typename NM::ST *s, MParam m, int32_t *a, Forest &f,
                           typename NM::ST *sigma,
                           const Buckets &bk, PositiveScratch &ps, cudaStream_t st,
                           long long *rounds_out, long long *visits_out,
                           int32_t *splits_per_graph, const int32_t *prev_root) {
    if (rounds_out) *rounds_out = 0;
    if (visits_out) *visits_out = 0;
    if (n <= 0) return 0;
    const size_t N = (size_t)n;
    for (DevBuf *b : {&ps.flag, &ps.kown, &ps.listA, &ps.listB, &ps.rlist, &ps.posr, &ps.L, &ps.coff})
        b->ensure(4 * (N + 1), st);
    for (DevBuf *b : {&ps.subS, &ps.subWA, &ps.subWin, &ps.credit, &ps.TS, &ps.msz, &ps.bestsc,
                      &ps.bestkey})
        b->ensure(8 * (N + 1), st);
    ps.cnt.ensure(64, st);
    ps.tot.ensure(16, st);
    int32_t *flag = ps.flag.as<int32_t>(), *kown = ps.kown.as<int32_t>();
    int32_t *rcnt = ps.cnt.as<int32_t>();

    // local gains for the current forest
    community_sigma(n, f.root, s, sigma, st);
    SLM_CUDA(cudaMemsetAsync(flag, 0, 4 * N, st));
    int32_t *M = ps.listA.as<int32_t>(), *M2 = ps.listB.as<int32_t>();
    int32_t cnt = 0;
    int32_t nd = n;
    if (prev_root) {
        // every community was left without a negative local gain by the last
        // POSITIVE; only those whose membership changed since can hold one
        ps.dirty.ensure(4 * (N + 1), st);
        SLM_CUDA(cudaMemsetAsync(ps.dirty.get(), 0, 4 * N, st));
        k_dirty<<<grid_for(n, 256), 256, 0, st>>>(n, f.root, prev_root, ps.dirty.as<int32_t>());
        SLM_LAUNCH_CHECK();
        nd = compact_members(n, nullptr, f.root, ps.dirty.as<int32_t>(), M2, ps.mark, ps.tot, st);
        if (nd == 0) return 0;
    }
    // the full pass when there is no list of communities to re-examine (the
    // first call of a level: M2 holds no list then), or when they hold most
    // of the graph (the bucketed pass is cheaper)
    if (!prev_root || nd * (long long)kOwnFullDiv > n) {
        own_weight_nodes<NM>(n, rp, col, w, s, m, f.root, sigma, bk, kown, flag, st);
        cnt = compact_members(n, nullptr, f.root, flag, M, ps.mark, ps.tot, st);
    } else {
        k_own_listed<NM><<<grid_for((long long)nd * 32, 256), 256, 0, st>>>(nd, M2, rp, col, w, s, m, f.root,
                                                                       sigma, kown, flag);
        SLM_LAUNCH_CHECK();
        k_own_listed_big<NM><<<long_row_blocks(nd), 256, 0, st>>>(nd, M2, rp, col, w, s, m, f.root,
                                                                       sigma, kown, flag);
        SLM_LAUNCH_CHECK();
        cnt = compact_members(nd, M2, f.root, flag, M, ps.mark, ps.tot, st);
    }

    if (cnt == 0) return 0;
    long long *subS = ps.subS.as<long long>(), *subWA = ps.subWA.as<long long>(),
              *subWin = ps.subWin.as<long long>(), *credit = ps.credit.as<long long>(),
              *TS = ps.TS.as<long long>(), *msz = ps.msz.as<long long>(),
              *bestsc = ps.bestsc.as<long long>();
    unsigned long long *bestkey = ps.bestkey.as<unsigned long long>();
    ps.epref.ensure(4 * (N + 1), st);
    ps.kacc.ensure(8 * (N + 1), st);
    ps.cut.ensure(16 * (N + 1), st);
    ps.nf.ensure(16 * (N + 1), st);
    ps.noc.ensure(N + 1, st);
    ps.recomp.ensure(N + 1, st);
    ps.moffN.ensure(8 * (N + 1), st);
    ps.cutsum.ensure(24 * (N + 1), st);
    ps.coffN.ensure(4 * (N + 1), st);
    ps.freshN.ensure(4 * (N + 1), st);
    ps.cutpar.ensure(4 * (N + 1), st);
    ps.oldroot.ensure(4 * (N + 1), st);
    ps.mark.ensure(4 * (N + 1), st);
    // pools sized once: the first round holds the longest cycles.  The
    // internal entries of a member get room for its whole row (the fill
    // counts them), so no separate counting pass reads the rows.
    ps.hdr.ensure(64, st);
    SLM_CUDA(cudaMemsetAsync(ps.hdr.get(), 0, 64, st));
    unsigned long long *bnd = ps.hdr.as<unsigned long long>();
    ps.rowlen.ensure(4 * (N + 1), st);
    ps.ioff.ensure(4 * (N + 1), st);
    k_pool_bound<<<grid_for(cnt, 256), 256, 0, st>>>(cnt, M, f.root, a, f.cdist, rp,
                                                     ps.rowlen.as<int32_t>(), bnd, bnd + 1);
    SLM_LAUNCH_CHECK();
    exclusive_scan_i32(ps.rowlen.as<int32_t>(), ps.ioff.as<int32_t>(), cnt,
                       reinterpret_cast<int32_t *>(bnd + 2), st);
    unsigned long long hb[3] = {0, 0, 0};
    SLM_CUDA(cudaMemcpyAsync(hb, bnd, 24, cudaMemcpyDeviceToHost, st));
    slm::stream_sync(st);
    const long long itot = (long long)(int32_t)(hb[2] & 0xffffffffu);
    ps.pool.ensure(8 * (size_t)(hb[0] > 0 ? hb[0] : 1), st);
    // prefix tables: (l + 1)^2 <= l^2 + 3 l entries per cycle
    ps.pool2.ensure(8 * ((size_t)(hb[0] > 0 ? hb[0] : 1) + 3 * (size_t)(hb[1] > 0 ? hb[1] : 1)), st);
    ps.cyc.ensure(4 * (size_t)(hb[1] > 0 ? hb[1] : 1), st);
    ps.istart.ensure(4 * (N + 1), st);
    ps.ideg.ensure(4 * (N + 1), st);
    ps.icol.ensure(4 * (size_t)(itot > 0 ? itot : 1), st);
    ps.iw.ensure(4 * (size_t)(itot > 0 ? itot : 1), st);
    k_int_fill<<<grid_for((long long)cnt * 32, 256), 256, 0, st>>>(
        cnt, M, rp, col, w, f.root, ps.ioff.as<int32_t>(), ps.istart.as<int32_t>(),
        ps.ideg.as<int32_t>(), ps.icol.as<int32_t>(), ps.iw.as<int32_t>());
    SLM_LAUNCH_CHECK();
    k_int_fill_big<<<long_row_blocks(cnt), 256, 0, st>>>(
        cnt, M, rp, col, w, f.root, ps.ioff.as<int32_t>(), ps.istart.as<int32_t>(),
        ps.ideg.as<int32_t>(), ps.icol.as<int32_t>(), ps.iw.as<int32_t>());
    SLM_LAUNCH_CHECK();
    // the rounds run in cooperative launches: a full grid while the member
    // lists are large, then a small grid for the tail of the rounds
    int dev = 0, sms = 0, per_sm = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    SLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_positive_rounds<NM, kPosThreads>,
                                                           kPosThreads, 0));
    // a one-block tail runs with kPosTailThreads threads when that block fits
    int per_sm_tail = 0;
    SLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_tail, k_positive_rounds<NM, kPosTailThreads>,
                                                           kPosTailThreads, 0));
    if (per_sm < 1) fail(SLM_ERR_CUDA, "POSITIVE kernel cannot be resident");
    const int nblocks_full = sms * std::min(per_sm, kPosBlocksPerSM);
    ps.bs.ensure(8 * (size_t)nblocks_full * 3, st);
    ps.ctrl.ensure(sizeof(PosCtrl), st);
    PosCtrl hc{};
    hc.cnt = cnt;
    hc.E = (int32_t)itot;  // bound on the first round's internal entries
    SLM_CUDA(cudaMemcpyAsync(ps.ctrl.get(), &hc, sizeof hc, cudaMemcpyHostToDevice, st));
    PosArgs<NM> A;
    A.n = n;
    A.istart = ps.istart.as<int32_t>();
    A.ideg = ps.ideg.as<int32_t>();
    A.icol = ps.icol.as<int32_t>();
    A.iw = ps.iw.as<int32_t>();
    A.s = s;
    A.m = m;
    A.a = a;
    A.root = f.root;
    A.entry = f.entry;
    A.depth = f.depth;
    A.cdist = f.cdist;
    A.oncycle = f.oncycle;
    A.sigma = sigma;
    A.flag = flag;
    A.kown = kown;
    A.listA = M;
    A.listB = M2;
    A.rlist = ps.rlist.as<int32_t>();
    A.posr = ps.posr.as<int32_t>();
    A.L = ps.L.as<int32_t>();
    A.coff = ps.coff.as<int32_t>();
    A.epref = ps.epref.as<int32_t>();
    A.mark = ps.mark.as<int32_t>();
    A.cyc = ps.cyc.as<int32_t>();
    A.msz = msz;
    A.subS = subS;
    A.subWA = subWA;
    A.subWin = subWin;
    A.credit = credit;
    A.TS = TS;
    A.bestsc = bestsc;
    A.kacc = ps.kacc.as<long long>();
    A.Mw = ps.pool.as<long long>();
    A.Mp = ps.pool2.as<long long>();
    A.bestkey = bestkey;
    A.cut = ps.cut.as<int4>();
    A.nf = ps.nf.as<int4>();
    A.noc = ps.noc.as<uint8_t>();
    A.recomp = ps.recomp.as<uint8_t>();
    A.moffN = ps.moffN.as<long long>();
    A.cutsum = ps.cutsum.as<long long>();
    A.coffN = ps.coffN.as<int32_t>();
    A.freshN = ps.freshN.as<int32_t>();
    A.cutpar = ps.cutpar.as<int32_t>();
    A.oldroot = ps.oldroot.as<int32_t>();
    A.splits_per_graph = splits_per_graph;
    A.bs64 = ps.bs.as<long long>();
    A.bs32a = reinterpret_cast<int32_t *>(ps.bs.as<long long>() + nblocks_full);
    A.bs32b = reinterpret_cast<int32_t *>(ps.bs.as<long long>() + 2 * nblocks_full);
    A.pool_cap = (long long)(hb[0] > 0 ? hb[0] : 1);
    A.cyc_cap = (long long)(hb[1] > 0 ? hb[1] : 1);
    A.max_rounds = (long long)n;  // every round splits at least one community
    A.ctrl = ps.ctrl.as<PosCtrl>();
    A.profile = ps.profile ? 1 : 0;
    A.bar = &A.ctrl->bar;
    A.barrier_ns = kBarrierLimitNs;
    const bool small_now = cnt <= kPosTailMembers && itot <= kPosTailEntries;
    for (int launch = 0; launch < 2; launch++) {
        const bool tail = small_now || launch == 1;
        A.first_round = launch == 0 ? 1 : 0;
        A.handoff_cnt = tail ? 0 : kPosTailMembers;
        A.handoff_edges = kPosTailEntries;
        const int nb = tail ? std::min(kPosTailBlocks, nblocks_full) : nblocks_full;
        const bool wide = nb == 1 && per_sm_tail >= 1;
        void *kargs[] = {&A};
        serialised_cooperative(st, [&] {
            if (wide)
                SLM_CUDA(cudaLaunchCooperativeKernel((const void *)k_positive_rounds<NM, kPosTailThreads>, dim3(1),
                                                     dim3(kPosTailThreads), kargs, 0, st));
            else
                SLM_CUDA(cudaLaunchCooperativeKernel((const void *)k_positive_rounds<NM, kPosThreads>, dim3(nb),
                                                     dim3(kPosThreads), kargs, 0, st));
            SLM_LAUNCH_CHECK();
        });
        SLM_CUDA(cudaMemcpyAsync(&hc, ps.ctrl.get(), sizeof hc, cudaMemcpyDeviceToHost, st));
        slm::stream_sync(st);
        if (tail || !hc.handoff || hc.error || hc.bar.failed) break;
        // continue from the list the full grid stopped on
        if (hc.list_b) std::swap(A.listA, A.listB);
        hc.handoff = 0;
        hc.bar = GridBarrier{};
        hc.R[0] = hc.R[1] = 0;  // the next launch sets up its first round afresh
        SLM_CUDA(cudaMemcpyAsync(ps.ctrl.get(), &hc, sizeof hc, cudaMemcpyHostToDevice, st));
    }
    if (hc.bar.failed) fail(SLM_ERR_TIMEOUT, "a POSITIVE grid barrier waited past its time limit");
    if (hc.error == 1) fail(SLM_ERR_TIMEOUT, "POSITIVE did not settle within n rounds");
    if (hc.error == 2) fail(SLM_ERR_CUDA, "POSITIVE cycle pools smaller than their bound");
    const long long splits = hc.splits, rounds = hc.rounds, visits = hc.visits;
    if (rounds_out) *rounds_out = rounds;
    if (visits_out) *visits_out = visits;
    if (ps.profile)
        for (int k = 0; k < kPosPhases; k++) ps.prof_ns[k] += hc.ph[k];
    return splits;
}

template long long positive_correct<NMSym>(int32_t, const int32_t *, const int32_t *,
                                          const int32_t *, const int32_t *, MParam, int32_t *,
                                          Forest &, int32_t *, const Buckets &,
                                          PositiveScratch &, cudaStream_t, long long *,
                                          long long *, int32_t *, const int32_t *);
template long long positive_correct<NMDir>(int32_t, const int32_t *, const int32_t *,
                                          const int32_t *, const unsigned long long *, MParam,
                                          int32_t *, Forest &, unsigned long long *,
                                          const Buckets &, PositiveScratch &, cudaStream_t,
                                          long long *, long long *, int32_t *, const int32_t *);

// ---------------------------------------------------------------------------
// Self-check of the grid barrier: `absent` (when >= 0) leaves before the first
// barrier, so the other blocks' waits run out after limit_ns.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_barrier_check(GridBarrier *b, int absent, long long limit_ns, int *passed) {
    if ((int)blockIdx.x == absent) return;
    for (int k = 0; k < 3; k++)
        if (!gbar(b, limit_ns)) return;
    if (threadIdx.x == 0) atomicAdd(passed, 1);
}
}  // namespace

bool barrier_check(int blocks, int absent, long long limit_ns, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    SLM_CUDA(cudaGetDevice(&dev));
    SLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_check, 128, 0));
    if (blocks < 1 || blocks > sms * per_sm) fail(SLM_ERR_INVALID_ARGUMENT, "block count not resident");
    DevBuf mem(sizeof(GridBarrier) + 16, st);
    SLM_CUDA(cudaMemsetAsync(mem.get(), 0, sizeof(GridBarrier) + 16, st));
    GridBarrier *b = mem.as<GridBarrier>();
    int *passed = reinterpret_cast<int *>(b + 1);
    void *kargs[] = {&b, &absent, &limit_ns, &passed};
    serialised_cooperative(st, [&] {
        SLM_CUDA(cudaLaunchCooperativeKernel((const void *)k_barrier_check, dim3(blocks), dim3(128),
                                             kargs, 0, st));
        SLM_LAUNCH_CHECK();
    });
    GridBarrier hb{};
    int hp = 0;
    SLM_CUDA(cudaMemcpyAsync(&hb, b, sizeof hb, cudaMemcpyDeviceToHost, st));
    SLM_CUDA(cudaMemcpyAsync(&hp, passed, sizeof hp, cudaMemcpyDeviceToHost, st));
    stream_sync(st);
    return hb.failed == 0 && hp == blocks;
}

}  // namespace slm
