/*
 * slm_oracle.c -- plain, slow, single-threaded CPU oracle of the Synchronised
 * Louvain Method (Chiem, Havelange, Van Dooren, "A parallel implementation of
 * the Synchronised Louvain Method", arXiv:1702.04645).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The library's product path
 * never calls it, links it or shares code with it.
 *
 * Every function follows one passage of the paper, cited beside it.  Where the
 * paper is silent or ambiguous the reading taken is stated at the function.
 * Graphs are symmetric CSR with int32 row pointers, sorted unique columns and
 * positive int32 weights; a self-loop W_ii is stored once.  With W symmetric,
 * the weighted modularity Q_w of Section 2.4 becomes
 *     Q = (1/m_w^2) * sum_C ( m_w * W_in(C) - Sigma_C^2 ),
 * with s_i = sum_j W_ij, m_w = sum_i s_i, Sigma_C = sum_{i in C} s_i and
 * W_in(C) = sum_{i,j in C} W_ij.  Every gain below is that numerator's change
 * divided by two, an exact int64 whenever m_w < 2^31.
 *
 * Random acceptance (Section 3.4, Algorithm MAXIMAL): the paper leaves the
 * probability p to Browet's thesis.  Reading: a parameter P in [0, 2^32];
 * node i at level t, sweep k is accepted iff
 *     (mix64(seed ^ mix64((t<<48) | (k<<32) | i)) >> 32) < P,
 * where mix64 is the splitmix64 output function (Steele, Lea, Flood 2014).
 *
 * The functions named ord_* at the end restate the method for a directed W
 * (Q_w with out- and in-strengths, Section 2.4), reusing the parts that do
 * not depend on the null model (components, tails, compaction, aggregation);
 * orc_louvain, last, is classical sequential-move Louvain for comparison.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int32_t i32;
typedef int64_t i64;
typedef uint64_t u64;

#define ORC_FLAG_NO_POSITIVE 1u

/* ------------------------------------------------------------------------- */
/* splitmix64 output function, written from its published definition.        */
/* ------------------------------------------------------------------------- */
u64 orc_mix64(u64 z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The 32-bit uniform draw p(i) of Algorithm MAXIMAL (reading above). */
uint32_t orc_draw(u64 seed, i32 level, i32 sweep, i32 i) {
    u64 ctr = ((u64)(uint32_t)level << 48) | ((u64)(uint32_t)sweep << 32) | (u64)(uint32_t)i;
    return (uint32_t)(orc_mix64(seed ^ orc_mix64(ctr)) >> 32);
}

/* ------------------------------------------------------------------------- */
/* Strengths s_i and total weight m_w (Section 2.4, definition of m_w).      */
/* ------------------------------------------------------------------------- */
i64 orc_strengths(i32 n, const i32 *rp, const i32 *col, const i32 *w, i64 *s) {
    i64 m = 0;
    for (i32 i = 0; i < n; i++) {
        i64 acc = 0;
        for (i32 p = rp[i]; p < rp[i + 1]; p++) acc += w[p];
        s[i] = acc;
        m += acc;
    }
    (void)col;
    return m;
}

/* ------------------------------------------------------------------------- */
/* Modularity (Section 2.4, Q_w) of a labelling, as the exact numerator      */
/* sum_C (m_w W_in(C) - Sigma_C^2) and the quotient by m_w^2.                */
/* labels take values in [0, n).                                             */
/* ------------------------------------------------------------------------- */
i64 orc_modularity_num(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i32 *labels) {
    i64 *s = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 *win = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 *sig = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 m = orc_strengths(n, rp, col, w, s);
    for (i32 u = 0; u < n; u++) {
        sig[labels[u]] += s[u];
        for (i32 p = rp[u]; p < rp[u + 1]; p++)
            if (labels[col[p]] == labels[u]) win[labels[u]] += w[p];
    }
    __int128 num = 0;
    for (i32 c = 0; c < n; c++)
        num += (__int128)m * win[c] - (__int128)sig[c] * sig[c];
    free(s); free(win); free(sig);
    return (i64)num; /* |num| <= m_w^2 < 2^62 */
}

double orc_modularity(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i32 *labels) {
    i64 m = 0;
    for (i32 p = 0; p < rp[n]; p++) m += w[p];
    if (m == 0) return 0.0;
    i64 num = orc_modularity_num(n, rp, col, w, labels);
    return (double)num / ((double)m * (double)m);
}

/* ------------------------------------------------------------------------- */
/* ASSIGN (Section 3.1, Algorithm ASSIGN): each node points at its best      */
/* neighbour.  From the all-singleton state, moving i into {j} changes the   */
/* numerator by 2 (m_w W_ij - s_i s_j).  Reading: self-assign when no        */
/* neighbour gives a strictly positive gain; ties go to the smallest j.      */
/* ------------------------------------------------------------------------- */
void orc_assign(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i64 *s, i64 m,
                i32 *a) {
    for (i32 i = 0; i < n; i++) {
        i32 bestj = -1;
        i64 bests = 0;
        for (i32 p = rp[i]; p < rp[i + 1]; p++) {
            i32 j = col[p];
            if (j == i) continue;
            i64 sc = m * (i64)w[p] - s[i] * s[j];
            if (bestj < 0 || sc > bests || (sc == bests && j < bestj)) {
                bestj = j;
                bests = sc;
            }
        }
        a[i] = (bestj >= 0 && bests > 0) ? bestj : i;
    }
}

/* ------------------------------------------------------------------------- */
/* COMPONENTS (Section 3.2, Algorithm ASSIGN's WCC): communities are the     */
/* weakly connected components of the assignment graph, each holding one     */
/* directed cycle.  Reading: a community is named by the smallest node id    */
/* on its cycle.  Linear-time walk with three colours.                      */
/* ------------------------------------------------------------------------- */
void orc_rootlabel(i32 n, const i32 *a, i32 *root) {
    unsigned char *state = (unsigned char *)calloc((size_t)n + 1, 1);
    i32 *stack = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    for (i32 v = 0; v < n; v++) {
        if (state[v] == 2) continue;
        i32 top = 0, x = v;
        while (state[x] == 0) {
            state[x] = 1;
            stack[top++] = x;
            x = a[x];
        }
        i32 r;
        if (state[x] == 1) {
            /* x lies on a cycle found in this walk: its name is the cycle minimum */
            r = x;
            for (i32 y = a[x]; y != x; y = a[y])
                if (y < r) r = y;
            root[x] = r;
            state[x] = 2;
            for (i32 y = a[x]; y != x; y = a[y]) { root[y] = r; state[y] = 2; }
        } else {
            r = root[x];
        }
        for (i32 k = 0; k < top; k++) {
            if (state[stack[k]] != 2) { root[stack[k]] = r; state[stack[k]] = 2; }
        }
    }
    free(state);
    free(stack);
}

/* Sigma_C = sum of s over the community named C (Section 2.4). */
void orc_sigma(i32 n, const i32 *root, const i64 *s, i64 *sigma) {
    for (i32 v = 0; v < n; v++) sigma[v] = 0;
    for (i32 v = 0; v < n; v++) sigma[root[v]] += s[v];
}

/* ------------------------------------------------------------------------- */
/* The per-node half of MAXIMAL (Section 3.4; Algorithm MAXIMAL's first      */
/* loop): best community c_i^* among the communities of i's neighbours, and  */
/* the local gain g(i) of Algorithm POSITIVE.  With k_{i,C} the weight from  */
/* i to C (self-loop excluded), score(C) = m_w k_{i,C} - s_i (Sigma_C -      */
/* [C = c_i] s_i); moving i from c_i to C changes the numerator by           */
/* 2 (score(C) - score(c_i)).  Reading: c_i^* differs from c_i only when its */
/* gain is strictly positive; ties go to the smallest community name.        */
/* ------------------------------------------------------------------------- */
void orc_scan(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i64 *s, i64 m,
              const i32 *root, const i64 *sigma, i32 *best, i64 *gain, i64 *g) {
    i64 *acc = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i32 *touched = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    for (i32 i = 0; i < n; i++) {
        i32 nt = 0, ci = root[i];
        for (i32 p = rp[i]; p < rp[i + 1]; p++) {
            i32 j = col[p];
            if (j == i) continue;
            i32 c = root[j];
            if (acc[c] == 0) touched[nt++] = c;
            acc[c] += w[p];
        }
        i64 own = m * acc[ci] - s[i] * (sigma[ci] - s[i]);
        i32 bc = -1;
        i64 bs = 0;
        for (i32 k = 0; k < nt; k++) {
            i32 c = touched[k];
            if (c == ci) continue;
            i64 sc = m * acc[c] - s[i] * sigma[c];
            if (bc < 0 || sc > bs || (sc == bs && c < bc)) { bc = c; bs = sc; }
        }
        for (i32 k = 0; k < nt; k++) acc[touched[k]] = 0;
        g[i] = own;
        if (bc >= 0 && bs - own > 0) { best[i] = bc; gain[i] = bs - own; }
        else { best[i] = ci; gain[i] = 0; }
    }
    free(acc);
    free(touched);
}

/* Children lists of the assignment graph (reverse of a, self-loops dropped). */
static void build_children(i32 n, const i32 *a, i32 *cp, i32 *ch) {
    for (i32 v = 0; v <= n; v++) cp[v] = 0;
    for (i32 v = 0; v < n; v++) if (a[v] != v) cp[a[v] + 1]++;
    for (i32 v = 0; v < n; v++) cp[v + 1] += cp[v];
    i32 *fill = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    memcpy(fill, cp, ((size_t)n + 1) * sizeof(i32));
    for (i32 v = 0; v < n; v++) if (a[v] != v) ch[fill[a[v]]++] = v;
    free(fill);
}

/* Tail of i (Section 3.4): every node with a directed path to i in the      */
/* assignment graph, plus i.  Reverse breadth-first search; returns size.    */
static i32 tail_of(i32 i, const i32 *cp, const i32 *ch, i32 *out, unsigned char *mark) {
    i32 head = 0, tl = 0;
    out[tl++] = i;
    mark[i] = 1;
    while (head < tl) {
        i32 x = out[head++];
        for (i32 k = cp[x]; k < cp[x + 1]; k++) {
            i32 y = ch[k];
            if (y >= 0 && !mark[y]) { mark[y] = 1; out[tl++] = y; }
        }
    }
    return tl;
}

/* ------------------------------------------------------------------------- */
/* Branch gain Delta H(c_i -> b(i) -> c_i^*) (Algorithm MAXIMAL): moving the */
/* tail S of i from A = c_i to B changes the numerator by twice              */
/*   m_w (W(S,B) - W(S, A\S)) - Sigma_S (Sigma_B - Sigma_A + Sigma_S).       */
/* ------------------------------------------------------------------------- */
static i64 branch_gain_impl(i32 i, i32 B, const i32 *rp, const i32 *col, const i32 *w,
                            const i64 *s, i64 m, const i32 *root, const i64 *sigma,
                            const i32 *cp, const i32 *ch, i32 *buf, unsigned char *mark) {
    i32 A = root[i];
    i32 k = tail_of(i, cp, ch, buf, mark);
    i64 sS = 0, wB = 0, wA = 0;
    for (i32 t = 0; t < k; t++) {
        i32 u = buf[t];
        sS += s[u];
        for (i32 p = rp[u]; p < rp[u + 1]; p++) {
            i32 v = col[p];
            if (root[v] == B) wB += w[p];
            else if (root[v] == A && !mark[v]) wA += w[p];
        }
    }
    for (i32 t = 0; t < k; t++) mark[buf[t]] = 0;
    return m * (wB - wA) - sS * (sigma[B] - sigma[A] + sS);
}

i64 orc_branch_gain(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i64 *s, i64 m,
                    const i32 *a, const i32 *root, const i64 *sigma, i32 i, i32 B) {
    i32 *cp = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *ch = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *buf = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    unsigned char *mark = (unsigned char *)calloc((size_t)n + 1, 1);
    build_children(n, a, cp, ch);
    i64 r = branch_gain_impl(i, B, rp, col, w, s, m, root, sigma, cp, ch, buf, mark);
    free(cp); free(ch); free(buf); free(mark);
    return r;
}

/* Target node (Algorithm MAXIMAL, update of a(i)): the neighbour j of i in  */
/* community B maximising m_w W_ij - s_i s_j.  Reading: ties go to the       */
/* smallest j; the maximum is taken even when negative.                      */
i32 orc_target(const i32 *rp, const i32 *col, const i32 *w, const i64 *s, i64 m,
               const i32 *root, i32 i, i32 B) {
    i32 bj = -1;
    i64 bs = 0;
    for (i32 p = rp[i]; p < rp[i + 1]; p++) {
        i32 j = col[p];
        if (j == i || root[j] != B) continue;
        i64 sc = m * (i64)w[p] - s[i] * s[j];
        if (bj < 0 || sc > bs || (sc == bs && j < bj)) { bj = j; bs = sc; }
    }
    return bj;
}

/* ------------------------------------------------------------------------- */
/* POSITIVE (Section 3.3, Algorithm POSITIVE).  The local gain of i is       */
/* g(i) = m_w k_{i,c_i} - s_i (Sigma_{c_i} - s_i).  A community holding a    */
/* node with g < 0 is bisected optimally, and the parts are examined again,  */
/* until no node has a negative local gain.  Candidate bisections:           */
/*   branch cut at a non-cycle node u: a(u) <- u, parts tail(u) and rest;    */
/*   cycle cut at two distinct cycle nodes u, v: a(u) <- u, a(v) <- v, each  */
/*   part being the nodes whose path reaches u (resp. v) first.              */
/* Splitting A into S and R changes the numerator by twice                   */
/*   Sigma_S Sigma_R - m_w W(S,R).                                           */
/* Readings: the best split is applied even when that value is not positive; */
/* ties prefer the larger value, then a branch cut over a cycle cut, then    */
/* the smaller u, then the smaller v.  Communities are independent (Section  */
/* 4.2), so the order in which they are examined does not matter.            */
/* ------------------------------------------------------------------------- */
typedef struct {
    i32 n;
    const i32 *rp, *col, *w;
    const i64 *s;
    i64 m;
    i32 *a, *root;
    /* scratch */
    i32 *cp, *ch, *buf, *entry, *cyc, *cidx, *stk;
    unsigned char *mark, *inpart, *oncyc, *state;
} pos_ctx;

/* Re-name the members of one community after its assignments changed. */
static void relabel_members(pos_ctx *c, const i32 *mem, i32 cnt) {
    /* the forward path of a member never leaves the member set */
    for (i32 k = 0; k < cnt; k++) c->state[mem[k]] = 0;
    for (i32 k = 0; k < cnt; k++) {
        i32 v = mem[k];
        if (c->state[v] == 2) continue;
        i32 top = 0, x = v;
        while (c->state[x] == 0) { c->state[x] = 1; c->stk[top++] = x; x = c->a[x]; }
        i32 r;
        if (c->state[x] == 1) {
            r = x;
            for (i32 y = c->a[x]; y != x; y = c->a[y]) if (y < r) r = y;
            c->root[x] = r; c->state[x] = 2;
            for (i32 y = c->a[x]; y != x; y = c->a[y]) { c->root[y] = r; c->state[y] = 2; }
        } else r = c->root[x];
        for (i32 t = 0; t < top; t++)
            if (c->state[c->stk[t]] != 2) { c->root[c->stk[t]] = r; c->state[c->stk[t]] = 2; }
    }
}

/* W(S, A\S) where S is marked in c->inpart and A is the community named A. */
static i64 cut_weight(pos_ctx *c, const i32 *S, i32 k, i32 A) {
    i64 tot = 0;
    for (i32 t = 0; t < k; t++) {
        i32 u = S[t];
        for (i32 p = c->rp[u]; p < c->rp[u + 1]; p++) {
            i32 v = c->col[p];
            if (c->root[v] == A && !c->inpart[v]) tot += c->w[p];
        }
    }
    return tot;
}

/* Remove x from the children list of its old parent (children lists are    */
/* kept consistent with a across splits).                                    */
static void drop_child(pos_ctx *c, i32 parent, i32 x) {
    for (i32 k = c->cp[parent]; k < c->cp[parent + 1]; k++)
        if (c->ch[k] == x) { c->ch[k] = -1; return; }
}

/* Examine one community (members mem[0..cnt)); split it if a member has a   */
/* negative local gain.  Returns 1 when split (mem reordered so that the     */
/* first *k1 members form one part), 0 otherwise.                            */
static int positive_one(pos_ctx *c, i32 *mem, i32 cnt, i32 *k1) {
    if (cnt < 2) return 0;
    i32 A = c->root[mem[0]];
    i64 sigA = 0;
    for (i32 t = 0; t < cnt; t++) sigA += c->s[mem[t]];
    int neg = 0;
    for (i32 t = 0; t < cnt && !neg; t++) {
        i32 i = mem[t];
        i64 kown = 0;
        for (i32 p = c->rp[i]; p < c->rp[i + 1]; p++) {
            i32 j = c->col[p];
            if (j != i && c->root[j] == A) kown += c->w[p];
        }
        i64 g = c->m * kown - c->s[i] * (sigA - c->s[i]);
        if (g < 0) neg = 1;
    }
    if (!neg) return 0;

    /* the cycle of the community, listed from its smallest node */
    i32 L = 0;
    {
        i32 x = mem[0];
        for (i32 t = 0; t < cnt; t++) c->mark[mem[t]] = 0;
        while (!c->mark[x]) { c->mark[x] = 1; x = c->a[x]; }
        i32 r = x;
        for (i32 y = c->a[x]; y != x; y = c->a[y]) if (y < r) r = y;
        i32 y = r;
        do { c->cyc[L] = y; c->cidx[y] = L; L++; y = c->a[y]; } while (y != r);
        for (i32 t = 0; t < cnt; t++) c->mark[mem[t]] = 0;
        for (i32 t = 0; t < cnt; t++) c->oncyc[mem[t]] = 0;
        for (i32 t = 0; t < L; t++) c->oncyc[c->cyc[t]] = 1;
    }

    int have = 0, btype = 0;
    i64 bscore = 0;
    i32 bu = -1, bv = -1;
#define ORC_BETTER(sc, ty, uu, vv) \
    (!have || (sc) > bscore || ((sc) == bscore && ((ty) < btype || ((ty) == btype && \
      ((uu) < bu || ((uu) == bu && (vv) < bv))))))

    /* branch cuts */
    for (i32 t = 0; t < cnt; t++) {
        i32 u = mem[t];
        if (c->oncyc[u]) continue;
        i32 k = tail_of(u, c->cp, c->ch, c->buf, c->inpart);
        i64 sS = 0;
        for (i32 q = 0; q < k; q++) sS += c->s[c->buf[q]];
        i64 cw = cut_weight(c, c->buf, k, A);
        for (i32 q = 0; q < k; q++) c->inpart[c->buf[q]] = 0;
        i64 sc = sS * (sigA - sS) - c->m * cw;
        if (ORC_BETTER(sc, 0, u, -1)) { have = 1; bscore = sc; btype = 0; bu = u; bv = -1; }
    }
    /* cycle cuts */
    if (L >= 2) {
        /* entry[v] = index of the first cycle node on v's path */
        for (i32 t = 0; t < cnt; t++) {
            i32 x = mem[t];
            while (!c->oncyc[x]) x = c->a[x];
            c->entry[mem[t]] = c->cidx[x];
        }
        for (i32 p = 0; p < L; p++) {
            for (i32 q = p + 1; q < L; q++) {
                /* part V: entries in (p, q] */
                i32 k = 0;
                i64 sV = 0;
                for (i32 t = 0; t < cnt; t++) {
                    i32 x = mem[t];
                    if (c->entry[x] > p && c->entry[x] <= q) {
                        c->buf[k++] = x; c->inpart[x] = 1; sV += c->s[x];
                    }
                }
                i64 cw = cut_weight(c, c->buf, k, A);
                for (i32 t = 0; t < k; t++) c->inpart[c->buf[t]] = 0;
                i64 sc = sV * (sigA - sV) - c->m * cw;
                i32 u = c->cyc[p] < c->cyc[q] ? c->cyc[p] : c->cyc[q];
                i32 v = c->cyc[p] < c->cyc[q] ? c->cyc[q] : c->cyc[p];
                if (ORC_BETTER(sc, 1, u, v)) { have = 1; bscore = sc; btype = 1; bu = u; bv = v; }
            }
        }
    }
#undef ORC_BETTER
    /* apply: the removed assignments become self-assignments */
    drop_child(c, c->a[bu], bu);
    c->a[bu] = bu;
    if (btype == 1) { drop_child(c, c->a[bv], bv); c->a[bv] = bv; }
    relabel_members(c, mem, cnt);
    /* reorder members: part of bu first */
    i32 r1 = c->root[bu];
    i32 lo = 0, hi = cnt - 1;
    while (lo <= hi) {
        if (c->root[mem[lo]] == r1) lo++;
        else { i32 tmp = mem[lo]; mem[lo] = mem[hi]; mem[hi] = tmp; hi--; }
    }
    *k1 = lo;
    return 1;
}

i32 orc_positive(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i64 *s, i64 m,
                 i32 *a, i32 *root) {
    pos_ctx c;
    c.n = n; c.rp = rp; c.col = col; c.w = w; c.s = s; c.m = m; c.a = a; c.root = root;
    size_t N = (size_t)n + 1;
    c.cp = (i32 *)malloc(N * sizeof(i32));
    c.ch = (i32 *)malloc(N * sizeof(i32));
    c.buf = (i32 *)malloc(N * sizeof(i32));
    c.entry = (i32 *)malloc(N * sizeof(i32));
    c.cyc = (i32 *)malloc(N * sizeof(i32));
    c.cidx = (i32 *)malloc(N * sizeof(i32));
    c.stk = (i32 *)malloc(N * sizeof(i32));
    c.mark = (unsigned char *)calloc(N, 1);
    c.inpart = (unsigned char *)calloc(N, 1);
    c.oncyc = (unsigned char *)calloc(N, 1);
    c.state = (unsigned char *)calloc(N, 1);
    build_children(n, a, c.cp, c.ch); /* entries set to -1 are removed children */
    /* members grouped by community name */
    i32 *mem = (i32 *)malloc(N * sizeof(i32));
    i32 *cnt = (i32 *)calloc(N, sizeof(i32));
    i32 *off = (i32 *)calloc(N + 1, sizeof(i32));
    for (i32 v = 0; v < n; v++) cnt[root[v]]++;
    for (i32 v = 0; v < n; v++) off[v + 1] = off[v] + cnt[v];
    for (i32 v = 0; v < n; v++) cnt[v] = 0;
    for (i32 v = 0; v < n; v++) mem[off[root[v]] + cnt[root[v]]++] = v;
    /* work list of member ranges */
    i32 *wl_off = (i32 *)malloc(2 * N * sizeof(i32));
    i32 *wl_len = (i32 *)malloc(2 * N * sizeof(i32));
    i32 nw = 0;
    for (i32 v = n - 1; v >= 0; v--)
        if (cnt[v] > 0) { wl_off[nw] = off[v]; wl_len[nw] = cnt[v]; nw++; }
    i32 splits = 0;
    while (nw > 0) {
        nw--;
        i32 o = wl_off[nw], l = wl_len[nw], k1 = 0;
        if (positive_one(&c, mem + o, l, &k1)) {
            splits++;
            wl_off[nw] = o; wl_len[nw] = k1; nw++;
            wl_off[nw] = o + k1; wl_len[nw] = l - k1; nw++;
        }
    }
    free(mem); free(cnt); free(off); free(wl_off); free(wl_len);
    free(c.cp); free(c.ch); free(c.buf); free(c.entry); free(c.cyc); free(c.cidx); free(c.stk);
    free(c.mark); free(c.inpart); free(c.oncyc); free(c.state);
    return splits;
}

/* ------------------------------------------------------------------------- */
/* Compaction of community names into ids 0..K-1, ordered by name (the       */
/* relabelling that AGGREGATE of Section 3.5 implies).                       */
/* ------------------------------------------------------------------------- */
i32 orc_compact(i32 n, const i32 *root, i32 *id) {
    i32 *rank = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 K = 0;
    for (i32 v = 0; v < n; v++) rank[v] = (root[v] == v) ? K++ : -1;
    for (i32 v = 0; v < n; v++) id[v] = rank[root[v]];
    free(rank);
    return K;
}

/* ------------------------------------------------------------------------- */
/* AGGREGATE (Section 3.5): each community becomes a super node; the weight  */
/* between super nodes A and B is the sum of W_uv over u in A, v in B, the   */
/* diagonal included, so strengths and m_w are preserved.  Output CSR with  */
/* sorted unique columns; returns nnz of the result.                          */
/* ------------------------------------------------------------------------- */
i32 orc_aggregate(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i32 *id, i32 K,
                  i32 *rp_out, i32 *col_out, i32 *w_out) {
    i64 *acc = (i64 *)calloc((size_t)K + 1, sizeof(i64));
    i32 *touched = (i32 *)malloc(((size_t)K + 1) * sizeof(i32));
    /* members of each super node */
    i32 *cnt = (i32 *)calloc((size_t)K + 1, sizeof(i32));
    i32 *off = (i32 *)calloc((size_t)K + 2, sizeof(i32));
    i32 *mem = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    for (i32 v = 0; v < n; v++) cnt[id[v]]++;
    for (i32 A = 0; A < K; A++) off[A + 1] = off[A] + cnt[A];
    for (i32 A = 0; A < K; A++) cnt[A] = 0;
    for (i32 v = 0; v < n; v++) mem[off[id[v]] + cnt[id[v]]++] = v;
    i32 nnz = 0;
    rp_out[0] = 0;
    for (i32 A = 0; A < K; A++) {
        i32 nt = 0;
        for (i32 t = off[A]; t < off[A + 1]; t++) {
            i32 u = mem[t];
            for (i32 p = rp[u]; p < rp[u + 1]; p++) {
                i32 B = id[col[p]];
                if (acc[B] == 0) touched[nt++] = B;
                acc[B] += w[p];
            }
        }
        /* sorted columns: insertion sort of the touched list */
        for (i32 x = 1; x < nt; x++) {
            i32 key = touched[x], y = x - 1;
            while (y >= 0 && touched[y] > key) { touched[y + 1] = touched[y]; y--; }
            touched[y + 1] = key;
        }
        for (i32 x = 0; x < nt; x++) {
            col_out[nnz] = touched[x];
            w_out[nnz] = (i32)acc[touched[x]];
            nnz++;
            acc[touched[x]] = 0;
        }
        rp_out[A + 1] = nnz;
    }
    free(acc); free(touched); free(cnt); free(off); free(mem);
    return nnz;
}

/* ------------------------------------------------------------------------- */
/* The whole method (Section 3, Algorithm 1).                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    i32 n0;
    i32 levels;
    i32 cap;
    i32 *level_n, *level_K;
    i32 **level_labels;
    i32 *final_labels;
    /* per level statistics */
    i32 *sweeps, *status; /* status: 0 converged, 1 stalled, 2 sweep limit */
    i64 *moves, *splits, *cands, *edges_scanned;
    /* per sweep trace: level, sweep, candidates, positive, accepted, splits */
    i64 *trace;
    i64 ntrace, trace_cap;
    int level_limit_hit;
    int top_status; /* sweep status of the last, unrecorded level */
    i32 top_sweeps;
} orc_run;

static void run_grow(orc_run *r) {
    if (r->levels < r->cap) return;
    r->cap = r->cap ? 2 * r->cap : 8;
    r->level_n = (i32 *)realloc(r->level_n, (size_t)r->cap * sizeof(i32));
    r->level_K = (i32 *)realloc(r->level_K, (size_t)r->cap * sizeof(i32));
    r->level_labels = (i32 **)realloc(r->level_labels, (size_t)r->cap * sizeof(i32 *));
    r->sweeps = (i32 *)realloc(r->sweeps, (size_t)r->cap * sizeof(i32));
    r->status = (i32 *)realloc(r->status, (size_t)r->cap * sizeof(i32));
    r->moves = (i64 *)realloc(r->moves, (size_t)r->cap * sizeof(i64));
    r->splits = (i64 *)realloc(r->splits, (size_t)r->cap * sizeof(i64));
    r->cands = (i64 *)realloc(r->cands, (size_t)r->cap * sizeof(i64));
    r->edges_scanned = (i64 *)realloc(r->edges_scanned, (size_t)r->cap * sizeof(i64));
}

static void trace_push(orc_run *r, i64 lv, i64 sw, i64 cand, i64 pos, i64 acc, i64 spl) {
    if (r->ntrace == r->trace_cap) {
        r->trace_cap = r->trace_cap ? 2 * r->trace_cap : 256;
        r->trace = (i64 *)realloc(r->trace, (size_t)r->trace_cap * 6 * sizeof(i64));
    }
    i64 *t = r->trace + 6 * r->ntrace++;
    t[0] = lv; t[1] = sw; t[2] = cand; t[3] = pos; t[4] = acc; t[5] = spl;
}

orc_run *orc_slm(i32 n0, const i32 *rp0, const i32 *col0, const i32 *w0, u64 seed, u64 P,
                 i32 max_sweeps, i32 max_levels, uint32_t flags) {
    orc_run *r = (orc_run *)calloc(1, sizeof(orc_run));
    r->n0 = n0;
    r->final_labels = (i32 *)malloc(((size_t)n0 + 1) * sizeof(i32));
    for (i32 v = 0; v < n0; v++) r->final_labels[v] = v;
    /* current level graph (owned copies) */
    i32 n = n0;
    i32 nnz = rp0[n0];
    i32 *rp = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *col = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    i32 *w = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    memcpy(rp, rp0, ((size_t)n + 1) * sizeof(i32));
    memcpy(col, col0, (size_t)nnz * sizeof(i32));
    memcpy(w, w0, (size_t)nnz * sizeof(i32));
    i32 t = 0;
    for (;;) {
        size_t N = (size_t)n + 1;
        i64 *s = (i64 *)malloc(N * sizeof(i64));
        i64 *sigma = (i64 *)malloc(N * sizeof(i64));
        i64 *gain = (i64 *)malloc(N * sizeof(i64));
        i64 *g = (i64 *)malloc(N * sizeof(i64));
        i64 *bg = (i64 *)malloc(N * sizeof(i64));
        i32 *a = (i32 *)malloc(N * sizeof(i32));
        i32 *root = (i32 *)malloc(N * sizeof(i32));
        i32 *best = (i32 *)malloc(N * sizeof(i32));
        i32 *tgt = (i32 *)malloc(N * sizeof(i32));
        i32 *cp = (i32 *)malloc(N * sizeof(i32));
        i32 *ch = (i32 *)malloc(N * sizeof(i32));
        i32 *buf = (i32 *)malloc(N * sizeof(i32));
        unsigned char *mark = (unsigned char *)calloc(N, 1);
        unsigned char *acc = (unsigned char *)calloc(N, 1);
        i64 m = orc_strengths(n, rp, col, w, s);

        /* ASSIGN, COMPONENTS, POSITIVE (Algorithm 1, first two lines of the loop) */
        orc_assign(n, rp, col, w, s, m, a);
        orc_rootlabel(n, a, root);
        i64 lv_splits = 0, lv_moves = 0, lv_cands = 0, lv_edges = 0;
        if (!(flags & ORC_FLAG_NO_POSITIVE)) lv_splits += orc_positive(n, rp, col, w, s, m, a, root);

        /* alternate MAXIMAL and POSITIVE while a positive move exists; on exit
           `sweep` counts the scans performed */
        i32 sweep = 0;
        int status = 2;
        for (; sweep < max_sweeps; sweep++) {
            orc_sigma(n, root, s, sigma);
            orc_scan(n, rp, col, w, s, m, root, sigma, best, gain, g);
            lv_edges += nnz;
            i64 ncand = 0, npos = 0, nacc = 0, nspl = 0;
            for (i32 i = 0; i < n; i++) if (gain[i] > 0) ncand++;
            lv_cands += ncand;
            if (ncand == 0) { status = 0; trace_push(r, t, sweep, 0, 0, 0, 0); sweep++; break; }
            build_children(n, a, cp, ch);
            for (i32 i = 0; i < n; i++) {
                acc[i] = 0;
                if (gain[i] <= 0) continue;
                bg[i] = branch_gain_impl(i, best[i], rp, col, w, s, m, root, sigma, cp, ch, buf, mark);
                if (bg[i] > 0) {
                    npos++;
                    if ((u64)orc_draw(seed, t, sweep, i) < P) acc[i] = 1;
                }
            }
            if (npos == 0) { status = 1; trace_push(r, t, sweep, ncand, 0, 0, 0); sweep++; break; }
            /* targets on the snapshot, then one synchronous write */
            for (i32 i = 0; i < n; i++)
                if (acc[i]) { tgt[i] = orc_target(rp, col, w, s, m, root, i, best[i]); nacc++; }
            for (i32 i = 0; i < n; i++) if (acc[i]) a[i] = tgt[i];
            lv_moves += nacc;
            if (nacc > 0) {
                orc_rootlabel(n, a, root);
                if (!(flags & ORC_FLAG_NO_POSITIVE)) nspl = orc_positive(n, rp, col, w, s, m, a, root);
                lv_splits += nspl;
            }
            trace_push(r, t, sweep, ncand, npos, nacc, nspl);
        }
        i32 *id = (i32 *)malloc(N * sizeof(i32));
        i32 K = orc_compact(n, root, id);
        free(s); free(sigma); free(gain); free(g); free(bg); free(a); free(root); free(best);
        free(tgt); free(cp); free(ch); free(buf); free(mark); free(acc);
        if (K == n) {
            /* no community structure left: stop without recording the level */
            r->top_status = status;
            r->top_sweeps = sweep;
            free(id);
            break;
        }
        run_grow(r);
        r->level_n[r->levels] = n;
        r->level_K[r->levels] = K;
        r->level_labels[r->levels] = id;
        r->sweeps[r->levels] = sweep;
        r->status[r->levels] = status;
        r->moves[r->levels] = lv_moves;
        r->splits[r->levels] = lv_splits;
        r->cands[r->levels] = lv_cands;
        r->edges_scanned[r->levels] = lv_edges;
        r->levels++;
        for (i32 v = 0; v < n0; v++) r->final_labels[v] = id[r->final_labels[v]];
        /* AGGREGATE */
        i32 *rp2 = (i32 *)malloc(((size_t)K + 1) * sizeof(i32));
        i32 *col2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 *w2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 nnz2 = orc_aggregate(n, rp, col, w, id, K, rp2, col2, w2);
        free(rp); free(col); free(w);
        rp = rp2; col = col2; w = w2; n = K; nnz = nnz2;
        t++;
        if (t >= max_levels) { r->level_limit_hit = 1; break; }
    }
    free(rp); free(col); free(w);
    return r;
}

/* accessors for the test harness */
i32 orc_run_levels(const orc_run *r) { return r->levels; }
i32 orc_run_level_n(const orc_run *r, i32 l) { return r->level_n[l]; }
i32 orc_run_level_K(const orc_run *r, i32 l) { return r->level_K[l]; }
void orc_run_level_labels(const orc_run *r, i32 l, i32 *out) {
    memcpy(out, r->level_labels[l], (size_t)r->level_n[l] * sizeof(i32));
}
void orc_run_final_labels(const orc_run *r, i32 *out) {
    memcpy(out, r->final_labels, (size_t)r->n0 * sizeof(i32));
}
/* stats: sweeps, status, moves, splits, candidates, edges scanned */
void orc_run_level_stats(const orc_run *r, i32 l, i64 *out6) {
    out6[0] = r->sweeps[l]; out6[1] = r->status[l]; out6[2] = r->moves[l];
    out6[3] = r->splits[l]; out6[4] = r->cands[l]; out6[5] = r->edges_scanned[l];
}
i64 orc_run_trace_len(const orc_run *r) { return r->ntrace; }
void orc_run_trace(const orc_run *r, i64 *out) {
    memcpy(out, r->trace, (size_t)r->ntrace * 6 * sizeof(i64));
}
void orc_run_top(const orc_run *r, i32 *out3) {
    out3[0] = r->top_status; out3[1] = r->top_sweeps; out3[2] = r->level_limit_hit;
}
void orc_run_free(orc_run *r) {
    if (!r) return;
    for (i32 l = 0; l < r->levels; l++) free(r->level_labels[l]);
    free(r->level_labels); free(r->level_n); free(r->level_K); free(r->final_labels);
    free(r->sweeps); free(r->status); free(r->moves); free(r->splits); free(r->cands);
    free(r->edges_scanned); free(r->trace);
    free(r);
}

/* ========================================================================= */
/* Directed graphs (Section 2.4: Q_w with out- and in-strengths).            */
/*                                                                           */
/* W is any non-negative integer matrix in CSR (row i lists W_ij > 0 with    */
/* sorted unique columns; W_ii stored once).  With s_i^out = sum_j W_ij,     */
/* s_j^in = sum_i W_ij and m_w = sum_ij W_ij the modularity numerator is     */
/*     sum_C ( m_w W_in(C) - Sigma_C^out Sigma_C^in ),  Q = num / m_w^2.     */
/* A move of a node or of a set S changes W_in by weights of U = W + W^T     */
/* (U(S,X) = W(S,X) + W(X,S)), and each null-model product s Sigma of the    */
/* symmetric functions above becomes s^out Sigma^in + s^in Sigma^out.  The   */
/* values below are the numerator's exact change (the symmetric functions    */
/* give half of it), so on a symmetric W each is twice the symmetric value   */
/* and every decision (argmax, sign, tie) is the same.  Exact in int64 when  */
/* m_w < 2^30.  The neighbours of a node are the nodes j with U_ij > 0.      */
/* ========================================================================= */

/* Out- and in-strengths of a directed CSR; returns m_w. */
i64 ord_strengths(i32 n, const i32 *rp, const i32 *col, const i32 *w, i64 *so, i64 *si) {
    for (i32 i = 0; i < n; i++) { so[i] = 0; si[i] = 0; }
    i64 m = 0;
    for (i32 i = 0; i < n; i++)
        for (i32 p = rp[i]; p < rp[i + 1]; p++) {
            so[i] += w[p];
            si[col[p]] += w[p];
            m += w[p];
        }
    return m;
}

/* U = W + W^T as a CSR with sorted unique columns (U_ii = 2 W_ii): row i of  */
/* W and row i of W^T (built by counting, so its columns ascend) are merged.  */
/* Output arrays hold up to 2 nnz(W) entries; returns nnz(U).                 */
i32 ord_symmetrise(i32 n, const i32 *rp, const i32 *col, const i32 *w, i32 *rpu, i32 *colu,
                   i32 *wu) {
    i32 nnz = rp[n];
    i32 *tp = (i32 *)calloc((size_t)n + 2, sizeof(i32));
    i32 *tc = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    i32 *tw = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    i32 *fill = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    for (i32 p = 0; p < nnz; p++) tp[col[p] + 1]++;
    for (i32 v = 0; v < n; v++) tp[v + 1] += tp[v];
    for (i32 v = 0; v < n; v++) fill[v] = tp[v];
    for (i32 i = 0; i < n; i++)
        for (i32 p = rp[i]; p < rp[i + 1]; p++) {
            i32 q = fill[col[p]]++;
            tc[q] = i;
            tw[q] = w[p];
        }
    i32 k = 0;
    rpu[0] = 0;
    for (i32 i = 0; i < n; i++) {
        i32 x = rp[i], y = tp[i];
        while (x < rp[i + 1] || y < tp[i + 1]) {
            if (y >= tp[i + 1] || (x < rp[i + 1] && col[x] < tc[y])) {
                colu[k] = col[x]; wu[k] = w[x]; x++;
            } else if (x >= rp[i + 1] || tc[y] < col[x]) {
                colu[k] = tc[y]; wu[k] = tw[y]; y++;
            } else {
                colu[k] = col[x]; wu[k] = w[x] + tw[y]; x++; y++;
            }
            k++;
        }
        rpu[i + 1] = k;
    }
    free(tp); free(tc); free(tw); free(fill);
    return k;
}

/* Modularity numerator of a labelling on a directed W (definition above). */
i64 ord_modularity_num(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i32 *labels) {
    i64 *so = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 *si = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 *win = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 *go = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 *gi = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i64 m = ord_strengths(n, rp, col, w, so, si);
    for (i32 u = 0; u < n; u++) {
        go[labels[u]] += so[u];
        gi[labels[u]] += si[u];
        for (i32 p = rp[u]; p < rp[u + 1]; p++)
            if (labels[col[p]] == labels[u]) win[labels[u]] += w[p];
    }
    __int128 num = 0;
    for (i32 c = 0; c < n; c++) num += (__int128)m * win[c] - (__int128)go[c] * gi[c];
    free(so); free(si); free(win); free(go); free(gi);
    return (i64)num; /* |num| <= m_w^2 */
}

double ord_modularity(i32 n, const i32 *rp, const i32 *col, const i32 *w, const i32 *labels) {
    i64 m = 0;
    for (i32 p = 0; p < rp[n]; p++) m += w[p];
    if (m == 0) return 0.0;
    return (double)ord_modularity_num(n, rp, col, w, labels) / ((double)m * (double)m);
}

/* Pair score of i joining the singleton {j} (ASSIGN, target): the change of  */
/* the numerator from the all-singleton state.                               */
static i64 ord_pair(i64 m, i64 uij, const i64 *so, const i64 *si, i32 i, i32 j) {
    return m * uij - (so[i] * si[j] + si[i] * so[j]);
}

/* ASSIGN (Section 3.1) on a directed graph, over the rows of U. */
void ord_assign(i32 n, const i32 *rpu, const i32 *colu, const i32 *wu, const i64 *so,
                const i64 *si, i64 m, i32 *a) {
    for (i32 i = 0; i < n; i++) {
        i32 bestj = -1;
        i64 bests = 0;
        for (i32 p = rpu[i]; p < rpu[i + 1]; p++) {
            i32 j = colu[p];
            if (j == i) continue;
            i64 sc = ord_pair(m, wu[p], so, si, i, j);
            if (bestj < 0 || sc > bests || (sc == bests && j < bestj)) { bestj = j; bests = sc; }
        }
        a[i] = (bestj >= 0 && bests > 0) ? bestj : i;
    }
}

/* Sigma_C^out and Sigma_C^in of the communities named by root. */
void ord_sigma(i32 n, const i32 *root, const i64 *so, const i64 *si, i64 *go, i64 *gi) {
    for (i32 v = 0; v < n; v++) { go[v] = 0; gi[v] = 0; }
    for (i32 v = 0; v < n; v++) { go[root[v]] += so[v]; gi[root[v]] += si[v]; }
}

/* MAXIMAL's per-node half (Section 3.4) on a directed graph.  With k_{i,C}  */
/* the U-weight between i and C (self-loop excluded),                        */
/*   score(C) = m_w k_{i,C} - (s_i^out (Sigma_C^in - [C = c_i] s_i^in)       */
/*                             + s_i^in (Sigma_C^out - [C = c_i] s_i^out)),  */
/* and moving i from c_i to C changes the numerator by score(C) - score(c_i);*/
/* g(i) = score(c_i).  Readings as in orc_scan.                              */
void ord_scan(i32 n, const i32 *rpu, const i32 *colu, const i32 *wu, const i64 *so,
              const i64 *si, i64 m, const i32 *root, const i64 *go, const i64 *gi, i32 *best,
              i64 *gain, i64 *g) {
    i64 *acc = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    i32 *touched = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    for (i32 i = 0; i < n; i++) {
        i32 nt = 0, ci = root[i];
        for (i32 p = rpu[i]; p < rpu[i + 1]; p++) {
            i32 j = colu[p];
            if (j == i) continue;
            i32 c = root[j];
            if (acc[c] == 0) touched[nt++] = c;
            acc[c] += wu[p];
        }
        i64 own = m * acc[ci] - (so[i] * (gi[ci] - si[i]) + si[i] * (go[ci] - so[i]));
        i32 bc = -1;
        i64 bs = 0;
        for (i32 k = 0; k < nt; k++) {
            i32 c = touched[k];
            if (c == ci) continue;
            i64 sc = m * acc[c] - (so[i] * gi[c] + si[i] * go[c]);
            if (bc < 0 || sc > bs || (sc == bs && c < bc)) { bc = c; bs = sc; }
        }
        for (i32 k = 0; k < nt; k++) acc[touched[k]] = 0;
        g[i] = own;
        if (bc >= 0 && bs - own > 0) { best[i] = bc; gain[i] = bs - own; }
        else { best[i] = ci; gain[i] = 0; }
    }
    free(acc);
    free(touched);
}

/* Branch gain on a directed graph: moving the tail S of i from A = c_i to B */
/* changes the numerator by                                                  */
/*   m_w (U(S,B) - U(S,A\S)) - (Sigma_S^out (Sigma_B^in - Sigma_A^in + Sigma_S^in)   */
/*                              + Sigma_S^in (Sigma_B^out - Sigma_A^out + Sigma_S^out)). */
static i64 ord_branch_gain_impl(i32 i, i32 B, const i32 *rpu, const i32 *colu, const i32 *wu,
                                const i64 *so, const i64 *si, i64 m, const i32 *root,
                                const i64 *go, const i64 *gi, const i32 *cp, const i32 *ch,
                                i32 *buf, unsigned char *mark) {
    i32 A = root[i];
    i32 k = tail_of(i, cp, ch, buf, mark);
    i64 sSo = 0, sSi = 0, uB = 0, uA = 0;
    for (i32 t = 0; t < k; t++) {
        i32 u = buf[t];
        sSo += so[u];
        sSi += si[u];
        for (i32 p = rpu[u]; p < rpu[u + 1]; p++) {
            i32 v = colu[p];
            if (root[v] == B) uB += wu[p];
            else if (root[v] == A && !mark[v]) uA += wu[p];
        }
    }
    for (i32 t = 0; t < k; t++) mark[buf[t]] = 0;
    return m * (uB - uA) - (sSo * (gi[B] - gi[A] + sSi) + sSi * (go[B] - go[A] + sSo));
}

i64 ord_branch_gain(i32 n, const i32 *rpu, const i32 *colu, const i32 *wu, const i64 *so,
                    const i64 *si, i64 m, const i32 *a, const i32 *root, const i64 *go,
                    const i64 *gi, i32 i, i32 B) {
    i32 *cp = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *ch = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *buf = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    unsigned char *mark = (unsigned char *)calloc((size_t)n + 1, 1);
    build_children(n, a, cp, ch);
    i64 r = ord_branch_gain_impl(i, B, rpu, colu, wu, so, si, m, root, go, gi, cp, ch, buf, mark);
    free(cp); free(ch); free(buf); free(mark);
    return r;
}

/* Target node on a directed graph: the U-neighbour j of i in B with the      */
/* largest pair score; ties to the smallest j, taken even when negative.     */
i32 ord_target(const i32 *rpu, const i32 *colu, const i32 *wu, const i64 *so, const i64 *si,
               i64 m, const i32 *root, i32 i, i32 B) {
    i32 bj = -1;
    i64 bs = 0;
    for (i32 p = rpu[i]; p < rpu[i + 1]; p++) {
        i32 j = colu[p];
        if (j == i || root[j] != B) continue;
        i64 sc = ord_pair(m, wu[p], so, si, i, j);
        if (bj < 0 || sc > bs || (sc == bs && j < bj)) { bj = j; bs = sc; }
    }
    return bj;
}

/* POSITIVE (Section 3.3) on a directed graph: local gain g(i) = score(c_i)  */
/* of ord_scan; splitting A into S and R changes the numerator by            */
/*   Sigma_S^out Sigma_R^in + Sigma_S^in Sigma_R^out - m_w U(S,R).           */
/* Candidate cuts, readings and tie order as in orc_positive.  The context's */
/* graph is U and its strengths are s^out; s^in travels beside it.           */
typedef struct {
    pos_ctx b;
    const i64 *si;
} pos_ctx_d;

static int ord_positive_one(pos_ctx_d *d, i32 *mem, i32 cnt, i32 *k1) {
    pos_ctx *c = &d->b;
    const i64 *so = c->s, *si = d->si;
    if (cnt < 2) return 0;
    i32 A = c->root[mem[0]];
    i64 sAo = 0, sAi = 0;
    for (i32 t = 0; t < cnt; t++) { sAo += so[mem[t]]; sAi += si[mem[t]]; }
    int neg = 0;
    for (i32 t = 0; t < cnt && !neg; t++) {
        i32 i = mem[t];
        i64 kown = 0;
        for (i32 p = c->rp[i]; p < c->rp[i + 1]; p++) {
            i32 j = c->col[p];
            if (j != i && c->root[j] == A) kown += c->w[p];
        }
        i64 g = c->m * kown - (so[i] * (sAi - si[i]) + si[i] * (sAo - so[i]));
        if (g < 0) neg = 1;
    }
    if (!neg) return 0;

    i32 L = 0;
    {
        i32 x = mem[0];
        for (i32 t = 0; t < cnt; t++) c->mark[mem[t]] = 0;
        while (!c->mark[x]) { c->mark[x] = 1; x = c->a[x]; }
        i32 r = x;
        for (i32 y = c->a[x]; y != x; y = c->a[y]) if (y < r) r = y;
        i32 y = r;
        do { c->cyc[L] = y; c->cidx[y] = L; L++; y = c->a[y]; } while (y != r);
        for (i32 t = 0; t < cnt; t++) c->mark[mem[t]] = 0;
        for (i32 t = 0; t < cnt; t++) c->oncyc[mem[t]] = 0;
        for (i32 t = 0; t < L; t++) c->oncyc[c->cyc[t]] = 1;
    }

    int have = 0, btype = 0;
    i64 bscore = 0;
    i32 bu = -1, bv = -1;
#define ORD_BETTER(sc, ty, uu, vv) \
    (!have || (sc) > bscore || ((sc) == bscore && ((ty) < btype || ((ty) == btype && \
      ((uu) < bu || ((uu) == bu && (vv) < bv))))))

    for (i32 t = 0; t < cnt; t++) {
        i32 u = mem[t];
        if (c->oncyc[u]) continue;
        i32 k = tail_of(u, c->cp, c->ch, c->buf, c->inpart);
        i64 sSo = 0, sSi = 0;
        for (i32 q = 0; q < k; q++) { sSo += so[c->buf[q]]; sSi += si[c->buf[q]]; }
        i64 cw = cut_weight(c, c->buf, k, A);
        for (i32 q = 0; q < k; q++) c->inpart[c->buf[q]] = 0;
        i64 sc = sSo * (sAi - sSi) + sSi * (sAo - sSo) - c->m * cw;
        if (ORD_BETTER(sc, 0, u, -1)) { have = 1; bscore = sc; btype = 0; bu = u; bv = -1; }
    }
    if (L >= 2) {
        for (i32 t = 0; t < cnt; t++) {
            i32 x = mem[t];
            while (!c->oncyc[x]) x = c->a[x];
            c->entry[mem[t]] = c->cidx[x];
        }
        for (i32 p = 0; p < L; p++) {
            for (i32 q = p + 1; q < L; q++) {
                i32 k = 0;
                i64 sVo = 0, sVi = 0;
                for (i32 t = 0; t < cnt; t++) {
                    i32 x = mem[t];
                    if (c->entry[x] > p && c->entry[x] <= q) {
                        c->buf[k++] = x; c->inpart[x] = 1; sVo += so[x]; sVi += si[x];
                    }
                }
                i64 cw = cut_weight(c, c->buf, k, A);
                for (i32 t = 0; t < k; t++) c->inpart[c->buf[t]] = 0;
                i64 sc = sVo * (sAi - sVi) + sVi * (sAo - sVo) - c->m * cw;
                i32 u = c->cyc[p] < c->cyc[q] ? c->cyc[p] : c->cyc[q];
                i32 v = c->cyc[p] < c->cyc[q] ? c->cyc[q] : c->cyc[p];
                if (ORD_BETTER(sc, 1, u, v)) { have = 1; bscore = sc; btype = 1; bu = u; bv = v; }
            }
        }
    }
#undef ORD_BETTER
    drop_child(c, c->a[bu], bu);
    c->a[bu] = bu;
    if (btype == 1) { drop_child(c, c->a[bv], bv); c->a[bv] = bv; }
    relabel_members(c, mem, cnt);
    i32 r1 = c->root[bu];
    i32 lo = 0, hi = cnt - 1;
    while (lo <= hi) {
        if (c->root[mem[lo]] == r1) lo++;
        else { i32 tmp = mem[lo]; mem[lo] = mem[hi]; mem[hi] = tmp; hi--; }
    }
    *k1 = lo;
    return 1;
}

i32 ord_positive(i32 n, const i32 *rpu, const i32 *colu, const i32 *wu, const i64 *so,
                 const i64 *si, i64 m, i32 *a, i32 *root) {
    pos_ctx_d d;
    pos_ctx *c = &d.b;
    d.si = si;
    c->n = n; c->rp = rpu; c->col = colu; c->w = wu; c->s = so; c->m = m; c->a = a; c->root = root;
    size_t N = (size_t)n + 1;
    c->cp = (i32 *)malloc(N * sizeof(i32));
    c->ch = (i32 *)malloc(N * sizeof(i32));
    c->buf = (i32 *)malloc(N * sizeof(i32));
    c->entry = (i32 *)malloc(N * sizeof(i32));
    c->cyc = (i32 *)malloc(N * sizeof(i32));
    c->cidx = (i32 *)malloc(N * sizeof(i32));
    c->stk = (i32 *)malloc(N * sizeof(i32));
    c->mark = (unsigned char *)calloc(N, 1);
    c->inpart = (unsigned char *)calloc(N, 1);
    c->oncyc = (unsigned char *)calloc(N, 1);
    c->state = (unsigned char *)calloc(N, 1);
    build_children(n, a, c->cp, c->ch);
    i32 *mem = (i32 *)malloc(N * sizeof(i32));
    i32 *cnt = (i32 *)calloc(N, sizeof(i32));
    i32 *off = (i32 *)calloc(N + 1, sizeof(i32));
    for (i32 v = 0; v < n; v++) cnt[root[v]]++;
    for (i32 v = 0; v < n; v++) off[v + 1] = off[v] + cnt[v];
    for (i32 v = 0; v < n; v++) cnt[v] = 0;
    for (i32 v = 0; v < n; v++) mem[off[root[v]] + cnt[root[v]]++] = v;
    i32 *wl_off = (i32 *)malloc(2 * N * sizeof(i32));
    i32 *wl_len = (i32 *)malloc(2 * N * sizeof(i32));
    i32 nw = 0;
    for (i32 v = n - 1; v >= 0; v--)
        if (cnt[v] > 0) { wl_off[nw] = off[v]; wl_len[nw] = cnt[v]; nw++; }
    i32 splits = 0;
    while (nw > 0) {
        nw--;
        i32 o = wl_off[nw], l = wl_len[nw], k1 = 0;
        if (ord_positive_one(&d, mem + o, l, &k1)) {
            splits++;
            wl_off[nw] = o; wl_len[nw] = k1; nw++;
            wl_off[nw] = o + k1; wl_len[nw] = l - k1; nw++;
        }
    }
    free(mem); free(cnt); free(off); free(wl_off); free(wl_len);
    free(c->cp); free(c->ch); free(c->buf); free(c->entry); free(c->cyc); free(c->cidx);
    free(c->stk); free(c->mark); free(c->inpart); free(c->oncyc); free(c->state);
    return splits;
}

/* The whole method (Algorithm 1) on a directed graph: every level works on  */
/* U = W + W^T with the strengths of W; AGGREGATE sums W itself (orc_aggregate */
/* makes no use of symmetry), so out- and in-strengths and m_w are kept.     */
/* Stats and trace as in orc_slm; entries scanned count the entries of U.    */
orc_run *ord_slm(i32 n0, const i32 *rp0, const i32 *col0, const i32 *w0, u64 seed, u64 P,
                 i32 max_sweeps, i32 max_levels, uint32_t flags) {
    orc_run *r = (orc_run *)calloc(1, sizeof(orc_run));
    r->n0 = n0;
    r->final_labels = (i32 *)malloc(((size_t)n0 + 1) * sizeof(i32));
    for (i32 v = 0; v < n0; v++) r->final_labels[v] = v;
    i32 n = n0;
    i32 nnz = rp0[n0];
    i32 *rp = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *col = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    i32 *w = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    memcpy(rp, rp0, ((size_t)n + 1) * sizeof(i32));
    memcpy(col, col0, (size_t)nnz * sizeof(i32));
    memcpy(w, w0, (size_t)nnz * sizeof(i32));
    i32 t = 0;
    for (;;) {
        size_t N = (size_t)n + 1;
        i32 *rpu = (i32 *)malloc(N * sizeof(i32));
        i32 *colu = (i32 *)malloc((2 * (size_t)nnz + 1) * sizeof(i32));
        i32 *wu = (i32 *)malloc((2 * (size_t)nnz + 1) * sizeof(i32));
        i32 nnzu = ord_symmetrise(n, rp, col, w, rpu, colu, wu);
        i64 *so = (i64 *)malloc(N * sizeof(i64));
        i64 *si = (i64 *)malloc(N * sizeof(i64));
        i64 *go = (i64 *)malloc(N * sizeof(i64));
        i64 *gi = (i64 *)malloc(N * sizeof(i64));
        i64 *gain = (i64 *)malloc(N * sizeof(i64));
        i64 *g = (i64 *)malloc(N * sizeof(i64));
        i64 *bg = (i64 *)malloc(N * sizeof(i64));
        i32 *a = (i32 *)malloc(N * sizeof(i32));
        i32 *root = (i32 *)malloc(N * sizeof(i32));
        i32 *best = (i32 *)malloc(N * sizeof(i32));
        i32 *tgt = (i32 *)malloc(N * sizeof(i32));
        i32 *cp = (i32 *)malloc(N * sizeof(i32));
        i32 *ch = (i32 *)malloc(N * sizeof(i32));
        i32 *buf = (i32 *)malloc(N * sizeof(i32));
        unsigned char *mark = (unsigned char *)calloc(N, 1);
        unsigned char *acc = (unsigned char *)calloc(N, 1);
        i64 m = ord_strengths(n, rp, col, w, so, si);

        ord_assign(n, rpu, colu, wu, so, si, m, a);
        orc_rootlabel(n, a, root);
        i64 lv_splits = 0, lv_moves = 0, lv_cands = 0, lv_edges = 0;
        if (!(flags & ORC_FLAG_NO_POSITIVE))
            lv_splits += ord_positive(n, rpu, colu, wu, so, si, m, a, root);

        i32 sweep = 0;
        int status = 2;
        for (; sweep < max_sweeps; sweep++) {
            ord_sigma(n, root, so, si, go, gi);
            ord_scan(n, rpu, colu, wu, so, si, m, root, go, gi, best, gain, g);
            lv_edges += nnzu;
            i64 ncand = 0, npos = 0, nacc = 0, nspl = 0;
            for (i32 i = 0; i < n; i++) if (gain[i] > 0) ncand++;
            lv_cands += ncand;
            if (ncand == 0) { status = 0; trace_push(r, t, sweep, 0, 0, 0, 0); sweep++; break; }
            build_children(n, a, cp, ch);
            for (i32 i = 0; i < n; i++) {
                acc[i] = 0;
                if (gain[i] <= 0) continue;
                bg[i] = ord_branch_gain_impl(i, best[i], rpu, colu, wu, so, si, m, root, go, gi,
                                             cp, ch, buf, mark);
                if (bg[i] > 0) {
                    npos++;
                    if ((u64)orc_draw(seed, t, sweep, i) < P) acc[i] = 1;
                }
            }
            if (npos == 0) { status = 1; trace_push(r, t, sweep, ncand, 0, 0, 0); sweep++; break; }
            for (i32 i = 0; i < n; i++)
                if (acc[i]) { tgt[i] = ord_target(rpu, colu, wu, so, si, m, root, i, best[i]); nacc++; }
            for (i32 i = 0; i < n; i++) if (acc[i]) a[i] = tgt[i];
            lv_moves += nacc;
            if (nacc > 0) {
                orc_rootlabel(n, a, root);
                if (!(flags & ORC_FLAG_NO_POSITIVE))
                    nspl = ord_positive(n, rpu, colu, wu, so, si, m, a, root);
                lv_splits += nspl;
            }
            trace_push(r, t, sweep, ncand, npos, nacc, nspl);
        }
        i32 *id = (i32 *)malloc(N * sizeof(i32));
        i32 K = orc_compact(n, root, id);
        free(rpu); free(colu); free(wu); free(so); free(si); free(go); free(gi); free(gain);
        free(g); free(bg); free(a); free(root); free(best); free(tgt); free(cp); free(ch);
        free(buf); free(mark); free(acc);
        if (K == n) {
            r->top_status = status;
            r->top_sweeps = sweep;
            free(id);
            break;
        }
        run_grow(r);
        r->level_n[r->levels] = n;
        r->level_K[r->levels] = K;
        r->level_labels[r->levels] = id;
        r->sweeps[r->levels] = sweep;
        r->status[r->levels] = status;
        r->moves[r->levels] = lv_moves;
        r->splits[r->levels] = lv_splits;
        r->cands[r->levels] = lv_cands;
        r->edges_scanned[r->levels] = lv_edges;
        r->levels++;
        for (i32 v = 0; v < n0; v++) r->final_labels[v] = id[r->final_labels[v]];
        i32 *rp2 = (i32 *)malloc(((size_t)K + 1) * sizeof(i32));
        i32 *col2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 *w2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 nnz2 = orc_aggregate(n, rp, col, w, id, K, rp2, col2, w2);
        free(rp); free(col); free(w);
        rp = rp2; col = col2; w = w2; n = K; nnz = nnz2;
        t++;
        if (t >= max_levels) { r->level_limit_hit = 1; break; }
    }
    free(rp); free(col); free(w);
    return r;
}

/* ========================================================================= */
/* Classical (sequential-move) Louvain, the method the paper builds on and   */
/* names for comparison in its conclusion (Section 6).  Restated from its    */
/* published definition (Blondel, Guillaume, Lambiotte, Lefebvre 2008) on    */
/* the symmetric W above: per level, nodes are visited one at a time in id   */
/* order; node i leaves its community A and joins the community C holding a  */
/* neighbour for which the numerator's change, twice                         */
/*   (m_w k_{i,C} - s_i Sigma_C) - (m_w k_{i,A} - s_i (Sigma_A - s_i)),      */
/* is largest, only when that change is strictly positive (else it stays).  */
/* Readings: ties go to the smallest community name (names are node ids of  */
/* the level graph, a community keeps the name it started with); passes     */
/* repeat until one moves no node; a level whose first pass moves nothing,  */
/* or that ends with every node alone, ends the run; otherwise the          */
/* communities are compacted in name order and aggregated (Section 3.5).    */
/* Stats per level: sweeps = passes, moves = node moves, edges scanned =    */
/* passes x entries; the trace holds (level, pass, 0, 0, moves, 0).         */
/* ========================================================================= */
orc_run *orc_louvain(i32 n0, const i32 *rp0, const i32 *col0, const i32 *w0, i32 max_passes,
                     i32 max_levels) {
    orc_run *r = (orc_run *)calloc(1, sizeof(orc_run));
    r->n0 = n0;
    r->final_labels = (i32 *)malloc(((size_t)n0 + 1) * sizeof(i32));
    for (i32 v = 0; v < n0; v++) r->final_labels[v] = v;
    i32 n = n0;
    i32 nnz = rp0[n0];
    i32 *rp = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *col = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    i32 *w = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    memcpy(rp, rp0, ((size_t)n + 1) * sizeof(i32));
    memcpy(col, col0, (size_t)nnz * sizeof(i32));
    memcpy(w, w0, (size_t)nnz * sizeof(i32));
    i32 t = 0;
    for (;;) {
        size_t N = (size_t)n + 1;
        i64 *s = (i64 *)malloc(N * sizeof(i64));
        i64 *sigma = (i64 *)calloc(N, sizeof(i64));
        i64 *acc = (i64 *)calloc(N, sizeof(i64));
        i32 *touched = (i32 *)malloc(N * sizeof(i32));
        i32 *comm = (i32 *)malloc(N * sizeof(i32));
        unsigned char *seen = (unsigned char *)calloc(N, 1);
        i64 m = orc_strengths(n, rp, col, w, s);
        for (i32 v = 0; v < n; v++) { comm[v] = v; sigma[v] = s[v]; }
        i32 passes = 0;
        i64 lv_moves = 0, first_moves = 0;
        while (passes < max_passes) {
            i64 moves = 0;
            for (i32 i = 0; i < n; i++) {
                i32 A = comm[i], nt = 0;
                for (i32 p = rp[i]; p < rp[i + 1]; p++) {
                    i32 j = col[p];
                    if (j == i) continue;
                    i32 c = comm[j];
                    if (!seen[c]) { seen[c] = 1; touched[nt++] = c; }
                    acc[c] += w[p];
                }
                i64 stay = m * acc[A] - s[i] * (sigma[A] - s[i]);
                i32 bc = -1;
                i64 bd = 0;
                for (i32 k = 0; k < nt; k++) {
                    i32 c = touched[k];
                    if (c == A) continue;
                    i64 d = (m * acc[c] - s[i] * sigma[c]) - stay;
                    if (d > 0 && (bc < 0 || d > bd || (d == bd && c < bc))) { bc = c; bd = d; }
                }
                for (i32 k = 0; k < nt; k++) { acc[touched[k]] = 0; seen[touched[k]] = 0; }
                if (bc >= 0) {
                    sigma[A] -= s[i];
                    sigma[bc] += s[i];
                    comm[i] = bc;
                    moves++;
                }
            }
            passes++;
            lv_moves += moves;
            if (passes == 1) first_moves = moves;
            trace_push(r, t, passes - 1, 0, 0, moves, 0);
            if (moves == 0) break;
        }
        /* compaction in name order */
        i32 *id = (i32 *)malloc(N * sizeof(i32));
        i32 *rank = (i32 *)malloc(N * sizeof(i32));
        for (i32 v = 0; v < n; v++) rank[v] = -1;
        for (i32 v = 0; v < n; v++) rank[comm[v]] = 0;
        i32 K = 0;
        for (i32 v = 0; v < n; v++) if (rank[v] == 0) rank[v] = ++K;
        for (i32 v = 0; v < n; v++) id[v] = rank[comm[v]] - 1;
        free(rank); free(s); free(sigma); free(acc); free(touched); free(comm); free(seen);
        if (first_moves == 0 || K == n) {
            r->top_status = 0;
            r->top_sweeps = passes;
            free(id);
            break;
        }
        run_grow(r);
        r->level_n[r->levels] = n;
        r->level_K[r->levels] = K;
        r->level_labels[r->levels] = id;
        r->sweeps[r->levels] = passes;
        r->status[r->levels] = 0;
        r->moves[r->levels] = lv_moves;
        r->splits[r->levels] = 0;
        r->cands[r->levels] = 0;
        r->edges_scanned[r->levels] = (i64)passes * nnz;
        r->levels++;
        for (i32 v = 0; v < n0; v++) r->final_labels[v] = id[r->final_labels[v]];
        i32 *rp2 = (i32 *)malloc(((size_t)K + 1) * sizeof(i32));
        i32 *col2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 *w2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 nnz2 = orc_aggregate(n, rp, col, w, id, K, rp2, col2, w2);
        free(rp); free(col); free(w);
        rp = rp2; col = col2; w = w2; n = K; nnz = nnz2;
        t++;
        if (t >= max_levels) { r->level_limit_hit = 1; break; }
    }
    free(rp); free(col); free(w);
    return r;
}

/* ========================================================================= */
/* Colour-synchronous Louvain: the parallel form of classical Louvain that   */
/* the conclusion (Section 6) leaves for later work, in the usual form of    */
/* parallel Louvain codes: the nodes of one colour class of a distance-1     */
/* colouring share no edge, so their moves are decided together.             */
/*                                                                           */
/* Colouring (readings; the paper gives none): at level t node v has the     */
/* key mix64(seed ^ mix64((t << 32) | v)); u precedes v when key(u) > key(v),*/
/* or the keys are equal and u < v.  Nodes are coloured one at a time in that */
/* order, each with the smallest colour held by none of its neighbours       */
/* already coloured (first fit; self-loops do not count).                   */
/*                                                                           */
/* A pass visits the colours 0, 1, ... in turn; every node of the colour    */
/* decides its move exactly as orc_louvain does, but all of them against    */
/* the communities and totals as they stand when the colour's turn begins,  */
/* and then all of them move at once.  Moves taken together can undo one    */
/* another's gains (two nodes joining one community each count its total    */
/* without the other), so passes need not settle; as parallel Louvain codes */
/* do, the level ends at a pass that moves no node (status 0), or that      */
/* raises the exact numerator sum_C (m_w W_in(C) - Sigma_C^2) by at most    */
/* floor(m_w^2 / 2^20), i.e. Q by at most 2^-20 (status 1), or after        */
/* max_passes passes (status 2).  Levels then compact, aggregate and stop   */
/* as in orc_louvain; the trace holds (level, pass, 0, 0, moves, 0).        */
/* ========================================================================= */
static u64 colour_key(u64 seed, i32 t, i32 v) {
    return orc_mix64(seed ^ orc_mix64(((u64)(uint32_t)t << 32) | (u64)(uint32_t)v));
}

/* Colours of the n nodes at level t (first fit in key order); returns the
 * number of colours. */
i32 orc_colour(i32 n, const i32 *rp, const i32 *col, u64 seed, i32 t, i32 *colour) {
    if (n <= 0) return 0;
    u64 *key = (u64 *)malloc((size_t)n * sizeof(u64));
    i32 *ord = (i32 *)malloc((size_t)n * sizeof(i32));
    i32 *used = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    for (i32 v = 0; v < n; v++) {
        key[v] = colour_key(seed, t, v);
        ord[v] = v;
        colour[v] = -1;
        used[v] = -1;
    }
    used[n] = -1;
    /* the key order: bottom-up merge sort on (key descending, id ascending) */
    i32 *tmp = (i32 *)malloc((size_t)n * sizeof(i32));
    for (i32 width = 1; width < n; width *= 2) {
        for (i32 lo = 0; lo < n; lo += 2 * width) {
            i32 mid = lo + width < n ? lo + width : n;
            i32 hi = lo + 2 * width < n ? lo + 2 * width : n;
            i32 a = lo, b = mid, o = lo;
            while (a < mid && b < hi) {
                i32 x = ord[a], y = ord[b];
                int x_first = key[x] > key[y] || (key[x] == key[y] && x < y);
                tmp[o++] = x_first ? ord[a++] : ord[b++];
            }
            while (a < mid) tmp[o++] = ord[a++];
            while (b < hi) tmp[o++] = ord[b++];
        }
        memcpy(ord, tmp, (size_t)n * sizeof(i32));
    }
    i32 ncol = 0;
    for (i32 k = 0; k < n; k++) {
        i32 v = ord[k];
        /* mark the colours of v's coloured neighbours with v's name */
        for (i32 p = rp[v]; p < rp[v + 1]; p++) {
            i32 u = col[p];
            if (u != v && colour[u] >= 0) used[colour[u]] = v;
        }
        i32 c = 0;
        while (used[c] == v) c++;
        colour[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(key); free(ord); free(used); free(tmp);
    return ncol;
}

orc_run *orc_louvain_colour(i32 n0, const i32 *rp0, const i32 *col0, const i32 *w0, u64 seed,
                            i32 max_passes, i32 max_levels) {
    orc_run *r = (orc_run *)calloc(1, sizeof(orc_run));
    r->n0 = n0;
    r->final_labels = (i32 *)malloc(((size_t)n0 + 1) * sizeof(i32));
    for (i32 v = 0; v < n0; v++) r->final_labels[v] = v;
    i32 n = n0;
    i32 nnz = rp0[n0];
    i32 *rp = (i32 *)malloc(((size_t)n + 1) * sizeof(i32));
    i32 *col = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    i32 *w = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
    memcpy(rp, rp0, ((size_t)n + 1) * sizeof(i32));
    memcpy(col, col0, (size_t)nnz * sizeof(i32));
    memcpy(w, w0, (size_t)nnz * sizeof(i32));
    i32 t = 0;
    for (;;) {
        size_t N = (size_t)n + 1;
        i64 *s = (i64 *)malloc(N * sizeof(i64));
        i64 *sigma = (i64 *)calloc(N, sizeof(i64));
        i64 *acc = (i64 *)calloc(N, sizeof(i64));
        i32 *touched = (i32 *)malloc(N * sizeof(i32));
        i32 *comm = (i32 *)malloc(N * sizeof(i32));
        i32 *colour = (i32 *)malloc(N * sizeof(i32));
        i32 *dest = (i32 *)malloc(N * sizeof(i32));
        unsigned char *seen = (unsigned char *)calloc(N, 1);
        i64 m = orc_strengths(n, rp, col, w, s);
        for (i32 v = 0; v < n; v++) { comm[v] = v; sigma[v] = s[v]; }
        i32 ncol = orc_colour(n, rp, col, seed, t, colour);
        i32 passes = 0;
        i64 lv_moves = 0, first_moves = 0;
        int status = 2;
        const i64 theta = (i64)(((unsigned __int128)m * (unsigned __int128)m) >> 20);
        i64 num = orc_modularity_num(n, rp, col, w, comm); /* singletons */
        while (passes < max_passes) {
            i64 moves = 0;
            for (i32 k = 0; k < ncol; k++) {
                /* every node of colour k decides on the same state ... */
                for (i32 i = 0; i < n; i++) {
                    dest[i] = -1;
                    if (colour[i] != k) continue;
                    i32 A = comm[i], nt = 0;
                    for (i32 p = rp[i]; p < rp[i + 1]; p++) {
                        i32 j = col[p];
                        if (j == i) continue;
                        i32 c = comm[j];
                        if (!seen[c]) { seen[c] = 1; touched[nt++] = c; }
                        acc[c] += w[p];
                    }
                    i64 stay = m * acc[A] - s[i] * (sigma[A] - s[i]);
                    i32 bc = -1;
                    i64 bd = 0;
                    for (i32 q = 0; q < nt; q++) {
                        i32 c = touched[q];
                        if (c == A) continue;
                        i64 d = (m * acc[c] - s[i] * sigma[c]) - stay;
                        if (d > 0 && (bc < 0 || d > bd || (d == bd && c < bc))) { bc = c; bd = d; }
                    }
                    for (i32 q = 0; q < nt; q++) { acc[touched[q]] = 0; seen[touched[q]] = 0; }
                    dest[i] = bc;
                }
                /* ... and then all of them move at once */
                for (i32 i = 0; i < n; i++) {
                    if (dest[i] < 0) continue;
                    sigma[comm[i]] -= s[i];
                    sigma[dest[i]] += s[i];
                    comm[i] = dest[i];
                    moves++;
                }
            }
            passes++;
            lv_moves += moves;
            if (passes == 1) first_moves = moves;
            trace_push(r, t, passes - 1, 0, 0, moves, 0);
            if (moves == 0) { status = 0; break; }
            const i64 num2 = orc_modularity_num(n, rp, col, w, comm);
            const i64 gain = num2 - num;
            num = num2;
            if (gain <= theta) { status = 1; break; }
        }
        i32 *id = (i32 *)malloc(N * sizeof(i32));
        i32 *rank = (i32 *)malloc(N * sizeof(i32));
        for (i32 v = 0; v < n; v++) rank[v] = -1;
        for (i32 v = 0; v < n; v++) rank[comm[v]] = 0;
        i32 K = 0;
        for (i32 v = 0; v < n; v++) if (rank[v] == 0) rank[v] = ++K;
        for (i32 v = 0; v < n; v++) id[v] = rank[comm[v]] - 1;
        free(rank); free(s); free(sigma); free(acc); free(touched); free(comm); free(seen);
        free(colour); free(dest);
        if (first_moves == 0 || K == n) {
            r->top_status = status;
            r->top_sweeps = passes;
            free(id);
            break;
        }
        run_grow(r);
        r->level_n[r->levels] = n;
        r->level_K[r->levels] = K;
        r->level_labels[r->levels] = id;
        r->sweeps[r->levels] = passes;
        r->status[r->levels] = status;
        r->moves[r->levels] = lv_moves;
        r->splits[r->levels] = 0;
        r->cands[r->levels] = 0;
        r->edges_scanned[r->levels] = (i64)passes * nnz;
        r->levels++;
        for (i32 v = 0; v < n0; v++) r->final_labels[v] = id[r->final_labels[v]];
        i32 *rp2 = (i32 *)malloc(((size_t)K + 1) * sizeof(i32));
        i32 *col2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 *w2 = (i32 *)malloc(((size_t)nnz + 1) * sizeof(i32));
        i32 nnz2 = orc_aggregate(n, rp, col, w, id, K, rp2, col2, w2);
        free(rp); free(col); free(w);
        rp = rp2; col = col2; w = w2; n = K; nnz = nnz2;
        t++;
        if (t >= max_levels) { r->level_limit_hit = 1; break; }
    }
    free(rp); free(col); free(w);
    return r;
}
