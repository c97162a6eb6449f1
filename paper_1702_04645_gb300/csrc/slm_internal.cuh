// slm_internal.cuh -- declarations shared by the CUDA translation units of the
// Synchronised Louvain Method library (sm_103a).
//
// Integer conventions: node ids, strengths s_i, community totals Sigma_C and
// every edge weight fit in int32 because m_w < 2^31; every product of two of
// them, and every gain, is computed in int64 and is exact.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <initializer_list>
#include <string>
#include <utility>
#include <vector>

#include "slm.h"

namespace slm {

// ---------------------------------------------------------------------------
// Errors: internal code throws slm::Error; the C ABI turns it into a status.
// ---------------------------------------------------------------------------
struct Error {
    slm_status status;
    std::string msg;
};

[[noreturn]] void fail(slm_status st, const std::string &msg);
unsigned long long launch_count();
// message returned by slm_last_error(NULL) on this thread
void set_global_error(const std::string &msg);
void check_cuda(cudaError_t e, const char *what, const char *file, int line);

// Every kernel launch of the library is followed by SLM_LAUNCH_CHECK(), which
// also counts it (the count is reported by slm_launch_count()).
void note_launch();
#define SLM_CUDA(call) ::slm::check_cuda((call), #call, __FILE__, __LINE__)
#define SLM_LAUNCH_CHECK()   \
    do {                     \
        ::slm::note_launch(); \
        ::slm::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); \
    } while (0)

constexpr int kWarp = 32;
constexpr int kNumSMs = 152;

// m_w of the graph a node belongs to: one value for a single graph, or per
// graph through the node -> graph map of a forest of graphs.
struct MParam {
    long long m = 0;
    const int32_t *gid = nullptr;
    const long long *mg = nullptr;
    __host__ __device__ MParam(long long v = 0) : m(v) {}
    __host__ __device__ MParam(const int32_t *g, const long long *per_graph) : gid(g), mg(per_graph) {}
    __device__ __forceinline__ long long of(int i) const { return gid ? mg[gid[i]] : m; }
};

// Key of the random acceptance draw: the seed and node id of a single graph,
// or per graph (seed of the node's graph, id local to that graph).
struct RngParam {
    unsigned long long seed = 0;
    const int32_t *gid = nullptr;
    const unsigned long long *seeds = nullptr;
    const int32_t *goff = nullptr;
    __host__ __device__ RngParam(unsigned long long s = 0) : seed(s) {}
    __device__ __forceinline__ unsigned long long seed_of(int i) const { return gid ? seeds[gid[i]] : seed; }
    __device__ __forceinline__ int local(int i) const { return gid ? i - goff[gid[i]] : i; }
};

// Null model of the modularity (Section 2.4, Q_w).  Every gain is
// m_w (weight term) minus null-model products of a strength and a total.
//  * NMSym, undirected graphs: one strength s_i per node (int32), totals
//    Sigma_C = sum of s, and a product is s * Sigma.
//  * NMDir, directed graphs: the scans read U = W + W^T, and a node carries
//    (s_i^out, s_i^in), a community (Sigma^out, Sigma^in), packed in one
//    64-bit word as out << 32 | in (each below 2^30).  The product of two
//    packed pairs is a^out b^in + a^in b^out.  Packed sums and differences
//    are plain 64-bit arithmetic whenever no component goes negative, which
//    holds for every sum of strengths and for the difference of a set's total
//    and a subset's; expressions whose components may be negative are
//    expanded into products of such terms instead.
// Every value then equals the exact change of the numerator, in NMDir twice
// what NMSym gives on a symmetric graph, so the decisions are the same.
struct NMSym {
    using ST = int32_t;  // stored strength or community total
    using V = int32_t;   // the same held in registers by the scan kernels
    static constexpr bool kDirected = false;
    static constexpr int kDiv = 1;  // numerator = sum_C (m W_in - cross(S, S)) / kDiv
    __host__ __device__ static long long cross(long long a, long long b) { return a * b; }
};
struct NMDir {
    using ST = unsigned long long;
    using V = long long;
    static constexpr bool kDirected = true;
    static constexpr int kDiv = 2;  // U counts every internal arc twice
    __host__ __device__ static long long cross(long long a, long long b) {
        const unsigned long long ua = (unsigned long long)a, ub = (unsigned long long)b;
        return (long long)(ua >> 32) * (long long)(ub & 0xffffffffull) +
               (long long)(ua & 0xffffffffull) * (long long)(ub >> 32);
    }
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
inline int grid_for(long long n, int block, int max_blocks = 152 * 32) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

// ---------------------------------------------------------------------------
// Stream-ordered device buffers (cudaMallocAsync / cudaFreeAsync).
// ---------------------------------------------------------------------------
// Host wait for the work queued on a stream.  By default the calling thread
// spins (lowest latency); a thread that set blocking waits sleeps on an event
// instead, leaving its core to other threads (the request server's slots).
void stream_sync(cudaStream_t st);
void set_thread_blocking_sync(bool on);

// Device memory comes from one memory pool per device owned by the library;
// freed blocks stay in the pool for the next allocation (no unmapping at each
// synchronisation) until trim_pool() returns them.
cudaMemPool_t lib_pool();
void trim_pool();

// While a ReleaseOnDefaultStream is alive on a thread, device buffers
// released by that thread are freed in order on the legacy default stream
// rather than on the stream that allocated them (which the caller may have
// destroyed).  Handles are destroyed this way: every entry point has
// finished its device work before it returns, so nothing still uses them.
struct ReleaseOnDefaultStream {
    ReleaseOnDefaultStream();
    ~ReleaseOnDefaultStream();
    bool prev;
};

// Byte count of the device buffers allocated while an accountant is current
// on the allocating thread (the request server measures each run with one).
struct MemAcct {
    long long cur = 0, peak = 0;  // updated under the accountant's own lock
    void add(long long b);
};
// the accountant of this thread (nullptr: none); returns the previous one
MemAcct *set_thread_acct(MemAcct *a);

// Test hook behind slm_debug_fail_allocation: the k-th device allocation
// from now on fails as if the device were out of memory (k = 0: off).
void set_alloc_failure(long long k);

// Host-side control of a run (the request server's cancellation and
// deadlines).  While a RunControl is installed on a thread, every run made on
// that thread checks it before each level and each sweep and stops with
// SLM_ERR_CANCELLED (cancel flag set) or SLM_ERR_DEADLINE (steady clock past
// the deadline).  Device work already queued finishes; nothing is abandoned
// in flight.
struct RunControl {
    const std::atomic<int> *cancel = nullptr;
    double deadline = 0;  // seconds of steady_seconds(); 0 = none
};
RunControl *set_thread_run_control(RunControl *c);  // returns the previous one
void check_run_control();
double steady_seconds();

class DevBuf {
  public:
    DevBuf() = default;
    DevBuf(size_t bytes, cudaStream_t s) { alloc(bytes, s); }
    ~DevBuf() { release(); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept { swap(o); }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); swap(o); }
        return *this;
    }
    void alloc(size_t bytes, cudaStream_t s);
    // grow-only: keeps the allocation when it is already large enough
    void ensure(size_t bytes, cudaStream_t s) {
        if (bytes > bytes_) alloc(bytes, s);
    }
    void release();
    template <class T> T *as() const { return static_cast<T *>(p_); }
    size_t bytes() const { return bytes_; }
    void *get() const { return p_; }

  private:
    void swap(DevBuf &o) {
        std::swap(p_, o.p_);
        std::swap(bytes_, o.bytes_);
        std::swap(s_, o.s_);
        std::swap(acct_, o.acct_);
    }
    void *p_ = nullptr;
    size_t bytes_ = 0;
    cudaStream_t s_ = nullptr;
    MemAcct *acct_ = nullptr;
};

// Cooperative launches (kernels whose blocks wait for one another at grid
// barriers) are ordered one after the other on the device, whatever stream
// they come from: two of them resident at once could each hold part of the
// GPU while waiting for the rest.  serialised_cooperative() makes `st` wait
// for the end of the previous cooperative launch of this device, runs
// `enqueue` (which launches on `st`) and records its end.
void coop_before(cudaStream_t st);
void coop_after(cudaStream_t st);
template <class F> void serialised_cooperative(cudaStream_t st, F &&enqueue) {
    coop_before(st);
    try {
        enqueue();
    } catch (...) {
        coop_after(st);
        throw;
    }
    coop_after(st);
}

// Small pinned host buffer for the counters read back each sweep (one per
// thread, shared by the runs made on that thread one after the other).
struct HostCounters {
    long long *h = nullptr;
    HostCounters();
    ~HostCounters();
};

// ---------------------------------------------------------------------------
// Device-wide primitives (k_basic.cu, k_sort.cu)
// ---------------------------------------------------------------------------
// Exclusive prefix sum of n int32 values (in may equal out); *total_dev (may
// be null) receives the sum.  All partial sums must stay below 2^31.
void exclusive_scan_i32(const int32_t *in, int32_t *out, long long n, int32_t *total_dev,
                        cudaStream_t s);
// Exclusive prefix sum of n int64 values.
void exclusive_scan_i64(const long long *in, long long *out, long long n, long long *total_dev,
                        cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
// keys/vals are sorted in place (the tmp buffers must hold n entries each).
void radix_sort_u64(unsigned long long *keys, int32_t *vals, unsigned long long *keys_tmp,
                    int32_t *vals_tmp, long long n, int bits, cudaStream_t s);
void radix_sort_u32(uint32_t *keys, int32_t *vals, uint32_t *keys_tmp, int32_t *vals_tmp,
                    long long n, int bits, cudaStream_t s);

// ---------------------------------------------------------------------------
// Graph-level kernels (k_basic.cu)
// ---------------------------------------------------------------------------
// Validation of a CSR: returns a bit mask of problems (1 bad column/order,
// 2 non-positive weight, 4 not symmetric, 8 bad row_ptr).
int validate_csr(int32_t n, long long nnz, const int32_t *rp, const int32_t *col, const int32_t *w,
                 cudaStream_t s);
// Number of the cnt entries of x outside [0, n) (host-synchronous).
int count_out_of_range(long long cnt, const int32_t *x, int32_t n, cudaStream_t s);
// s_i = sum_j W_ij (int32) and m_w (returned, int64).
long long strengths(int32_t n, const int32_t *rp, const int32_t *w, int32_t *s_out,
                    cudaStream_t s);
// Sigma[C] = sum of s over root == C (Sigma zeroed here).
void community_sigma(int32_t n, const int32_t *root, const int32_t *s, int32_t *sigma,
                     cudaStream_t st);
// The same for packed (out, in) strengths of a directed graph.
void community_sigma(int32_t n, const int32_t *root, const unsigned long long *s,
                     unsigned long long *sigma, cudaStream_t st);
// out[id[v]] += s[v] for packed strengths (out zeroed here): the strengths of
// the next level of a directed graph.
void sum_strengths_by(int32_t n, const int32_t *id, const unsigned long long *s, int32_t K,
                      unsigned long long *out, cudaStream_t st);
// id[v] = rank of root[v] among names in use; returns K (host-synchronous).
int32_t compact_labels(int32_t n, const int32_t *root, int32_t *id, int32_t *scratch_n,
                       cudaStream_t s);
// comp[v] = id[comp[v]]
void compose_labels(int32_t n0, int32_t *comp, const int32_t *id, cudaStream_t s);
// exact modularity numerator of labels (values in [0, n)); host-synchronous.
long long modularity_num(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                         const int32_t *labels, long long m_w, cudaStream_t s);
// The same on a directed graph given as U = W + W^T with packed strengths:
// sum_C (m_w U_in(C) - 2 Sigma_C^out Sigma_C^in) / 2.
long long modularity_num_directed(int32_t n, const int32_t *rp, const int32_t *col,
                                  const int32_t *w, const unsigned long long *s2,
                                  const int32_t *labels, long long m_w, cudaStream_t s);
double modularity_from_num(long long num, long long m_w);

// ---------------------------------------------------------------------------
// Degree buckets and the neighbourhood scans (k_scan.cu)
// ---------------------------------------------------------------------------
enum { kBucketEmpty = 0, kBucketG4, kBucketG8, kBucketG16, kBucketG32, kBucketWarpHash,
       kBucketBlockS, kBucketBlockM, kBucketBlockL, kBucketHub, kNumBuckets };
constexpr int kWarpHashMaxDeg = 256;
constexpr int kBlockSmallMaxDeg = 1024; // block shape with a 16 KB table up to here
constexpr int kBlockMidMaxDeg = 2048;   // block shape with a 32 KB table up to here
constexpr int kBlockSmemMaxDeg = 4096;  // block shape with a 64 KB table up to here; above: hub
constexpr int kHubChunk = 2048;         // edges of a hub handled by one block

// Fine degree classes: the launch shapes of the MAXIMAL scan.  The nodes are
// sorted by fine class, and every coarse bucket above is a contiguous run of
// fine classes (G4 = F4, G8 = F8, G16 = F16, G32 = F32, WarpHash = F64..F256,
// BlockS = F512..F1024, BlockM = F2048, BlockL = F4096, Hub = FHub).
enum { kFineEmpty = 0, kFine4, kFine8, kFine16, kFine32, kFine64, kFine128, kFine256, kFine512,
       kFine1024, kFine2048, kFine4096, kFineHub, kNumFine };

// Launch shapes of the MAXIMAL scan (results never depend on them): the
// number of streams the degree buckets run on (1 or 4) and, per kernel
// shape, the largest grid as blocks per SM.  Process-wide; set by
// slm_set_scan_tuning (for instance from the autotuner).
struct ScanTuning {
    int streams = 4;
    int blocks_large = 3;   // 2049..4096 edges, 64 KB table
    int blocks_mid = 6;     // 1025..2048 edges, 32 KB table
    int blocks_small = 8;   // 257..1024 edges, 16 KB table
    int blocks_warp = 8;    // 33..256 edges, warp tables
    int blocks_hub = 8;     // hub chunks and table slices
    int blocks_group = 16;  // 1..32 edges, lane groups
    int shape_alt = 0;      // bit f-1: the second launch shape of fine class f
};
ScanTuning scan_tuning();
void set_scan_tuning(const ScanTuning &t);

struct Buckets {
    DevBuf order;                       // int32[n]: nodes sorted by fine class (stable)
    int32_t off[kNumBuckets + 1] = {0}; // host copy of bucket offsets
    int32_t foff[kNumFine + 1] = {0};   // host copy of fine class offsets
    // The scan's own copy of the level graph, built on first use by
    // scan_nodes and kept until the next build: the rows of the bucketed
    // nodes in bucket order as packed (column, weight) pairs, one record
    // (node, first entry, degree, strength) per bucketed node in bucket
    // order, and per node of the graph (community, community total),
    // refreshed by every scan.
    DevBuf ent, nrec, cs;
    // when set, the (community, total) array lives there instead of in cs, so
    // that the layouts of several node lists of one graph share it
    DevBuf *cs_shared = nullptr;
    DevBuf &csbuf() { return cs_shared ? *cs_shared : cs; }
    const DevBuf &csbuf() const { return cs_shared ? *cs_shared : cs; }
    // no side streams: every kernel of a scan runs on the caller's stream
    bool one_stream = false;
    cudaTextureObject_t cs_tex = 0;  // cs through the texture path (0: plain loads)
    int cs_elem = 0;                 // bytes of one cs element the texture object was made for
    const void *lay_src[4] = {nullptr, nullptr, nullptr, nullptr};  // rp, col, w, s of the copy
    bool lay_ready = false;
    // hubs: per hub its global table (offset, log2 capacity), and the chunks
    // (hub index, first edge, end edge) that split its row across blocks
    int32_t nhub = 0, nchunk = 0, ntchunk = 0;
    // tslot: 64-bit slots (community + 1) << 32 | weight, 0 = empty; hub_own:
    // each hub's weight to its own community during a scan; hub_acc: the same
    // for the own-weight pass
    DevBuf hub_off, hub_lg, chunks, tslot, hub_acc, hub_own;
    // per hub: its list of occupied table slots (offset, count), so that the
    // decision reads the distinct communities only
    DevBuf hub_uoff, hub_ucnt, ulist;
    // slices of the hubs' slot lists read by one block each, and their partial results
    DevBuf tchunks, tc_off, part_sc, part_cc;
    // side streams on which the independent bucket kernels of a scan overlap
    // (owned here so that concurrent runs never share fork/join events)
    static constexpr int kSide = 3;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
    // optional per-bucket timing of the scans (milliseconds added to
    // prof_ms[bucket]; events recorded on the bucket's stream)
    double *prof_ms = nullptr;
    cudaEvent_t pev[kNumBuckets][2] = {};
    void build(int32_t n, const int32_t *rp, cudaStream_t s);
    // the same over the n listed nodes only (the scans then cover those nodes)
    void build_list(int32_t n, const int32_t *list, const int32_t *rp, cudaStream_t s);
    Buckets() = default;
    Buckets(const Buckets &) = delete;
    Buckets &operator=(const Buckets &) = delete;
    ~Buckets();
};

// Every function below that takes strengths s and totals sigma exists for
// both null models (NM = NMSym or NMDir, whose stored type is NM::ST); for a
// directed graph rp/col/w are U = W + W^T.
//
// The scan's copy of the level graph (Buckets::ent, nrec), built when the
// buckets changed or the graph is another one; cs is sized for n nodes.
template <class NM>
void build_scan_layout(Buckets &bk, int32_t n, const int32_t *rp, const int32_t *col,
                       const int32_t *w, const typename NM::ST *s, cudaStream_t st);
// cs[v] = (root_v, sigma[root_v]) for v < n.
template <class NM>
void pack_community_totals(int32_t n, const int32_t *root, const typename NM::ST *sigma,
                           Buckets &bk, cudaStream_t st);
// The MAXIMAL scan of the nodes of fine class f (kFine4 .. kFine4096) on the
// layout and community totals above (k_scan_fine.cu).
template <class NM>
void scan_fine_class(int f, const Buckets &bk, const typename NM::ST *s, MParam mp, int32_t *best,
                     long long *gain, int32_t *kown, unsigned long long *ncand,
                     const ScanTuning &tu, cudaStream_t so);

// ASSIGN: a[i] = best neighbour by m_w W_ij - s_i s_j (the null model's product).
template <class NM>
void assign_nodes(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                  const typename NM::ST *s, MParam m_w, const Buckets &bk, int32_t *a,
                  cudaStream_t st);

// The MAXIMAL scan: best community, gain (int64) and own-community weight
// kown (int32); counts candidates into *ncand_dev (unsigned long long).
template <class NM>
void scan_nodes(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                const typename NM::ST *s, MParam m_w, const int32_t *root,
                const typename NM::ST *sigma, const Buckets &bk, int32_t *best, long long *gain,
                int32_t *kown, unsigned long long *ncand_dev, cudaStream_t st);

// Own-community weight only (kown) for POSITIVE's local gains; flags the
// communities holding a node with g < 0 (flag[root] = 1) and counts them.
template <class NM>
void own_weight_nodes(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                      const typename NM::ST *s, MParam m_w, const int32_t *root,
                      const typename NM::ST *sigma, const Buckets &bk, int32_t *kown,
                      int32_t *flag, cudaStream_t st);

// Local gain g(i) = m_w kown_i - s_i (Sigma_{root_i} - s_i) of Algorithm POSITIVE.
template <class NM>
void local_gain_nodes(int32_t n, const typename NM::ST *s, MParam m, const int32_t *root,
                      const typename NM::ST *sigma, const int32_t *kown, long long *g,
                      cudaStream_t st);

// Target node for the accepted nodes listed in list[0..cnt).
template <class NM>
void target_nodes(const int32_t *list, const int32_t *cnt_dev, int32_t max_cnt,
                  const int32_t *rp, const int32_t *col, const int32_t *w,
                  const typename NM::ST *s, MParam m_w, const int32_t *root, const int32_t *best,
                  int32_t *tgt, cudaStream_t st);

// ---------------------------------------------------------------------------
// Assignment-forest kernels (k_forest.cu)
// ---------------------------------------------------------------------------
struct Forest {
    // per node
    int32_t *root = nullptr;    // smallest node on the reached cycle
    uint8_t *oncycle = nullptr; // 1 for cycle nodes
    int32_t *entry = nullptr;   // first cycle node on the forward path (self on cycle)
    int32_t *depth = nullptr;   // distance to entry
    int32_t *cdist = nullptr;   // for cycle nodes: forward distance to root
    // scratch
    int2 *jmpA = nullptr, *jmpB = nullptr;
};
// Components, cycle flags, entry, depth and cycle distances of a.
void forest_analyse(int32_t n, const int32_t *a, Forest &f, cudaStream_t st);
// The same for the cnt listed nodes only: the list must be closed under a
// (the forward path of a listed node stays in the list); the other nodes'
// values are left as they are.
void forest_analyse_subset(int32_t cnt, const int32_t *list, const int32_t *a, Forest &f,
                           cudaStream_t st);

struct BranchScratch {
    int32_t *haschild, *active, *covered, *treeact, *commcyc;
    long long *subS, *subWA, *subWin, *credit, *WB;
};
// Branch gains bg for candidates (gain > 0); counts positive ones and the
// accepted ones, and lists the accepted nodes.
template <class NM>
void branch_gains(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                  const typename NM::ST *s, MParam m_w, const int32_t *a, const Forest &f,
                  const typename NM::ST *sigma, const int32_t *best, const long long *gain,
                  const int32_t *kown, BranchScratch &bs, long long *bg, cudaStream_t st);
// Acceptance draw and list of accepted nodes.
// With a forest (rng.gid set), per_graph gets, for every graph, the counts
// of positive branch gains [0] and accepted moves [1] (int32 pairs), and
// nodes of graphs whose active[g] is 0 are skipped.
void accept_moves(int32_t n, const long long *bg, RngParam rng, unsigned long long P,
                  int32_t level, int32_t sweep, int32_t *acc_list, int32_t *acc_cnt_dev,
                  unsigned long long *npos_dev, cudaStream_t st,
                  const int32_t *active = nullptr, int32_t *per_graph = nullptr);
void apply_moves(const int32_t *list, const int32_t *cnt_dev, int32_t max_cnt,
                 const int32_t *tgt, int32_t *a, cudaStream_t st);

// Phases of a POSITIVE round, for the optional profile: 0 round set-up,
// 1 offsets (prefix sums), 2 ancestor walks and edge credits, 3 subtree
// credits, 4 best cut, 5 cut application, 6 new components, 7 local gains,
// 8 next member list (nanoseconds); then two counts: 9 rounds run on the
// full grid, 10 member visits of those rounds.
constexpr int kPosPhases = 11;
struct PositiveScratch {
    DevBuf flag, kown, listA, listB, rlist, posr, L, coff, subS, subWA, subWin, credit, TS, msz,
        bestsc, bestkey, pool, pool2, cyc, cnt, mark, tot, hdr, epref, kacc, cut, nf, noc, bs, ctrl;
    DevBuf rowlen, ioff, istart, ideg, icol, iw;  // internal entries of the members (room: whole rows)
    DevBuf recomp, moffN, cutsum, coffN, freshN, cutpar, oldroot;  // incremental rounds
    DevBuf dirty;  // communities whose membership changed since the last call
    bool profile = false;              // stamp the phases of every round
    long long prof_ns[kPosPhases] = {};  // summed nanoseconds per phase
};
// Algorithm POSITIVE until no node has a negative local gain.  a and the
// forest f are updated in place (only the members of split communities are
// recomputed); sigma is used as scratch.  Returns the number of splits;
// *rounds_out gets the number of rounds and *visits_out the member visits
// summed over the rounds.
// With a forest, splits_per_graph (int32[G], may be null) counts each graph's splits.
// prev_root (may be null): the names after the last POSITIVE on this state;
// when given, only communities whose membership changed since are examined
// (the others cannot hold a negative local gain).
template <class NM>
long long positive_correct(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                           const typename NM::ST *s, MParam m, int32_t *a, Forest &f,
                           typename NM::ST *sigma,
                           const Buckets &bk, PositiveScratch &ps, cudaStream_t st,
                           long long *rounds_out, long long *visits_out,
                           int32_t *splits_per_graph = nullptr,
                           const int32_t *prev_root = nullptr);

// Nodes (listed in node order) of the communities flagged in flag[name],
// taken from the cnt listed nodes (list == nullptr: every node); returns the
// count (host-synchronous).  mark and tot are scratch.
int32_t compact_members(long long cnt, const int32_t *list, const int32_t *root,
                        const int32_t *flag, int32_t *out, DevBuf &mark, DevBuf &tot,
                        cudaStream_t st);
// Nodes of the communities that the last synchronous write touched (the old
// and the target community of every accepted node, names of `root` before
// the components are updated): a set closed under the new assignments.
// Returns the count (host-synchronous).
int32_t moved_members(int32_t n, const int32_t *acc, const int32_t *acc_cnt, int32_t max_acc,
                      const int32_t *root, const int32_t *best, int32_t *out, DevBuf &mark,
                      DevBuf &scratch, DevBuf &tot, cudaStream_t st);

// Self-check of the time-limited grid barrier of the cooperative kernels:
// `blocks` resident blocks pass three barriers; block `absent` (>= 0) leaves
// first, so the others give up after limit_ns.  True when every block passed.
bool barrier_check(int blocks, int absent, long long limit_ns, cudaStream_t st);

// ---------------------------------------------------------------------------
// Aggregation (k_sort.cu)
// ---------------------------------------------------------------------------
// Builds the aggregated CSR; returns its nnz.  Output buffers are allocated
// by the callee (row_ptr_out K+1, col_out/w_out nnz').
// With a forest, rows of the graphs marked in drop_graph (gid: node -> graph)
// are left out; `dropped` is their number of entries.
int32_t aggregate_graph(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                        const int32_t *id, int32_t K, DevBuf &rp_out, DevBuf &col_out,
                        DevBuf &w_out, cudaStream_t st, const int32_t *gid = nullptr,
                        const int32_t *drop_graph = nullptr, long long dropped = 0);

// ---------------------------------------------------------------------------
// Forests of graphs (k_basic.cu)
// ---------------------------------------------------------------------------
// gid[v] = the graph whose node range [goff[g], goff[g+1]) holds v.
void graph_of_nodes(int32_t n, const int32_t *goff, int32_t G, int32_t *gid, cudaStream_t st);
// per graph: m_w (int64) from the strengths; returns the number of entries
// whose endpoints lie in different graphs (host-synchronous).
long long forest_check_and_weights(int32_t n, const int32_t *rp, const int32_t *col,
                                   const int32_t *s, const int32_t *gid, int32_t G,
                                   long long *mg, cudaStream_t st);
// per graph: number of names in use (root[v] == v)
void roots_per_graph(int32_t n, const int32_t *root, const int32_t *gid, int32_t *Kg,
                     cudaStream_t st);
// per graph: candidates (gain > 0) of active graphs; gains of inactive graphs zeroed
void candidates_per_graph(int32_t n, const int32_t *gid, const int32_t *active, long long *gain,
                          int32_t *cand_g, cudaStream_t st);
// per graph exact modularity numerator of labels (global ids in [0, nlab)),
// labels of graph g lying in [loff[g], loff[g+1]); nums[g] = m_g sum W_in - sum Sigma^2
void modularity_forest(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                       const int32_t *labels, int32_t nlab, const int32_t *gid,
                       const int32_t *loff, int32_t G, const long long *mg, long long *nums,
                       cudaStream_t st);

// ---------------------------------------------------------------------------
// Colour-synchronous Louvain (k_louvain.cu)
// ---------------------------------------------------------------------------
// First-fit colouring of the n nodes in the key order of level `level`:
// colour[v], and order = the nodes sorted by colour (stable, so ascending
// within a class); returns the class offsets into order (ncolours + 1
// entries; host-synchronous).
std::vector<int32_t> colour_nodes(int32_t n, const int32_t *rp, const int32_t *col,
                                  unsigned long long seed, int32_t level, int32_t *colour,
                                  int32_t *order, cudaStream_t st);
// the longest row of the n-node graph (host-synchronous)
int32_t max_row_length(int32_t n, const int32_t *rp, cudaStream_t st);
// per colour class (colour[v] in [0, ncol)) its longest row (host-synchronous)
std::vector<int32_t> class_max_rows(int32_t n, const int32_t *rp, const int32_t *colour, int32_t ncol,
                                    cudaStream_t st);
// The MAXIMAL scan's decision (best[i]) for the cnt listed nodes, one block
// per node with a shared-memory table: for graphs whose rows have at most
// kLouvainDecideMaxRow entries (the table holds 2^kLouvainDecideMaxLg slots).
constexpr int kLouvainDecideMaxLg = 14;
constexpr int32_t kLouvainDecideMaxRow = 1 << (kLouvainDecideMaxLg - 1);
void louvain_decide(const int32_t *list, int32_t cnt, const int32_t *rp, const int32_t *col,
                    const int32_t *w, const int32_t *s, long long m, const int32_t *comm,
                    const int32_t *sigma, int32_t max_row, int32_t *best, cudaStream_t st);
// comm[v] = v, sigma[v] = s[v]
void louvain_init(int32_t n, const int32_t *s, int32_t *comm, int32_t *sigma, cudaStream_t st);
// the moves of the cnt listed nodes (best[i] != comm[i]), with their totals;
// *moves += their number
void louvain_move(const int32_t *list, int32_t cnt, const int32_t *best, int32_t *comm,
                  const int32_t *s, int32_t *sigma, unsigned long long *moves, cudaStream_t st);
// id[v] = rank of comm[v] among the names in use (ascending); returns K
// (host-synchronous)
int32_t compact_names(int32_t n, const int32_t *comm, int32_t *id, int32_t *scratch_n,
                      cudaStream_t st);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
// Adds, for every lane with `pred`, one to ctr[g]: one atomic per distinct g
// in the warp.  Every lane of the warp must call it.
__device__ __forceinline__ void warp_count(int32_t *ctr, int g, bool pred) {
    const unsigned act = __ballot_sync(0xffffffffu, pred);
    if (pred) {
        const unsigned grp = __match_any_sync(act, g);
        if ((int)(threadIdx.x & 31) == __ffs((int)grp) - 1) atomicAdd(&ctr[g], __popc(grp));
    }
}

// splitmix64 output function (Steele, Lea, Flood 2014).
__host__ __device__ inline unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline unsigned int accept_draw(unsigned long long seed, int level, int sweep,
                                                    int node) {
    unsigned long long ctr = ((unsigned long long)(unsigned)level << 48) |
                             ((unsigned long long)(unsigned)sweep << 32) |
                             (unsigned long long)(unsigned)node;
    return (unsigned int)(mix64(seed ^ mix64(ctr)) >> 32);
}

}  // namespace slm
